// weno_api.cu -- the C ABI (include/weno_gb300.h): handles, scratch,
// argument checking and the launch sequences of a residual, a stage, a step
// and a CUDA-graph-captured run.  No arithmetic of the scheme lives here.
#include <algorithm>
#include <climits>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <string>
#include <vector>

#include "../../include/weno_gb300.h"
#include "weno_dev.cuh"
#include "weno_internal.h"
#include "cross_internal.h"
#include "tt_internal.h"

using namespace wg;

struct weno_ctx {
    int dim = 0, nf = 0;
    long long n[3] = {1, 1, 1};
    double h[3] = {1, 1, 1};
    long long N = 0;
    weno_params p{};
    cudaStream_t stream = nullptr;   // caller's stream
    cudaStream_t capture = nullptr;  // owned side stream used only for graph capture
    double *S1 = nullptr, *S2 = nullptr, *Udev = nullptr;
    void *acc = nullptr;
    double *partials = nullptr, *sums_dev = nullptr;
    int nblocks_sum = 0;
    Ctl *ctl = nullptr;
    Ctl *ctl_host = nullptr;  // pinned mirror for reads
    cudaGraphExec_t gexec = nullptr;
    const double *g_U = nullptr;
    int g_steps = 0;
    // cross-eval scratch
    void *xbuf = nullptr;
    size_t xbuf_bytes = 0;
    // cross-eval autotuning (workload class -> variant, CTAs per SM) and captured graphs
    std::map<std::string, std::pair<int, int>> tune;
    struct XGraph {
        uint64_t key;
        cudaGraphExec_t exec;
        void *buf;
        unsigned long long last;
    };
    std::vector<XGraph> xgraphs;
    unsigned long long xgraph_clock = 0;
    // TT-rounding scratch
    void *tbuf = nullptr;
    size_t tbuf_bytes = 0;
    // maxvol / TT-cross scratch
    void *mbuf = nullptr;
    size_t mbuf_bytes = 0;
    void *cbuf = nullptr;
    size_t cbuf_bytes = 0;
    // kernel timing (weno_profile_*)
    struct EvPair { cudaEvent_t a, b; int kind; };
    bool prof = false;
    bool capturing = false;
    std::vector<EvPair> pending;
    std::vector<cudaEvent_t> pool;
    double prof_ms[WENO_PROFILE_KINDS] = {};
    long long prof_n[WENO_PROFILE_KINDS] = {};
    long long launches = 0;
    long long g_kernels = 0;  // kernels per replay of the captured graph
    std::string err;
};

static cudaEvent_t get_event(weno_ctx *h)
{
    if (!h->pool.empty()) {
        cudaEvent_t e = h->pool.back();
        h->pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

// Every kernel launch of the API goes through here: it counts the launch and,
// when timing is on and the stream is not being captured, brackets it with a
// CUDA event pair on the launch stream.
template <class F> static cudaError_t launch(weno_ctx *h, int kind, cudaStream_t s, F &&f, int nk = 1)
{
    const bool rec = h->prof && !h->capturing;
    weno_ctx::EvPair ev{nullptr, nullptr, kind};
    if (rec) {
        ev.a = get_event(h);
        ev.b = get_event(h);
        cudaEventRecord(ev.a, s);
    }
    cudaError_t e = f();
    if (rec) {
        cudaEventRecord(ev.b, s);
        h->pending.push_back(ev);
    }
    if (h->capturing) h->g_kernels += nk;
    else h->launches += nk;
    return e;
}

static thread_local std::string g_init_error;

namespace wg {
// Error text for calls made without a handle (read back by weno_last_error(NULL)).
void set_thread_error(const std::string &msg) { g_init_error = msg; }
}  // namespace wg

static int fail(weno_ctx *h, int code, const std::string &msg)
{
    if (h) h->err = msg;
    else g_init_error = msg;
    return code;
}

static int grow(weno_ctx *h, void **buf, size_t *have, size_t bytes);

#define CK(h, call)                                                                                 \
    do {                                                                                            \
        cudaError_t e_ = (call);                                                                    \
        if (e_ != cudaSuccess)                                                                      \
            return fail((h), WENO_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_));   \
    } while (0)

__global__ static void k_set_run(Ctl *c, double t_end, double dt_req, double cfl_h, long long max_steps)
{
    c->t_end = t_end;
    c->dt_req = dt_req;
    c->cfl_h = cfl_h;
    c->max_steps = (max_steps > LLONG_MAX - c->steps) ? LLONG_MAX : c->steps + max_steps;
}

__global__ static void k_set_time(Ctl *c, double t)
{
    c->t = t;
    c->t_next = t;
    c->steps = 0;
}

__global__ static void k_clear_status(Ctl *c) { c->status = 0; }

static void free_all(weno_ctx *h)
{
    if (h->gexec) cudaGraphExecDestroy(h->gexec);
    cudaFree(h->S1);
    cudaFree(h->S2);
    cudaFree(h->Udev);
    cudaFree(h->acc);
    cudaFree(h->partials);
    cudaFree(h->sums_dev);
    cudaFree(h->ctl);
    cudaFree(h->xbuf);
    for (auto &g : h->xgraphs) {
        cudaGraphExecDestroy(g.exec);
        cudaFree(g.buf);
    }
    cudaFree(h->tbuf);
    cudaFree(h->mbuf);
    cudaFree(h->cbuf);
    if (h->ctl_host) cudaFreeHost(h->ctl_host);
    if (h->capture) cudaStreamDestroy(h->capture);
    for (auto &ev : h->pending) {
        cudaEventDestroy(ev.a);
        cudaEventDestroy(ev.b);
    }
    for (auto e : h->pool) cudaEventDestroy(e);
}

static double min_h(const weno_ctx *h)
{
    double m = h->h[0];
    for (int d = 1; d < h->dim; ++d) m = h->h[d] < m ? h->h[d] : m;
    return m;
}

extern "C" int weno_init(weno_handle *out, const weno_grid *grid, const weno_params *params, void *cuda_stream)
{
    if (!out || !params) return fail(nullptr, WENO_ERR_ARG, "weno_init: null out or params");
    *out = nullptr;
    const weno_params &p = *params;
    if (!(p.gamma > 1.0) || !(p.eps_weno > 0.0) || !(p.cfl >= 0.0))
        return fail(nullptr, WENO_ERR_ARG, "weno_init: need gamma > 1, eps_weno > 0, cfl >= 0");
    if (p.precision != WENO_FP64 && p.precision != WENO_FP32_BULK)
        return fail(nullptr, WENO_ERR_ARG, "weno_init: bad precision");
    if (p.alpha_mode != WENO_ALPHA_GLOBAL_NORM && p.alpha_mode != WENO_ALPHA_PER_DIR)
        return fail(nullptr, WENO_ERR_ARG, "weno_init: bad alpha_mode");
    for (int d = 0; d < 3; ++d)
        for (int s = 0; s < 2; ++s)
            if (p.bc[d][s] < 0 || p.bc[d][s] > 3) return fail(nullptr, WENO_ERR_ARG, "weno_init: bad boundary rule");
    if (p.model < WENO_MODEL_EULER || p.model > WENO_MODEL_BURGERS)
        return fail(nullptr, WENO_ERR_ARG, "weno_init: bad model");
    if (p.model != WENO_MODEL_EULER && p.precision != WENO_FP64)
        return fail(nullptr, WENO_ERR_UNSUPPORTED, "weno_init: the scalar models run in FP64 only");
    weno_ctx *h = new weno_ctx();
    h->p = p;
    h->stream = (cudaStream_t)cuda_stream;
    if (grid) {
        if (grid->dim < 1 || grid->dim > 3) {
            delete h;
            return fail(nullptr, WENO_ERR_ARG, "weno_init: dim must be 1, 2 or 3");
        }
        h->dim = grid->dim;
        h->nf = p.model == WENO_MODEL_EULER ? grid->dim + 2 : 1;
        h->N = 1;
        for (int d = 0; d < 3; ++d) {
            const long long nd = d < grid->dim ? grid->n[d] : 1;
            if (d < grid->dim && (nd < 3 || nd > (1ll << 30) || !(grid->hi[d] > grid->lo[d]))) {
                delete h;
                return fail(nullptr, WENO_ERR_ARG, "weno_init: need 3 <= n[d] and lo < hi on every used direction");
            }
            if (d >= grid->dim && grid->n[d] != 1 && grid->n[d] != 0) {
                delete h;
                return fail(nullptr, WENO_ERR_ARG, "weno_init: n[d] must be 1 beyond dim");
            }
            h->n[d] = nd;
            h->h[d] = d < grid->dim ? (grid->hi[d] - grid->lo[d]) / (double)nd : 1.0;
            h->N *= nd;
        }
        // launch-grid limits (y and z grid dimensions hold at most 65535 blocks)
        if ((h->dim == 2 && h->n[1] > 65535ll * 8) || (h->dim == 3 && (h->n[1] > 65535 || h->n[2] > 65535))) {
            delete h;
            return fail(nullptr, WENO_ERR_ARG, "weno_init: need ny <= 524280 (2D), ny, nz <= 65535 (3D)");
        }
        if (p.model != WENO_MODEL_EULER && h->dim == 2 && h->n[1] > 65535ll * 2) {
            delete h;
            return fail(nullptr, WENO_ERR_ARG, "weno_init: scalar models need ny <= 131070 (2D)");
        }
    }
    static bool attrs = false;
    if (!attrs) {
        cudaError_t e = sweep_set_attributes();
        if (e != cudaSuccess) {
            delete h;
            return fail(nullptr, WENO_ERR_CUDA, std::string("weno_init: kernel attributes: ") + cudaGetErrorString(e));
        }
        attrs = true;
    }
    auto alloc = [&](void **ptr, size_t bytes) -> bool {
        if (cudaMalloc(ptr, bytes) != cudaSuccess) {
            cudaGetLastError();
            return false;
        }
        return true;
    };
    bool ok = alloc((void **)&h->ctl, sizeof(Ctl)) && cudaMallocHost((void **)&h->ctl_host, sizeof(Ctl)) == cudaSuccess &&
              cudaStreamCreateWithFlags(&h->capture, cudaStreamNonBlocking) == cudaSuccess;
    if (ok && grid) {
        const size_t sb = sizeof(double) * (size_t)h->nf * (size_t)h->N;
        const size_t ab = (p.precision == WENO_FP32_BULK ? sizeof(float) : sizeof(double)) * (size_t)h->nf * (size_t)h->N;
        h->nblocks_sum = sums_blocks(h->N);
        ok = alloc((void **)&h->S1, sb) && alloc((void **)&h->S2, sb) && alloc(&h->acc, ab) &&
             alloc((void **)&h->partials, sizeof(double) * (size_t)h->nblocks_sum * h->nf) &&
             alloc((void **)&h->sums_dev, sizeof(double) * h->nf);
    }
    if (!ok) {
        free_all(h);
        delete h;
        return fail(nullptr, WENO_ERR_CUDA, "weno_init: device allocation failed");
    }
    Ctl c{};
    c.max_steps = LLONG_MAX;
    if (cudaMemcpyAsync(h->ctl, &c, sizeof(Ctl), cudaMemcpyHostToDevice, h->stream) != cudaSuccess ||
        cudaStreamSynchronize(h->stream) != cudaSuccess) {
        free_all(h);
        delete h;
        return fail(nullptr, WENO_ERR_CUDA, "weno_init: control block upload failed");
    }
    *out = h;
    return WENO_OK;
}

extern "C" int weno_destroy(weno_handle h)
{
    if (!h) return WENO_ERR_ARG;
    cudaStreamSynchronize(h->stream);
    free_all(h);
    delete h;
    return WENO_OK;
}

extern "C" int weno_set_stream(weno_handle h, void *cuda_stream)
{
    if (!h) return WENO_ERR_ARG;
    h->stream = (cudaStream_t)cuda_stream;
    return WENO_OK;
}

extern "C" const char *weno_last_error(weno_handle h) { return h ? h->err.c_str() : g_init_error.c_str(); }

static int need_grid(weno_ctx *h, const char *who)
{
    if (!h) return WENO_ERR_ARG;
    if (h->dim == 0) return fail(h, WENO_ERR_ARG, std::string(who) + ": handle has no grid");
    return WENO_OK;
}

static SweepArgs base_args(weno_ctx *h)
{
    SweepArgs a{};
    a.ctl = h->ctl;
    a.N = h->N;
    for (int d = 0; d < 3; ++d) {
        a.n[d] = (int)h->n[d];
        a.inv_h[d] = 1.0 / h->h[d];
        a.bc[d][0] = h->p.bc[d][0];
        a.bc[d][1] = h->p.bc[d][1];
        for (int sd = 0; sd < 2; ++sd)
            for (int f = 0; f < 5; ++f) a.bc_state[d][sd][f] = h->p.bc_state[d][sd][f];
    }
    a.stride[0] = 1;
    a.stride[1] = h->n[0];
    a.stride[2] = h->n[0] * h->n[1];
    a.gamma = h->p.gamma;
    a.eps = h->p.eps_weno;
    a.gamma_f = (float)h->p.gamma;
    a.gm1_f = (float)(h->p.gamma - 1.0);
    a.eps_f = (float)h->p.eps_weno;
    for (int d = 0; d < 3; ++d) a.inv_h_f[d] = (float)a.inv_h[d];
    a.acc = h->acc;
    // a scalar law has one wavespeed |f'(u)| for every direction
    a.per_dir = h->p.alpha_mode == WENO_ALPHA_PER_DIR && h->p.model == WENO_MODEL_EULER ? 1 : 0;
    return a;
}

static bool bulk(const weno_ctx *h) { return h->p.precision == WENO_FP32_BULK; }

// One residual evaluation; the last kernel runs epilogue `last`.
//   1D: the x sweep.  2D: the fused x+y tile kernel.  3D: the fused x+y kernel
//   per z-plane (stores), then the z kernel (adds, and runs `last`).
static int enqueue_sweeps(weno_ctx *h, SweepArgs a, int last, cudaStream_t s)
{
    if (h->p.model != WENO_MODEL_EULER) {  // scalar laws: one sweep per direction
        for (int d = 0; d < h->dim; ++d) {
            const int epi = d == h->dim - 1 ? last : (d == 0 ? EPI_STORE : EPI_ADD);
            CK(h, launch(h, 3, s, [&] { return launch_sweep(h->p.model, h->dim, d, false, epi, a, s); }));
        }
    } else if (h->dim == 1) {
        CK(h, launch(h, 3, s, [&] { return launch_sweep(MODEL_EULER, 1, 0, bulk(h), last, a, s); }));
    } else if (h->dim == 2) {
        CK(h, launch(h, 4, s, [&] { return launch_xy(2, bulk(h), last, a, s); }));
    } else {
        CK(h, launch(h, 2, s, [&] { return launch_xy(3, bulk(h), EPI_STORE, a, s); }));
        CK(h, launch(h, 5, s, [&] { return launch_z(bulk(h), last, a, s); }));
    }
    return WENO_OK;
}

// One SSP-RK3 step (Eq. tt-ssprk3 without rounding) on U in place; alpha(U^n)
// must be in slot 0.  Capturable: no host synchronisation.
static int enqueue_step(weno_ctx *h, double *U, cudaStream_t s)
{
    CK(h, launch(h, 7, s, [&] { return launch_step_begin(h->ctl, s); }));
    double *in[3] = {U, h->S1, h->S2};
    double *outs[3] = {h->S1, h->S2, U};
    for (int k = 0; k < 3; ++k) {
        SweepArgs a = base_args(h);
        a.U = in[k];
        a.Un = U;
        a.Uout = outs[k];
        a.stage = k;
        a.slot_in = k;
        a.slot_out = k + 1;
        a.check_dt = 1;
        int r = enqueue_sweeps(h, a, EPI_STAGE, s);
        if (r) return r;
    }
    CK(h, launch(h, 7, s, [&] { return launch_step_end(h->ctl, s); }));
    return WENO_OK;
}

static int enqueue_alpha0(weno_ctx *h, const double *U, cudaStream_t s)
{
    CK(h, launch(h, 7, s, [&] { return launch_reset_slot(h->ctl, 0, s); }));
    CK(h, launch(h, 6, s, [&] {
           return launch_alpha(h->p.model, h->dim, bulk(h), U, h->N, h->p.gamma, h->ctl, 0,
                               h->p.alpha_mode == WENO_ALPHA_PER_DIR && h->p.model == WENO_MODEL_EULER ? 1 : 0, s);
       }));
    return WENO_OK;
}

static int read_ctl(weno_ctx *h)
{
    CK(h, cudaMemcpyAsync(h->ctl_host, h->ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, h->stream));
    CK(h, cudaStreamSynchronize(h->stream));
    return WENO_OK;
}

static int take_status(weno_ctx *h)
{
    int r = read_ctl(h);
    if (r) return r;
    if (h->ctl_host->status & ST_BADINDEX) {
        CK(h, launch(h, 7, h->stream, [&] {
               k_clear_status<<<1, 1, 0, h->stream>>>(h->ctl);
               return cudaGetLastError();
           }));
        return fail(h, WENO_ERR_ARG, "weno_cross_eval: an index set held an index outside its mode (fiber skipped)");
    }
    if (h->ctl_host->status & ST_NONPHYSICAL) {
        CK(h, launch(h, 7, h->stream, [&] {
               k_clear_status<<<1, 1, 0, h->stream>>>(h->ctl);
               return cudaGetLastError();
           }));
        return fail(h, WENO_ERR_NONPHYSICAL, "device saw a non-physical state (NaN/Inf, rho <= 0 or p <= 0)");
    }
    return WENO_OK;
}

extern "C" int weno_alpha(weno_handle h, const double *U, double *alpha_dev)
{
    int r = need_grid(h, "weno_alpha");
    if (r) return r;
    if (!U || !alpha_dev) return fail(h, WENO_ERR_ARG, "weno_alpha: null pointer");
    if ((r = enqueue_alpha0(h, U, h->stream))) return r;
    CK(h, launch(h, 7, h->stream, [&] { return launch_copy_alpha(h->ctl, 0, alpha_dev, h->stream); }));
    return WENO_OK;
}

extern "C" int weno_rhs(weno_handle h, const double *U, double *R, double *alpha_dev)
{
    int r = need_grid(h, "weno_rhs");
    if (r) return r;
    if (!U || !R) return fail(h, WENO_ERR_ARG, "weno_rhs: null U or R");
    if (R == U) return fail(h, WENO_ERR_ARG, "weno_rhs: R must not alias U");
    if ((r = enqueue_alpha0(h, U, h->stream))) return r;
    SweepArgs a = base_args(h);
    a.U = U;
    a.Rout = R;
    a.slot_in = 0;
    a.check_dt = 0;
    if ((r = enqueue_sweeps(h, a, EPI_RHS, h->stream))) return r;
    if (alpha_dev) CK(h, launch(h, 7, h->stream, [&] { return launch_copy_alpha(h->ctl, 0, alpha_dev, h->stream); }));
    return WENO_OK;
}

extern "C" int weno_set_time(weno_handle h, double t)
{
    if (!h) return WENO_ERR_ARG;
    CK(h, launch(h, 7, h->stream, [&] {
           k_set_time<<<1, 1, 0, h->stream>>>(h->ctl, t);
           return cudaGetLastError();
       }));
    return WENO_OK;
}

extern "C" int weno_get_time(weno_handle h, double *t, int64_t *steps)
{
    if (!h) return WENO_ERR_ARG;
    int r = take_status(h);
    if (t) *t = h->ctl_host->t;
    if (steps) *steps = h->ctl_host->steps;
    return r;
}

extern "C" int weno_ssprk3_step(weno_handle h, double *U, double t_end, double dt)
{
    int r = need_grid(h, "weno_ssprk3_step");
    if (r) return r;
    if (!U) return fail(h, WENO_ERR_ARG, "weno_ssprk3_step: null U");
    if (dt <= 0.0 && !(h->p.cfl > 0.0)) return fail(h, WENO_ERR_ARG, "weno_ssprk3_step: dt <= 0 needs cfl > 0");
    CK(h, launch(h, 7, h->stream, [&] {
           k_set_run<<<1, 1, 0, h->stream>>>(h->ctl, t_end, dt, h->p.cfl * min_h(h), LLONG_MAX);
           return cudaGetLastError();
       }));
    if ((r = enqueue_alpha0(h, U, h->stream))) return r;
    return enqueue_step(h, U, h->stream);
}

static int ensure_graph(weno_ctx *h, double *U, int steps)
{
    if (h->gexec && h->g_U == U && h->g_steps == steps) return WENO_OK;
    if (h->gexec) {
        cudaGraphExecDestroy(h->gexec);
        h->gexec = nullptr;
    }
    cudaGraph_t g = nullptr;
    CK(h, cudaStreamBeginCapture(h->capture, cudaStreamCaptureModeThreadLocal));
    h->capturing = true;
    h->g_kernels = 0;
    int r = WENO_OK;
    for (int k = 0; k < steps && r == WENO_OK; ++k) r = enqueue_step(h, U, h->capture);
    h->capturing = false;
    cudaError_t e = cudaStreamEndCapture(h->capture, &g);
    if (r) {
        if (g) cudaGraphDestroy(g);
        return r;
    }
    if (e != cudaSuccess) return fail(h, WENO_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(e));
    e = cudaGraphInstantiate(&h->gexec, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return fail(h, WENO_ERR_CUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
    h->g_U = U;
    h->g_steps = steps;
    return WENO_OK;
}

extern "C" int weno_run(weno_handle h, double *U, double t_end, double dt, int64_t max_steps, int32_t graph_steps,
                        int64_t *steps_out)
{
    int r = need_grid(h, "weno_run");
    if (r) return r;
    if (!U || max_steps < 0) return fail(h, WENO_ERR_ARG, "weno_run: null U or negative max_steps");
    if (dt <= 0.0 && !(h->p.cfl > 0.0)) return fail(h, WENO_ERR_ARG, "weno_run: dt <= 0 needs cfl > 0");
    if (steps_out) *steps_out = 0;
    CK(h, launch(h, 7, h->stream, [&] {
           k_set_run<<<1, 1, 0, h->stream>>>(h->ctl, t_end, dt, h->p.cfl * min_h(h), max_steps);
           return cudaGetLastError();
       }));
    if ((r = enqueue_alpha0(h, U, h->stream))) return r;
    if ((r = read_ctl(h))) return r;
    const long long s0 = h->ctl_host->steps;
    const int chunk = graph_steps > 0 ? graph_steps : 8;
    if (graph_steps > 0 && (r = ensure_graph(h, U, graph_steps))) return r;
    for (;;) {
        if (graph_steps > 0) {
            CK(h, cudaGraphLaunch(h->gexec, h->stream));
            h->launches += h->g_kernels;
        } else {
            // plain launches: enqueue no step beyond max_steps
            const long long left = max_steps - (h->ctl_host->steps - s0);
            for (long long k = 0; k < chunk && k < left; ++k)
                if ((r = enqueue_step(h, U, h->stream))) return r;
        }
        if ((r = read_ctl(h))) return r;
        const Ctl &c = *h->ctl_host;
        if (steps_out) *steps_out = c.steps - s0;
        if ((c.status & ST_NONPHYSICAL) || !(c.t < t_end) || c.steps - s0 >= max_steps) break;
    }
    return take_status(h);
}

extern "C" int weno_run_host(weno_handle h, double *U_host, double t_end, double dt, int64_t max_steps,
                             int32_t graph_steps, int64_t *steps_out)
{
    int r = need_grid(h, "weno_run_host");
    if (r) return r;
    if (!U_host) return fail(h, WENO_ERR_ARG, "weno_run_host: null U_host");
    const size_t bytes = sizeof(double) * (size_t)h->nf * (size_t)h->N;
    if (!h->Udev) CK(h, cudaMalloc((void **)&h->Udev, bytes));
    CK(h, cudaMemcpyAsync(h->Udev, U_host, bytes, cudaMemcpyHostToDevice, h->stream));
    r = weno_run(h, h->Udev, t_end, dt, max_steps, graph_steps, steps_out);
    if (r != WENO_OK && r != WENO_ERR_NONPHYSICAL) return r;
    CK(h, cudaMemcpyAsync(U_host, h->Udev, bytes, cudaMemcpyDeviceToHost, h->stream));
    CK(h, cudaStreamSynchronize(h->stream));
    return r;
}

extern "C" int weno_sums(weno_handle h, const double *U, double *sums_host)
{
    int r = need_grid(h, "weno_sums");
    if (r) return r;
    if (!U || !sums_host) return fail(h, WENO_ERR_ARG, "weno_sums: null pointer");
    CK(h, launch(h, 7, h->stream, [&] { return launch_sums(U, h->nf, h->N, h->partials, h->nblocks_sum, h->sums_dev, h->stream); }, 2));
    CK(h, cudaMemcpyAsync(sums_host, h->sums_dev, sizeof(double) * h->nf, cudaMemcpyDeviceToHost, h->stream));
    CK(h, cudaStreamSynchronize(h->stream));
    return WENO_OK;
}

extern "C" int weno_sync(weno_handle h)
{
    if (!h) return WENO_ERR_ARG;
    return take_status(h);
}

// ------------------------------------------------------------- cross eval

namespace {
struct CrossPrep {
    std::vector<CrossInst> ci;
    std::vector<CrossSet> cs;
    long long work = 0, nvec = 0, samples = 0;
    int fp64 = 0, max_rank = 1;
    size_t off_inst = 0, off_sets = 0, off_vecs = 0, bytes = 0;
    std::string key;  // workload class of the autotuner
};
}  // namespace

static int cross_prepare(weno_ctx *h, const weno_tt_instance *inst, int32_t n_inst, const weno_fiber_set *sets,
                         int32_t n_sets, int32_t flags, CrossPrep &P)
{
    if (!inst || !sets || n_inst < 1 || n_sets < 1) return fail(h, WENO_ERR_ARG, "weno_cross_eval: empty input");
    P.ci.resize(n_inst);
    for (int k = 0; k < n_inst; ++k) {
        const weno_tt_instance &I = inst[k];
        CrossInst &c = P.ci[k];
        for (int m = 0; m < 3; ++m) {
            if (I.n[m] < 3 || !(I.h[m] > 0.0))
                return fail(h, WENO_ERR_ARG, "weno_cross_eval: instance needs n >= 3 and h > 0 per mode");
            c.n[m] = I.n[m];
            c.h[m] = I.h[m];
            for (int sd = 0; sd < 2; ++sd) {
                if (I.bc[m][sd] == WENO_BC_INFLOW)
                    return fail(h, WENO_ERR_UNSUPPORTED, "weno_cross_eval: inflow boundaries are not implemented for TT cores");
                if (I.bc[m][sd] < 0 || I.bc[m][sd] > 2) return fail(h, WENO_ERR_ARG, "weno_cross_eval: bad boundary rule");
                c.bc[m][sd] = I.bc[m][sd];
            }
        }
        for (int m = 0; m < 2; ++m) {
            if (I.r[m] < 1 || I.r[m] > cross_max_rank())
                return fail(h, WENO_ERR_ARG, "weno_cross_eval: TT ranks must be in 1..32");
            c.r[m] = I.r[m];
            P.max_rank = std::max(P.max_rank, (int)I.r[m]);
        }
        for (int f = 0; f < 5; ++f)
            for (int m = 0; m < 3; ++m) {
                if (!I.core[f][m]) return fail(h, WENO_ERR_ARG, "weno_cross_eval: null core");
                c.core[f][m] = I.core[f][m];
            }
        if (!(I.alpha >= 0.0) || !std::isfinite(I.alpha)) return fail(h, WENO_ERR_ARG, "weno_cross_eval: bad alpha");
        c.alpha = I.alpha;
    }
    P.cs.resize(n_sets);
    for (int k = 0; k < n_sets; ++k) {
        const weno_fiber_set &F = sets[k];
        CrossSet &c = P.cs[k];
        if (F.instance < 0 || F.instance >= n_inst || F.mode < 0 || F.mode > 2 || F.flux_dir < 0 || F.flux_dir > 2)
            return fail(h, WENO_ERR_ARG, "weno_cross_eval: bad instance, mode or flux_dir");
        if (F.n_left < 1 || F.n_right < 1 || !F.out || (F.mode > 0 && !F.left) || (F.mode < 2 && !F.right) ||
            (F.mode == 0 && F.n_left != 1) || (F.mode == 2 && F.n_right != 1))
            return fail(h, WENO_ERR_ARG, "weno_cross_eval: inconsistent index sets");
        c.inst = F.instance;
        c.mode = F.mode;
        c.fd = F.flux_dir;
        c.n_mode = P.ci[F.instance].n[F.mode];
        c.n_left = F.n_left;
        c.n_right = F.n_right;
        c.left = F.left;
        c.right = F.right;
        c.out = F.out;
        c.work_begin = P.work;
        // a work item fixes the index of the side the stencil does not move
        P.work += F.flux_dir > F.mode ? F.n_left : F.n_right;
        P.samples += F.n_left * F.n_right * c.n_mode;
        c.nsl = F.flux_dir < F.mode ? 7 : 1;
        c.nsr = F.flux_dir > F.mode ? 7 : 1;
        c.lvec_off = P.nvec;
        P.nvec += F.n_left * c.nsl * 5 * cross_vec_len();
        c.rvec_off = P.nvec;
        P.nvec += F.n_right * c.nsr * 5 * cross_vec_len();
    }
    if (P.work >= (1ll << 31)) return fail(h, WENO_ERR_ARG, "weno_cross_eval: more than 2^31 work items");
    P.fp64 = (flags & WENO_CROSS_FP64_CHECK) ? 1 : 0;
    const size_t esz = P.fp64 ? sizeof(double) : sizeof(float);
    P.off_inst = 64 + ((sizeof(int) * n_sets + 15) & ~size_t(15));
    P.off_sets = P.off_inst + ((sizeof(CrossInst) * n_inst + 15) & ~size_t(15));
    P.off_vecs = P.off_sets + ((sizeof(CrossSet) * n_sets + 15) & ~size_t(15));
    P.bytes = P.off_vecs + esz * (size_t)P.nvec;
    // workload class: precision, rank bucket, samples per launch to a factor of 4
    int sb = 0;
    for (long long x = P.samples; x >= 4; x >>= 2) ++sb;
    P.key = std::string(P.fp64 ? "f64" : "f32") + "_r" + std::to_string(P.max_rank <= 8 ? 8 : P.max_rank <= 16 ? 16 : 32) +
            "_s4^" + std::to_string(sb);
    return WENO_OK;
}

// Descriptor upload and the launch arguments for scratch at `base`.
static int cross_upload(weno_ctx *h, const CrossPrep &P, char *base, cudaStream_t s, CrossArgs &a)
{
    unsigned long long *counter = (unsigned long long *)base;
    int *dbad = (int *)(base + 64);
    CrossInst *dinst = (CrossInst *)(base + P.off_inst);
    CrossSet *dsets = (CrossSet *)(base + P.off_sets);
    // pageable sources: each copy returns once the data is staged
    CK(h, cudaMemcpyAsync(dinst, P.ci.data(), sizeof(CrossInst) * P.ci.size(), cudaMemcpyHostToDevice, s));
    CK(h, cudaMemcpyAsync(dsets, P.cs.data(), sizeof(CrossSet) * P.cs.size(), cudaMemcpyHostToDevice, s));
    a = CrossArgs{};
    a.inst = dinst;
    a.sets = dsets;
    a.n_sets = (int)P.cs.size();
    a.n_work = P.work;
    a.gamma = h->p.gamma;
    a.eps = h->p.eps_weno;
    a.counter = counter;
    a.status = &h->ctl->status;
    a.bad = dbad;
    a.vecs = base + P.off_vecs;
    a.fp64 = P.fp64;
    return WENO_OK;
}

static void cross_config(const weno_ctx *h, const std::string &key, int &variant, int &cpsm)
{
    variant = 0;
    cpsm = 4;
    auto it = h->tune.find(key);
    if (it != h->tune.end()) {
        variant = it->second.first;
        cpsm = it->second.second;
    }
}

static uint64_t fnv1a(uint64_t hsh, const void *p, size_t n)
{
    const unsigned char *b = (const unsigned char *)p;
    for (size_t i = 0; i < n; ++i) hsh = (hsh ^ b[i]) * 1099511628211ull;
    return hsh;
}

extern "C" int weno_cross_eval(weno_handle h, const weno_tt_instance *inst, int32_t n_inst, const weno_fiber_set *sets,
                               int32_t n_sets, int32_t flags)
{
    if (!h) return WENO_ERR_ARG;
    CrossPrep P;
    int r = cross_prepare(h, inst, n_inst, sets, n_sets, flags, P);
    if (r) return r;
    int variant, cpsm;
    cross_config(h, P.key, variant, cpsm);
    if (flags & WENO_CROSS_GRAPH) {
        // replay the graph captured for these exact descriptors (the device
        // arrays they point to may have new contents), or capture it now
        uint64_t key = 1469598103934665603ull;
        key = fnv1a(key, P.ci.data(), sizeof(CrossInst) * P.ci.size());
        key = fnv1a(key, P.cs.data(), sizeof(CrossSet) * P.cs.size());
        const double ge[2] = {h->p.gamma, h->p.eps_weno};
        const int cfg[3] = {P.fp64, variant, cpsm};
        key = fnv1a(key, ge, sizeof(ge));
        key = fnv1a(key, cfg, sizeof(cfg));
        for (auto &g : h->xgraphs)
            if (g.key == key) {
                g.last = ++h->xgraph_clock;
                CK(h, cudaGraphLaunch(g.exec, h->stream));
                h->launches += 2;
                return WENO_OK;
            }
        CK(h, cross_set_attributes());
        weno_ctx::XGraph g{};
        g.key = key;
        CK(h, cudaMalloc(&g.buf, P.bytes));
        CrossArgs a;
        if ((r = cross_upload(h, P, (char *)g.buf, h->stream, a))) {
            cudaFree(g.buf);
            return r;
        }
        CK(h, cudaStreamSynchronize(h->stream));
        cudaGraph_t graph = nullptr;
        CK(h, cudaStreamBeginCapture(h->capture, cudaStreamCaptureModeThreadLocal));
        cudaError_t e1 = cudaMemsetAsync(a.counter, 0, sizeof(unsigned long long), h->capture);
        cudaError_t e2 = e1 == cudaSuccess ? launch_cross(a, variant, cpsm, h->capture) : e1;
        cudaError_t e3 = cudaStreamEndCapture(h->capture, &graph);
        if (e2 != cudaSuccess || e3 != cudaSuccess) {
            if (graph) cudaGraphDestroy(graph);
            cudaFree(g.buf);
            return fail(h, WENO_ERR_CUDA, std::string("weno_cross_eval: graph capture: ") +
                                              cudaGetErrorString(e2 != cudaSuccess ? e2 : e3));
        }
        cudaError_t e4 = cudaGraphInstantiate(&g.exec, graph, 0);
        cudaGraphDestroy(graph);
        if (e4 != cudaSuccess) {
            cudaFree(g.buf);
            return fail(h, WENO_ERR_CUDA, std::string("weno_cross_eval: graph instantiate: ") + cudaGetErrorString(e4));
        }
        if (h->xgraphs.size() >= 16) {  // evict the least recently used
            auto lru = std::min_element(h->xgraphs.begin(), h->xgraphs.end(),
                                        [](const weno_ctx::XGraph &x, const weno_ctx::XGraph &y) { return x.last < y.last; });
            cudaGraphExecDestroy(lru->exec);
            cudaFree(lru->buf);
            h->xgraphs.erase(lru);
        }
        g.last = ++h->xgraph_clock;
        h->xgraphs.push_back(g);
        CK(h, cudaGraphLaunch(g.exec, h->stream));
        h->launches += 2;
        return WENO_OK;
    }
    if ((r = grow(h, &h->xbuf, &h->xbuf_bytes, P.bytes))) return r;
    CrossArgs a;
    if ((r = cross_upload(h, P, (char *)h->xbuf, h->stream, a))) return r;
    CK(h, cudaMemsetAsync(a.counter, 0, sizeof(unsigned long long), h->stream));
    CK(h, launch(h, 7, h->stream, [&] { return launch_cross(a, variant, cpsm, h->stream); }, 2));
    return WENO_OK;
}

// Times every compiled k_cross variant and persistent grid size on this
// workload and keeps the fastest for its workload class.
extern "C" int weno_cross_autotune(weno_handle h, const weno_tt_instance *inst, int32_t n_inst,
                                   const weno_fiber_set *sets, int32_t n_sets, int32_t flags, int32_t reps,
                                   int32_t *choice, double *ms_out)
{
    if (!h) return WENO_ERR_ARG;
    if (reps < 1) return fail(h, WENO_ERR_ARG, "weno_cross_autotune: reps must be >= 1");
    CrossPrep P;
    int r = cross_prepare(h, inst, n_inst, sets, n_sets, flags, P);
    if (r) return r;
    if ((r = grow(h, &h->xbuf, &h->xbuf_bytes, P.bytes))) return r;
    CrossArgs a;
    if ((r = cross_upload(h, P, (char *)h->xbuf, h->stream, a))) return r;
    cudaEvent_t e0, e1;
    CK(h, cudaEventCreate(&e0));
    CK(h, cudaEventCreate(&e1));
    double best = 1e300;
    int bv = 0, bc = 4;
    for (int v = 0; v < cross_num_variants(); ++v)
        for (int c = 1; c <= 4; ++c) {
            for (int k = 0; k <= reps; ++k) {  // the first run is a warm-up
                if (k == 1) CK(h, cudaEventRecord(e0, h->stream));
                CK(h, cudaMemsetAsync(a.counter, 0, sizeof(unsigned long long), h->stream));
                CK(h, launch_cross(a, v, c, h->stream));
            }
            CK(h, cudaEventRecord(e1, h->stream));
            CK(h, cudaEventSynchronize(e1));
            float ms = 0.0f;
            CK(h, cudaEventElapsedTime(&ms, e0, e1));
            if (ms / reps < best) {
                best = ms / reps;
                bv = v;
                bc = c;
            }
        }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    h->tune[P.key] = std::make_pair(bv, bc);
    if (choice) {
        int t, ch;
        cross_variant(bv, &t, &ch);
        choice[0] = t;
        choice[1] = ch;
        choice[2] = bc;
    }
    if (ms_out) *ms_out = best;
    return take_status(h);
}

// Tuning cache: a text file whose first line names the GPU and its SM count;
// each further line is "<workload class> <variant> <CTAs per SM>".
static std::string device_tag()
{
    int dev = 0;
    cudaDeviceProp prop{};
    if (cudaGetDevice(&dev) != cudaSuccess || cudaGetDeviceProperties(&prop, dev) != cudaSuccess) return "unknown";
    std::string name(prop.name);
    for (auto &c : name)
        if (c == ' ') c = '_';
    return name + "_sm" + std::to_string(prop.multiProcessorCount);
}

extern "C" int weno_tune_save(weno_handle h, const char *path)
{
    if (!h) return WENO_ERR_ARG;
    if (!path) return fail(h, WENO_ERR_ARG, "weno_tune_save: null path");
    FILE *f = fopen(path, "w");
    if (!f) return fail(h, WENO_ERR_ARG, std::string("weno_tune_save: cannot open ") + path);
    fprintf(f, "device %s\n", device_tag().c_str());
    for (auto &kv : h->tune) fprintf(f, "%s %d %d\n", kv.first.c_str(), kv.second.first, kv.second.second);
    fclose(f);
    return WENO_OK;
}

extern "C" int weno_tune_load(weno_handle h, const char *path, int32_t *n_loaded)
{
    if (!h) return WENO_ERR_ARG;
    if (n_loaded) *n_loaded = 0;
    if (!path) return fail(h, WENO_ERR_ARG, "weno_tune_load: null path");
    FILE *f = fopen(path, "r");
    if (!f) return fail(h, WENO_ERR_ARG, std::string("weno_tune_load: cannot open ") + path);
    char tag[256] = {0}, dev[256] = {0};
    int n = 0;
    if (fscanf(f, "%255s %255s", tag, dev) == 2 && std::string(tag) == "device" && std::string(dev) == device_tag()) {
        char key[256];
        int v, c;
        while (fscanf(f, "%255s %d %d", key, &v, &c) == 3)
            if (v >= 0 && v < cross_num_variants() && c >= 1 && c <= 4) {
                h->tune[key] = std::make_pair(v, c);
                ++n;
            }
    }
    fclose(f);
    if (n_loaded) *n_loaded = n;
    return WENO_OK;
}

extern "C" int weno_profile_enable(weno_handle h, int32_t enable)
{
    if (!h) return WENO_ERR_ARG;
    CK(h, cudaStreamSynchronize(h->stream));
    for (auto &ev : h->pending) {
        h->pool.push_back(ev.a);
        h->pool.push_back(ev.b);
    }
    h->pending.clear();
    for (int k = 0; k < WENO_PROFILE_KINDS; ++k) {
        h->prof_ms[k] = 0.0;
        h->prof_n[k] = 0;
    }
    h->launches = 0;
    h->prof = enable != 0;
    return WENO_OK;
}

extern "C" int weno_profile_read(weno_handle h, double *ms, int64_t *launches, int64_t *total_launches)
{
    if (!h) return WENO_ERR_ARG;
    CK(h, cudaStreamSynchronize(h->stream));
    for (auto &ev : h->pending) {
        float t = 0.0f;
        CK(h, cudaEventElapsedTime(&t, ev.a, ev.b));
        h->prof_ms[ev.kind] += t;
        h->prof_n[ev.kind] += 1;
        h->pool.push_back(ev.a);
        h->pool.push_back(ev.b);
    }
    h->pending.clear();
    for (int k = 0; k < WENO_PROFILE_KINDS; ++k) {
        if (ms) ms[k] = h->prof_ms[k];
        if (launches) launches[k] = h->prof_n[k];
    }
    if (total_launches) *total_launches = h->launches;
    return WENO_OK;
}

// ------------------------------------------------------------ TT-rounding
// weno_tt_round: round(sum_t c_t X_t, eps) for a batch of 3D TTs (Sec. 3
// "TT-rounding"; the stages of Eq. tt-ssprk3 are such sums).  Phase 1
// (right-to-left orthogonalisation and the first truncated SVD) and phase 2
// (the second SVD) end with a host read of the ranks they chose, which size
// the launches that follow.

namespace {

struct QRPlan {
    long long m = 0;
    int k = 0, b = 32, C = 1, sub = 1, top_sub = 0;
    long long chunk_rows = 0;
    double *A = nullptr, *tau = nullptr, *Rc = nullptr, *tau_top = nullptr, *T = nullptr;
};

// Chunking of an m x k QR: sub-blocks of b >= k rows, at most 16 per chunk,
// every chunk at least k rows long when there are several.
void qr_plan(QRPlan &q, long long m, int k)
{
    q.m = m;
    q.k = k;
    q.b = k <= 32 ? 32 : (k + 31) / 32 * 32;
    int C = (int)std::max(1LL, (m + 16LL * q.b - 1) / (16LL * q.b));
    for (;; --C) {
        const long long cr = (m + C - 1) / C;
        if (C == 1 || (cr >= k && m - (long long)(C - 1) * cr >= k)) {
            q.C = C;
            q.chunk_rows = std::max(1LL, cr);
            break;
        }
    }
    q.sub = (int)((q.chunk_rows + q.b - 1) / q.b);
    q.top_sub = q.C > 1 ? (int)(((long long)q.C * k + q.b - 1) / q.b) : 0;
}

struct Bump {  // counts (base == nullptr) or hands out 256-byte aligned pieces
    char *base = nullptr;
    size_t off = 0;
    template <class T> T *take(size_t n)
    {
        off = (off + 255) & ~size_t(255);
        T *p = base ? reinterpret_cast<T *>(base + off) : nullptr;
        off += sizeof(T) * n;
        return p;
    }
};

void qr_take(Bump &bp, QRPlan &q)
{
    q.tau = bp.take<double>((size_t)q.C * q.sub * q.k);
    q.Rc = bp.take<double>((size_t)q.C * q.k * q.k);
    if (q.C > 1) {
        q.tau_top = bp.take<double>((size_t)q.top_sub * q.k);
        q.T = bp.take<double>((size_t)q.k * q.k);
    } else {
        q.T = q.Rc;
    }
}

struct TTPlan {
    int n[3] = {0, 0, 0};
    int R1 = 0, R2 = 0, k3 = 0, k2 = 0, kc = 0, ke = 0;
    long long mB = 0;
    double *C1 = nullptr, *MA = nullptr, *MB = nullptr, *MC = nullptr, *ME = nullptr;
    QRPlan qa, qb, qc, qe, qe_max;
    double *VC = nullptr, *WC = nullptr, *svC = nullptr, *VE = nullptr, *WE = nullptr, *svE = nullptr;
    double *delta = nullptr;
    double *XSa = nullptr, *XSb = nullptr, *XSc = nullptr, *XSe = nullptr;
    int r1 = 0, r2 = 0;
};

}  // namespace

// Factor every plan (leaf chunks, then the stacked chunk R factors).
static int tt_factor(weno_ctx *h, std::vector<QRPlan *> &ps, QRDesc *dev)
{
    const int n = (int)ps.size();
    std::vector<QRDesc> leaf(n), top(n);
    int maxC = 1, maxk = 1, maxb = 32;
    bool any_top = false;
    for (int i = 0; i < n; ++i) {
        const QRPlan &q = *ps[i];
        leaf[i] = QRDesc{q.A, q.m, q.k, q.k, q.b, q.C, q.chunk_rows, q.sub, q.tau, q.Rc};
        top[i] = QRDesc{q.Rc, q.C > 1 ? (long long)q.C * q.k : 0, q.k, q.k, q.b, 1, (long long)q.C * q.k,
                        q.top_sub, q.tau_top, q.T};
        maxC = std::max(maxC, q.C);
        maxk = std::max(maxk, q.k);
        maxb = std::max(maxb, q.b);
        any_top |= q.C > 1;
    }
    const size_t smem = qr_factor_smem(maxk, maxb);
    CK(h, cudaMemcpyAsync(dev, leaf.data(), sizeof(QRDesc) * n, cudaMemcpyHostToDevice, h->stream));
    CK(h, launch(h, 0, h->stream, [&] { return launch_qr_factor(dev, n, maxC, smem, h->stream); }));
    if (any_top) {
        CK(h, cudaMemcpyAsync(dev + n, top.data(), sizeof(QRDesc) * n, cudaMemcpyHostToDevice, h->stream));
        CK(h, launch(h, 0, h->stream, [&] { return launch_qr_factor(dev + n, n, 1, smem, h->stream); }));
    }
    return WENO_OK;
}

struct ApplyReq {  // Q [X; 0] of one plan into an output row map
    const QRPlan *q;
    const double *X;
    int ldx, p;
    double *XS;  // stack of the chunks' top rows (C > 1)
    double *out;
    long long P, sP, sQ, sC;
};

static int tt_apply(weno_ctx *h, std::vector<ApplyReq> &rs, QApplyDesc *dev)
{
    const int n = (int)rs.size();
    std::vector<QApplyDesc> leaf(n), top(n);
    int maxC = 1, maxk = 1, maxb = 32, maxp = 1;
    bool any_top = false;
    for (int i = 0; i < n; ++i) {
        const ApplyReq &r = rs[i];
        const QRPlan &q = *r.q;
        const bool two = q.C > 1;
        const long long mt = (long long)q.C * q.k;
        top[i] = QApplyDesc{q.Rc, q.tau_top, two ? mt : 0, q.k, q.k, q.b, 1, mt, q.top_sub, r.X, 0, r.ldx, r.p,
                            r.XS, mt, r.p, 0, 1};
        leaf[i] = QApplyDesc{q.A, q.tau, q.m, q.k, q.k, q.b, q.C, q.chunk_rows, q.sub, two ? r.XS : r.X,
                             two ? (long long)q.k * r.p : 0, two ? r.p : r.ldx, r.p, r.out, r.P, r.sP, r.sQ, r.sC};
        maxC = std::max(maxC, q.C);
        maxk = std::max(maxk, q.k);
        maxb = std::max(maxb, q.b);
        maxp = std::max(maxp, r.p);
        any_top |= two;
    }
    const size_t smem = qr_apply_smem(maxk, maxb, maxp);
    if (any_top) {
        CK(h, cudaMemcpyAsync(dev + n, top.data(), sizeof(QApplyDesc) * n, cudaMemcpyHostToDevice, h->stream));
        CK(h, launch(h, 0, h->stream, [&] { return launch_qr_apply(dev + n, n, 1, smem, h->stream); }));
    }
    CK(h, cudaMemcpyAsync(dev, leaf.data(), sizeof(QApplyDesc) * n, cudaMemcpyHostToDevice, h->stream));
    CK(h, launch(h, 0, h->stream, [&] { return launch_qr_apply(dev, n, maxC, smem, h->stream); }));
    return WENO_OK;
}

static int tt_svd(weno_ctx *h, std::vector<SvdDesc> &ds, SvdDesc *dev)
{
    const int n = (int)ds.size();
    int maxpk = 1, maxq = 1;
    for (auto &d : ds) {
        maxpk = std::max(maxpk, d.pk);
        maxq = std::max(maxq, d.q);
    }
    const size_t smem = svd_smem(maxpk, maxq);
    CK(h, cudaMemcpyAsync(dev, ds.data(), sizeof(SvdDesc) * n, cudaMemcpyHostToDevice, h->stream));
    CK(h, launch(h, 1, h->stream, [&] { return launch_svd_jacobi(dev, n, smem, h->stream); }));
    return WENO_OK;
}

extern "C" int weno_tt_round(weno_handle h, weno_tt_round_problem *probs, int32_t n_probs, double eps_tt)
{
    if (!h) return WENO_ERR_ARG;
    if (!probs || n_probs < 1 || n_probs > 65535) return fail(h, WENO_ERR_ARG, "weno_tt_round: need 1..65535 problems");
    if (!(eps_tt >= 0.0)) return fail(h, WENO_ERR_ARG, "weno_tt_round: need eps_tt >= 0");
    const int np = n_probs;
    std::vector<TTPlan> pl(np);
    std::vector<TTSumDesc> sd(np);
    for (int i = 0; i < np; ++i) {
        const weno_tt_round_problem &P = probs[i];
        TTPlan &t = pl[i];
        TTSumDesc &s = sd[i];
        if (P.n_terms < 1 || P.n_terms > WENO_TT_MAX_TERMS) return fail(h, WENO_ERR_ARG, "weno_tt_round: 1..4 terms");
        s.nt = P.n_terms;
        for (int m = 0; m < 3; ++m) t.n[m] = s.n[m] = P.term[0].n[m];
        int a = 0, b = 0;
        for (int k = 0; k < P.n_terms; ++k) {
            const weno_tt3 &X = P.term[k];
            for (int m = 0; m < 3; ++m) {
                if (X.n[m] != t.n[m] || X.n[m] < 1 || X.n[m] > (1 << 20))
                    return fail(h, WENO_ERR_ARG, "weno_tt_round: terms need equal mode sizes in 1..2^20");
                if (!X.core[m]) return fail(h, WENO_ERR_ARG, "weno_tt_round: null core");
                s.core[k][m] = X.core[m];
            }
            if (X.r[0] < 1 || X.r[1] < 1) return fail(h, WENO_ERR_ARG, "weno_tt_round: ranks must be >= 1");
            s.a0[k] = a;
            s.b0[k] = b;
            s.r1[k] = X.r[0];
            s.r2[k] = X.r[1];
            s.coef[k] = P.coef[k];
            a += X.r[0];
            b += X.r[1];
        }
        if (a > TT_KMAX || b > TT_KMAX)
            return fail(h, WENO_ERR_UNSUPPORTED, "weno_tt_round: the ranks of a sum may add up to 96 at most");
        for (int m = 0; m < 3; ++m)
            if (!P.out.core[m]) return fail(h, WENO_ERR_ARG, "weno_tt_round: null output core");
        t.R1 = s.R1 = a;
        t.R2 = s.R2 = b;
        t.k3 = s.k3 = std::min(t.n[2], t.R2);
        t.mB = (long long)t.n[1] * t.k3;
        t.k2 = (int)std::min<long long>(t.mB, t.R1);
        t.kc = std::min(t.n[0], t.k2);
        qr_plan(t.qa, t.n[2], t.R2);
        qr_plan(t.qb, t.mB, t.R1);
        qr_plan(t.qc, t.n[0], t.k2);
        qr_plan(t.qe_max, (long long)t.kc * t.n[1], t.k3);
        t.ke = (int)std::min<long long>((long long)t.kc * t.n[1], t.k3);
    }
    // scratch: descriptors, ranks, then per problem matrices and QR data
    const int NDESC = 24;
    const size_t dsz = std::max({sizeof(QRDesc), sizeof(QApplyDesc), sizeof(SvdDesc), sizeof(TTSumDesc), sizeof(GemmDesc)});
    auto layout = [&](Bump &bp) -> char * {
        char *desc = bp.take<char>(dsz * NDESC * (size_t)np);
        for (auto &t : pl) {
            t.C1 = bp.take<double>((size_t)t.n[0] * t.R1);
            t.MA = bp.take<double>((size_t)t.n[2] * t.R2);
            t.MB = bp.take<double>((size_t)t.mB * t.R1);
            t.MC = bp.take<double>((size_t)t.n[0] * t.k2);
            t.ME = bp.take<double>((size_t)t.kc * t.n[1] * t.k3);
            qr_take(bp, t.qa);
            qr_take(bp, t.qb);
            qr_take(bp, t.qc);
            qr_take(bp, t.qe_max);
            t.VC = bp.take<double>((size_t)t.kc * t.kc);
            t.WC = bp.take<double>((size_t)t.k2 * t.kc);
            t.svC = bp.take<double>(t.kc);
            t.VE = bp.take<double>((size_t)t.ke * t.ke);
            t.WE = bp.take<double>((size_t)t.k3 * t.ke);
            t.svE = bp.take<double>(t.ke);
            t.delta = bp.take<double>(2);
            t.XSa = bp.take<double>((size_t)t.qa.C * t.qa.k * t.ke);
            t.XSb = bp.take<double>((size_t)t.qb.C * t.qb.k * t.kc);
            t.XSc = bp.take<double>((size_t)t.qc.C * t.qc.k * t.kc);
            t.XSe = bp.take<double>((size_t)t.qe_max.C * t.qe_max.k * t.ke);
        }
        return desc;
    };
    Bump count;
    layout(count);
    const size_t rank_off = (count.off + 255) & ~size_t(255);
    const size_t bytes = rank_off + sizeof(int) * 2 * (size_t)np;
    if (bytes > h->tbuf_bytes) {
        CK(h, cudaStreamSynchronize(h->stream));
        cudaFree(h->tbuf);
        h->tbuf = nullptr;
        h->tbuf_bytes = 0;
        CK(h, cudaMalloc(&h->tbuf, bytes));
        h->tbuf_bytes = bytes;
    }
    Bump bp;
    bp.base = (char *)h->tbuf;
    char *desc = layout(bp);
    int *ranks = (int *)((char *)h->tbuf + rank_off);
    int slot = 0;
    auto next_desc = [&]() { return desc + dsz * (size_t)np * (slot++); };

    for (int i = 0; i < np; ++i) {
        TTPlan &t = pl[i];
        sd[i].C1 = t.C1;
        sd[i].MA = t.MA;
        sd[i].MB = t.MB;
        sd[i].TA = t.qa.T;
        t.qa.A = t.MA;
        t.qb.A = t.MB;
        t.qc.A = t.MC;
        t.qe_max.A = t.ME;
    }
    // ---- phase 1: sum unfoldings; QR of the last core; middle core times TA^T; QR; first core; QR; SVD
    {
        TTSumDesc *d = (TTSumDesc *)next_desc();
        CK(h, cudaMemcpyAsync(d, sd.data(), sizeof(TTSumDesc) * np, cudaMemcpyHostToDevice, h->stream));
        CK(h, launch(h, 1, h->stream, [&] { return launch_tt_build(d, np, h->stream); }));
        std::vector<QRPlan *> ps;
        for (auto &t : pl) ps.push_back(&t.qa);
        int r = tt_factor(h, ps, (QRDesc *)next_desc());
        if (r) return r;
        ++slot;
        CK(h, launch(h, 1, h->stream, [&] { return launch_tt_contract(d, np, h->stream); }));
        ps.clear();
        for (auto &t : pl) ps.push_back(&t.qb);
        if ((r = tt_factor(h, ps, (QRDesc *)next_desc()))) return r;
        ++slot;
        std::vector<GemmDesc> gd(np);
        for (int i = 0; i < np; ++i)
            gd[i] = GemmDesc{pl[i].C1, pl[i].qb.T, pl[i].MC, pl[i].n[0], pl[i].k2, pl[i].R1};
        GemmDesc *gdev = (GemmDesc *)next_desc();
        CK(h, cudaMemcpyAsync(gdev, gd.data(), sizeof(GemmDesc) * np, cudaMemcpyHostToDevice, h->stream));
        CK(h, launch(h, 1, h->stream, [&] { return launch_tt_gemm_tr(gdev, np, h->stream); }));
        ps.clear();
        for (auto &t : pl) ps.push_back(&t.qc);
        if ((r = tt_factor(h, ps, (QRDesc *)next_desc()))) return r;
        ++slot;
        std::vector<SvdDesc> sv(np);
        for (int i = 0; i < np; ++i) {
            TTPlan &t = pl[i];
            sv[i] = SvdDesc{t.qc.T, t.k2, t.kc, t.k2, eps_tt, 1, t.delta, ranks + 2 * i, t.kc, t.svC, t.VC, t.WC, t.kc};
        }
        if ((r = tt_svd(h, sv, (SvdDesc *)next_desc()))) return r;
    }
    std::vector<int> rk(2 * np);
    CK(h, cudaMemcpyAsync(rk.data(), ranks, sizeof(int) * 2 * np, cudaMemcpyDeviceToHost, h->stream));
    CK(h, cudaStreamSynchronize(h->stream));
    for (int i = 0; i < np; ++i) {
        TTPlan &t = pl[i];
        t.r1 = rk[2 * i];
        if (t.r1 < 1 || t.r1 > t.kc) return fail(h, WENO_ERR_CUDA, "weno_tt_round: device returned a bad rank");
        if (probs[i].cap[0] < (long long)t.n[0] * t.r1)
            return fail(h, WENO_ERR_ARG, "weno_tt_round: output core 1 capacity too small");
        t.qe = t.qe_max;
        qr_plan(t.qe, (long long)t.r1 * t.n[1], t.k3);
        t.qe.A = t.ME;
        t.qe.tau = t.qe_max.tau;
        t.qe.Rc = t.qe_max.Rc;
        t.qe.tau_top = t.qe_max.tau_top;
        t.qe.T = t.qe.C > 1 ? t.qe_max.T : t.qe.Rc;
    }
    // ---- phase 2: first output core; the middle core into the (r1 n2) x k3 unfolding; QR; SVD
    {
        std::vector<ApplyReq> ar(np);
        for (int i = 0; i < np; ++i) {
            TTPlan &t = pl[i];
            ar[i] = ApplyReq{&t.qc, t.VC, t.kc, t.r1, t.XSc, probs[i].out.core[0], t.n[0], t.r1, 0, 1};
        }
        int r = tt_apply(h, ar, (QApplyDesc *)next_desc());
        if (r) return r;
        ++slot;
        for (int i = 0; i < np; ++i) {
            TTPlan &t = pl[i];
            ar[i] = ApplyReq{&t.qb, t.WC, t.kc, t.r1, t.XSb, t.ME, t.mB, 1, 0, t.mB};
        }
        if ((r = tt_apply(h, ar, (QApplyDesc *)next_desc()))) return r;
        ++slot;
        std::vector<QRPlan *> ps;
        for (auto &t : pl) ps.push_back(&t.qe);
        if ((r = tt_factor(h, ps, (QRDesc *)next_desc()))) return r;
        ++slot;
        std::vector<SvdDesc> sv(np);
        for (int i = 0; i < np; ++i) {
            TTPlan &t = pl[i];
            const int pk = (int)std::min<long long>((long long)t.r1 * t.n[1], t.k3);
            sv[i] = SvdDesc{t.qe.T, t.k3, pk, t.k3, eps_tt, 0, t.delta, ranks + 2 * i + 1, pk, t.svE, t.VE, t.WE, t.ke};
        }
        if ((r = tt_svd(h, sv, (SvdDesc *)next_desc()))) return r;
    }
    std::vector<double> norms(2 * np);
    CK(h, cudaMemcpyAsync(rk.data(), ranks, sizeof(int) * 2 * np, cudaMemcpyDeviceToHost, h->stream));
    for (int i = 0; i < np; ++i)
        CK(h, cudaMemcpyAsync(&norms[2 * i], pl[i].delta, sizeof(double) * 2, cudaMemcpyDeviceToHost, h->stream));
    CK(h, cudaStreamSynchronize(h->stream));
    for (int i = 0; i < np; ++i) {
        TTPlan &t = pl[i];
        t.r2 = rk[2 * i + 1];
        if (t.r2 < 1 || t.r2 > t.ke) return fail(h, WENO_ERR_CUDA, "weno_tt_round: device returned a bad rank");
        if (probs[i].cap[1] < (long long)t.n[1] * t.r1 * t.r2 || probs[i].cap[2] < (long long)t.n[2] * t.r2)
            return fail(h, WENO_ERR_ARG, "weno_tt_round: output core 2 or 3 capacity too small");
    }
    // ---- phase 3: middle and last output cores
    {
        std::vector<ApplyReq> ar(np);
        for (int i = 0; i < np; ++i) {
            TTPlan &t = pl[i];
            ar[i] = ApplyReq{&t.qe, t.VE, t.ke, t.r2, t.XSe, probs[i].out.core[1], t.n[1], (long long)t.r1 * t.r2,
                             t.r2, 1};
        }
        int r = tt_apply(h, ar, (QApplyDesc *)next_desc());
        if (r) return r;
        ++slot;
        for (int i = 0; i < np; ++i) {
            TTPlan &t = pl[i];
            ar[i] = ApplyReq{&t.qa, t.WE, t.ke, t.r2, t.XSa, probs[i].out.core[2], t.n[2], t.r2, 0, 1};
        }
        if ((r = tt_apply(h, ar, (QApplyDesc *)next_desc()))) return r;
        ++slot;
    }
    for (int i = 0; i < np; ++i) {
        weno_tt3 &o = probs[i].out;
        for (int m = 0; m < 3; ++m) o.n[m] = pl[i].n[m];
        o.r[0] = pl[i].r1;
        o.r[1] = pl[i].r2;
        probs[i].norm = norms[2 * i + 1];
    }
    return WENO_OK;
}

// ------------------------------------------------------------------ maxvol

static int grow(weno_ctx *h, void **buf, size_t *have, size_t bytes)
{
    if (bytes <= *have) return WENO_OK;
    CK(h, cudaStreamSynchronize(h->stream));
    cudaFree(*buf);
    *buf = nullptr;
    *have = 0;
    CK(h, cudaMalloc(buf, bytes));
    *have = bytes;
    return WENO_OK;
}

extern "C" int weno_maxvol(weno_handle h, const weno_maxvol_problem *probs, int32_t n_probs, double delta,
                           int32_t max_iters, int32_t *swaps)
{
    if (!h) return WENO_ERR_ARG;
    if (!probs || n_probs < 1) return fail(h, WENO_ERR_ARG, "weno_maxvol: empty input");
    if (!(delta >= 0.0) || max_iters < 0) return fail(h, WENO_ERR_ARG, "weno_maxvol: need delta >= 0, max_iters >= 0");
    std::vector<MaxvolDesc> ds(n_probs);
    size_t w_total = 0;
    int max_r = 1;
    for (int i = 0; i < n_probs; ++i) {
        const weno_maxvol_problem &P = probs[i];
        if (P.r < 1 || P.r > MV_RMAX || P.n < P.r || !P.A || !P.B || !P.idx)
            return fail(h, WENO_ERR_ARG, "weno_maxvol: need 1 <= r <= 64, n >= r and non-null A, B, idx");
        w_total += (((size_t)P.n * P.r + 31) & ~size_t(31));
        max_r = std::max(max_r, (int)P.r);
    }
    const size_t off_desc = 0;
    const size_t off_int = (sizeof(MaxvolDesc) * n_probs + 255) & ~size_t(255);
    const size_t off_w = (off_int + sizeof(int) * 2 * n_probs + 255) & ~size_t(255);
    int r = grow(h, &h->mbuf, &h->mbuf_bytes, off_w + sizeof(double) * w_total);
    if (r) return r;
    char *base = (char *)h->mbuf;
    int *ints = (int *)(base + off_int);
    double *w = (double *)(base + off_w);
    for (int i = 0; i < n_probs; ++i) {
        const weno_maxvol_problem &P = probs[i];
        ds[i] = MaxvolDesc{P.A, P.B, w, P.idx, ints + 2 * i, ints + 2 * i + 1, P.n, P.r};
        w += (((size_t)P.n * P.r + 31) & ~size_t(31));
    }
    MaxvolDesc *dd = (MaxvolDesc *)(base + off_desc);
    CK(h, cudaMemcpyAsync(dd, ds.data(), sizeof(MaxvolDesc) * n_probs, cudaMemcpyHostToDevice, h->stream));
    CK(h, launch(h, 1, h->stream, [&] { return launch_maxvol(dd, n_probs, max_r, delta, max_iters, h->stream); }));
    std::vector<int> st(2 * n_probs);
    CK(h, cudaMemcpyAsync(st.data(), ints, sizeof(int) * 2 * n_probs, cudaMemcpyDeviceToHost, h->stream));
    CK(h, cudaStreamSynchronize(h->stream));
    for (int i = 0; i < n_probs; ++i) {
        if (st[2 * i]) return fail(h, WENO_ERR_ARG, "weno_maxvol: the pivot rows of a matrix are singular (rank < r)");
        if (swaps) swaps[i] = st[2 * i + 1];
    }
    return WENO_OK;
}

// ---------------------------------------------------------------- TT-cross
// weno_tt_cross: fixed-rank alternating TT-cross of A(i, j, k, f), the flux_dir
// residual contribution of component f of each TT instance (evaluated on
// fibers by weno_cross_eval), with maxvol selecting the index sets.  Every
// step is batched over the instances and runs on the handle's stream without
// a host round trip; the call synchronises once at the end to read maxvol's
// status words.

namespace {
struct XProb {
    int n[3] = {0, 0, 0};
    int r1 = 0, r2 = 0;
    void *outL0 = nullptr, *outL1 = nullptr, *outL2 = nullptr;
    int *right0 = nullptr, *left1 = nullptr, *right1 = nullptr, *left2 = nullptr;
    double *M0 = nullptr, *M1 = nullptr, *MR2 = nullptr, *MR1 = nullptr;
    double *Q0 = nullptr, *Q1 = nullptr, *QR2 = nullptr, *QR1 = nullptr;
    double *B1 = nullptr, *BR = nullptr, *Wmv = nullptr;
    int *idx = nullptr;
    QRPlan q0, q1, qr2, qr1;
};
}  // namespace

extern "C" int weno_tt_cross(weno_handle h, const weno_tt_instance *inst, int32_t n_inst, int32_t flux_dir,
                             weno_tt_cross_problem *probs, int32_t sweeps, double delta, int32_t flags)
{
    if (!h) return WENO_ERR_ARG;
    if (!inst || !probs || n_inst < 1 || n_inst > 65535) return fail(h, WENO_ERR_ARG, "weno_tt_cross: need 1..65535 instances");
    if (flux_dir < 0 || flux_dir > 2 || sweeps < 0 || sweeps > 64 || !(delta >= 0.0))
        return fail(h, WENO_ERR_ARG, "weno_tt_cross: need flux_dir 0..2, sweeps 0..64, delta >= 0");
    const bool fp64 = (flags & WENO_CROSS_FP64_CHECK) != 0;
    const size_t esz = fp64 ? sizeof(double) : sizeof(float);
    const int np = n_inst;
    std::vector<XProb> xp(np);
    int max_r = 1;
    for (int i = 0; i < np; ++i) {
        XProb &x = xp[i];
        const weno_tt_cross_problem &P = probs[i];
        for (int m = 0; m < 3; ++m) x.n[m] = inst[i].n[m];
        x.r1 = P.r[0];
        x.r2 = P.r[1];
        const long long n1 = x.n[0], n2 = x.n[1], n3 = x.n[2];
        if (x.r1 < 1 || x.r1 > MV_RMAX || x.r1 > n1 || x.r1 > 5 * n2 * n3 || x.r2 < 1 || x.r2 > MV_RMAX ||
            x.r2 > (long long)x.r1 * n2 || x.r2 > 5 * n3 || x.r1 > n2 * x.r2)
            return fail(h, WENO_ERR_ARG, "weno_tt_cross: need 1 <= r1 <= min(n1, n2 r2, 64), 1 <= r2 <= min(r1 n2, 5 n3, 64)");
        if (!P.J1 || !P.J2 || !P.I1 || !P.I2 || !P.core[0] || !P.core[1] || !P.core[2])
            return fail(h, WENO_ERR_ARG, "weno_tt_cross: null index set or core");
        max_r = std::max({max_r, x.r1, x.r2});
        qr_plan(x.q0, n1, x.r1);
        qr_plan(x.q1, (long long)x.r1 * n2, x.r2);
        qr_plan(x.qr2, 5 * n3, x.r2);
        qr_plan(x.qr1, n2 * x.r2, x.r1);
    }
    const int n_mv = 2 * (sweeps + 1) + 2 * sweeps;  // maxvol calls of the whole run
    const int NSLOT = 6;
    const size_t dsz = std::max({sizeof(QRDesc), sizeof(QApplyDesc), sizeof(MaxvolDesc), sizeof(CrossDrvDesc)});
    auto layout = [&](Bump &bp) -> char * {
        char *desc = bp.take<char>(dsz * NSLOT * 2 * (size_t)np);
        for (auto &x : xp) {
            const size_t n1 = x.n[0], n2 = x.n[1], n3 = x.n[2], r1 = x.r1, r2 = x.r2;
            x.outL0 = bp.take<char>(esz * 5 * n1 * r1);
            x.outL1 = bp.take<char>(esz * 5 * r1 * n2 * r2);
            x.outL2 = bp.take<char>(esz * 5 * r2 * n3);
            x.right0 = bp.take<int>(2 * r1);
            x.left1 = bp.take<int>(r1);
            x.right1 = bp.take<int>(r2);
            x.left2 = bp.take<int>(2 * r2);
            x.M0 = bp.take<double>(n1 * r1);
            x.M1 = bp.take<double>(r1 * n2 * r2);
            x.MR2 = bp.take<double>(5 * n3 * r2);
            x.MR1 = bp.take<double>(n2 * r2 * r1);
            x.Q0 = bp.take<double>(n1 * r1);
            x.Q1 = bp.take<double>(r1 * n2 * r2);
            x.QR2 = bp.take<double>(5 * n3 * r2);
            x.QR1 = bp.take<double>(n2 * r2 * r1);
            x.B1 = bp.take<double>(r1 * n2 * r2);
            const size_t mk = std::max({n1 * r1, r1 * n2 * r2, 5 * n3 * r2, n2 * r2 * r1});
            x.BR = bp.take<double>(mk);
            x.Wmv = bp.take<double>(mk);
            x.idx = bp.take<int>(std::max(r1, r2));
            qr_take(bp, x.q0);
            qr_take(bp, x.q1);
            qr_take(bp, x.qr2);
            qr_take(bp, x.qr1);
        }
        return desc;
    };
    Bump count;
    layout(count);
    const size_t st_off = (count.off + 255) & ~size_t(255);
    int r = grow(h, &h->cbuf, &h->cbuf_bytes, st_off + sizeof(int) * 2 * (size_t)n_mv * np);
    if (r) return r;
    Bump bp;
    bp.base = (char *)h->cbuf;
    char *desc = layout(bp);
    int *status = (int *)((char *)h->cbuf + st_off);
    auto slot = [&](int k) { return desc + dsz * 2 * (size_t)np * k; };
    CK(h, cudaMemsetAsync(status, 0, sizeof(int) * 2 * (size_t)n_mv * np, h->stream));

    std::vector<CrossDrvDesc> cd(np);
    auto drv = [&](int kind, auto &&fill) -> int {
        for (int i = 0; i < np; ++i) {
            XProb &x = xp[i];
            const weno_tt_cross_problem &P = probs[i];
            CrossDrvDesc &c = cd[i];
            c = CrossDrvDesc{};
            for (int m = 0; m < 3; ++m) c.n[m] = x.n[m];
            c.r1 = x.r1;
            c.r2 = x.r2;
            c.fp64 = fp64 ? 1 : 0;
            c.I1 = P.I1;
            c.I2 = P.I2;
            c.J1 = P.J1;
            c.J2 = P.J2;
            c.idx = x.idx;
            fill(x, P, c);
        }
        CrossDrvDesc *dd = (CrossDrvDesc *)slot(0);
        CK(h, cudaMemcpyAsync(dd, cd.data(), sizeof(CrossDrvDesc) * np, cudaMemcpyHostToDevice, h->stream));
        CK(h, launch(h, 1, h->stream, [&] { return launch_cross_drv(dd, np, kind, h->stream); }));
        return WENO_OK;
    };
    auto evaluate = [&](int mode) -> int {
        std::vector<weno_fiber_set> fs(np);
        for (int i = 0; i < np; ++i) {
            XProb &x = xp[i];
            weno_fiber_set &f = fs[i];
            f = weno_fiber_set{};
            f.instance = i;
            f.mode = mode;
            f.flux_dir = flux_dir;
            if (mode == 0) { f.n_left = 1; f.left = nullptr; f.n_right = x.r1; f.right = x.right0; f.out = x.outL0; }
            if (mode == 1) { f.n_left = x.r1; f.left = x.left1; f.n_right = x.r2; f.right = x.right1; f.out = x.outL1; }
            if (mode == 2) { f.n_left = x.r2; f.left = x.left2; f.n_right = 1; f.right = nullptr; f.out = x.outL2; }
        }
        return weno_cross_eval(h, inst, np, fs.data(), np, fp64 ? WENO_CROSS_FP64_CHECK : 0);
    };
    int mv_call = 0;
    // QR (explicit Q) of every problem's matrix for this step, then maxvol on Q
    auto select = [&](QRPlan XProb::*qp, double *XProb::*Mp, double *XProb::*Qp, double *XProb::*Bp,
                      bool b_is_core0) -> int {
        std::vector<QRPlan *> ps;
        std::vector<ApplyReq> ar(np);
        std::vector<MaxvolDesc> md(np);
        for (int i = 0; i < np; ++i) {
            XProb &x = xp[i];
            QRPlan &q = x.*qp;
            q.A = x.*Mp;
            ps.push_back(&q);
        }
        int rr = tt_factor(h, ps, (QRDesc *)slot(1));
        if (rr) return rr;
        for (int i = 0; i < np; ++i) {
            XProb &x = xp[i];
            QRPlan &q = x.*qp;
            // explicit Q (m x k): apply to the identity, row-major; the chunk stack reuses W
            ar[i] = ApplyReq{&q, nullptr, q.k, q.k, x.Wmv, x.*Qp, q.m, q.k, 0, 1};
        }
        if ((rr = tt_apply(h, ar, (QApplyDesc *)slot(2)))) return rr;
        int mr = 1;
        for (int i = 0; i < np; ++i) {
            XProb &x = xp[i];
            QRPlan &q = x.*qp;
            double *Bout = b_is_core0 ? probs[i].core[0] : x.*Bp;
            int *st = status + 2 * ((size_t)mv_call * np + i);
            md[i] = MaxvolDesc{x.*Qp, Bout, x.Wmv, x.idx, st, st + 1, (int)q.m, q.k};
            mr = std::max(mr, q.k);
        }
        MaxvolDesc *dd = (MaxvolDesc *)slot(3);
        CK(h, cudaMemcpyAsync(dd, md.data(), sizeof(MaxvolDesc) * np, cudaMemcpyHostToDevice, h->stream));
        CK(h, launch(h, 1, h->stream, [&] { return launch_maxvol(dd, np, mr, delta, 200, h->stream); }));
        ++mv_call;
        return WENO_OK;
    };
    auto nofill = [](XProb &, const weno_tt_cross_problem &, CrossDrvDesc &) {};
    for (int it = 0; it <= sweeps; ++it) {
        // ---- left to right
        if ((r = drv(XD_PREP_L0, [](XProb &x, const weno_tt_cross_problem &, CrossDrvDesc &c) { c.right = x.right0; })))
            return r;
        if ((r = evaluate(0))) return r;
        if ((r = drv(XD_GATHER_L0, [](XProb &x, const weno_tt_cross_problem &, CrossDrvDesc &c) {
                 c.out = x.outL0;
                 c.M = x.M0;
             })))
            return r;
        if ((r = select(&XProb::q0, &XProb::M0, &XProb::Q0, &XProb::BR, true))) return r;
        if ((r = drv(XD_UPDATE_L0, nofill))) return r;
        if ((r = drv(XD_PREP_L1, [](XProb &x, const weno_tt_cross_problem &, CrossDrvDesc &c) {
                 c.left = x.left1;
                 c.right = x.right1;
             })))
            return r;
        if ((r = evaluate(1))) return r;
        if ((r = drv(XD_GATHER_L1, [](XProb &x, const weno_tt_cross_problem &, CrossDrvDesc &c) {
                 c.out = x.outL1;
                 c.M = x.M1;
             })))
            return r;
        if ((r = select(&XProb::q1, &XProb::M1, &XProb::Q1, &XProb::B1, false))) return r;
        if ((r = drv(XD_UPDATE_L1, [](XProb &x, const weno_tt_cross_problem &P, CrossDrvDesc &c) {
                 c.B = x.B1;
                 c.core = P.core[1];
             })))
            return r;
        if ((r = drv(XD_PREP_L2, [](XProb &x, const weno_tt_cross_problem &, CrossDrvDesc &c) { c.left = x.left2; })))
            return r;
        if ((r = evaluate(2))) return r;
        if ((r = drv(XD_GATHER_L2, [](XProb &x, const weno_tt_cross_problem &P, CrossDrvDesc &c) {
                 c.out = x.outL2;
                 c.M = x.MR2;
                 c.core = P.core[2];
             })))
            return r;
        if (it == sweeps) break;
        // ---- right to left
        if ((r = select(&XProb::qr2, &XProb::MR2, &XProb::QR2, &XProb::BR, false))) return r;
        if ((r = drv(XD_UPDATE_R2, nofill))) return r;
        if ((r = drv(XD_PREP_L1, [](XProb &x, const weno_tt_cross_problem &, CrossDrvDesc &c) {
                 c.left = x.left1;
                 c.right = x.right1;
             })))
            return r;
        if ((r = evaluate(1))) return r;
        if ((r = drv(XD_GATHER_R1, [](XProb &x, const weno_tt_cross_problem &, CrossDrvDesc &c) {
                 c.out = x.outL1;
                 c.M = x.MR1;
             })))
            return r;
        if ((r = select(&XProb::qr1, &XProb::MR1, &XProb::QR1, &XProb::BR, false))) return r;
        if ((r = drv(XD_UPDATE_R1, nofill))) return r;
    }
    std::vector<int> st(2 * (size_t)n_mv * np);
    CK(h, cudaMemcpyAsync(st.data(), status, sizeof(int) * st.size(), cudaMemcpyDeviceToHost, h->stream));
    CK(h, cudaStreamSynchronize(h->stream));
    for (size_t k = 0; k < st.size(); k += 2)
        if (st[k]) return fail(h, WENO_ERR_ARG, "weno_tt_cross: a fiber matrix had rank below the cross rank");
    return WENO_OK;
}
