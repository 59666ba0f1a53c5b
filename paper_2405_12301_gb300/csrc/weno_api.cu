// weno_api.cu -- the C ABI (include/weno_gb300.h) of the grid path: handles,
// scratch, argument checking and the launch sequences of a residual, a stage,
// a step and a CUDA-graph-captured run; kernel timing; the shared helpers of
// api_ctx.h.  Cross evaluation lives in api_cross.cu, the TT algebra in
// api_tt.cu.  No arithmetic of the scheme lives here.
#include "api_ctx.h"

using namespace wg;

cudaEvent_t wg::get_event(weno_ctx *h)
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

static thread_local std::string g_init_error;

namespace wg {
// Error text for calls made without a handle (read back by weno_last_error(NULL)).
void set_thread_error(const std::string &msg) { g_init_error = msg; }
}  // namespace wg

int wg::fail(weno_ctx *h, int code, const std::string &msg)
{
    if (h) h->err = msg;
    else g_init_error = msg;
    return code;
}



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
    cudaFree(h->bcs_dev);
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
             alloc((void **)&h->sums_dev, sizeof(double) * h->nf) &&
             alloc((void **)&h->bcs_dev, sizeof(p.bc_state));
    }
    if (!ok) {
        free_all(h);
        delete h;
        return fail(nullptr, WENO_ERR_CUDA, "weno_init: device allocation failed");
    }
    Ctl c{};
    c.max_steps = LLONG_MAX;
    if ((h->bcs_dev && cudaMemcpyAsync(h->bcs_dev, p.bc_state, sizeof(p.bc_state), cudaMemcpyHostToDevice,
                                       h->stream) != cudaSuccess) ||
        cudaMemcpyAsync(h->ctl, &c, sizeof(Ctl), cudaMemcpyHostToDevice, h->stream) != cudaSuccess ||
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
    // work already queued on the old stream (a graph replay included) finishes
    // before its graphs go away
    CK(h, cudaStreamSynchronize(h->stream));
    if (h->gexec) {
        cudaGraphExecDestroy(h->gexec);
        h->gexec = nullptr;
        h->g_U = nullptr;
        h->g_steps = 0;
    }
    for (auto &g : h->xgraphs) {
        cudaGraphExecDestroy(g.exec);
        cudaFree(g.buf);
    }
    h->xgraphs.clear();
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
    for (int d = 0; d < 3; ++d) {
        a.inv_h_f[d] = (float)a.inv_h[d];
        const double x = -(2.0 / 3.0) * a.inv_h[d];
        const float hi = (float)x;
        a.ih23[d] = make_float2(hi, (float)(x - (double)hi));
    }
    a.acc = h->acc;
    a.bcs = h->bcs_dev;
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
        if (bulk(h)) CK(h, launch(h, 4, s, [&] { return launch_xy2(last, a, s); }));
        else CK(h, launch(h, 4, s, [&] { return launch_xy(2, false, last, a, s); }));
    } else {
        CK(h, launch(h, 2, s, [&] { return launch_xy(3, bulk(h), EPI_STORE, a, s); }));
        if (bulk(h)) CK(h, launch(h, 5, s, [&] { return launch_z2(last, a, s); }));
        else CK(h, launch(h, 5, s, [&] { return launch_z(false, last, a, s); }));
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
    // FP32-bulk (2D and 3D) keeps the split of U^n in S1 and the FP32 increments in S2
    const bool inc = h->dim >= 2 && bulk(h) && h->p.model == WENO_MODEL_EULER;
    // 2D: Delta_1 and Delta_2 as float [cell][4] one after the other; 3D: their
    // float4 planes (first four fields) one after the other, then their E planes
    float *delta[2] = {reinterpret_cast<float *>(h->S2), reinterpret_cast<float *>(h->S2) + 4 * h->N};
    float *delta1[2] = {reinterpret_cast<float *>(h->S2) + 8 * h->N, reinterpret_cast<float *>(h->S2) + 9 * h->N};
    for (int k = 0; k < 3; ++k) {
        SweepArgs a = base_args(h);
        a.U = inc ? U : in[k];
        a.Un = U;
        a.Uout = inc ? (k == 2 ? U : nullptr) : outs[k];
        if (inc) {
            a.hl = reinterpret_cast<float2 *>(h->S1);
            a.din = k > 0 ? delta[k - 1] : nullptr;
            a.dout = k < 2 ? delta[k] : nullptr;
            a.din1 = h->dim == 3 && k > 0 ? delta1[k - 1] : nullptr;
            a.dout1 = h->dim == 3 && k < 2 ? delta1[k] : nullptr;
        }
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

int wg::take_status(weno_ctx *h)
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

int wg::grow(weno_ctx *h, void **buf, size_t *have, size_t bytes)
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
