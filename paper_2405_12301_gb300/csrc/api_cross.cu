// api_cross.cu -- the C ABI of the pointwise residual at TT-cross samples
// (weno_cross_eval), its autotuner and tuning cache, and the CUDA graphs it
// replays for repeated descriptors.
#include "api_ctx.h"

using namespace wg;

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
    cross_default(&variant, &cpsm);
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
