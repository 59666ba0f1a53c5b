// api_ctx.h -- private to the library: the handle behind weno_handle and the
// helpers every part of the C ABI uses (error text, the launch wrapper that
// counts launches and times kernels, scratch growth, the device status read).
// weno_api.cu defines them; api_cross.cu and api_tt.cu use them.
#pragma once
#include <algorithm>
#include <climits>
#include <cmath>
#include <cstdint>
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
    double *bcs_dev = nullptr;  // weno_params.bc_state in device memory
    int nblocks_sum = 0;
    wg::Ctl *ctl = nullptr;
    wg::Ctl *ctl_host = nullptr;  // pinned mirror for reads
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

namespace wg {

cudaEvent_t get_event(weno_ctx *h);

// Every kernel launch of the API goes through here: it counts the launch and,
// when timing is on and the stream is not being captured, brackets it with a
// CUDA event pair on the launch stream.
template <class F> inline cudaError_t launch(weno_ctx *h, int kind, cudaStream_t s, F &&f, int nk = 1)
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

// Records msg as the handle's error text (or the thread's, h == NULL) and returns code.
int fail(weno_ctx *h, int code, const std::string &msg);
// Grows a handle-owned device buffer to at least `bytes` (synchronises the stream first).
int grow(weno_ctx *h, void **buf, size_t *have, size_t bytes);
// Reads the device status word: WENO_ERR_ARG / WENO_ERR_NONPHYSICAL if a kernel latched one.
int take_status(weno_ctx *h);

}  // namespace wg

#define CK(h, call)                                                                                 \
    do {                                                                                            \
        cudaError_t e_ = (call);                                                                    \
        if (e_ != cudaSuccess)                                                                      \
            return fail((h), WENO_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_));   \
    } while (0)
