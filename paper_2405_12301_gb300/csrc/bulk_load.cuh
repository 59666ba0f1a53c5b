// bulk_load.cuh -- the FP32 hi/lo state of one grid point for the FP32-bulk
// kernels, read either as the split of the FP64 state U (stage 1, L(U)) or as
// the stored split of U^n plus the FP32 stage increment Delta_k (stages 2 and
// 3, see the stage-state comment of k_xy2.cu).
#pragma once
#include "weno_dev.cuh"
#include "weno_internal.h"

namespace wg {

template <int NF, bool FROM_HL>
__device__ __forceinline__ void bulk_point(const SweepArgs &a, long long src, float *h, float *l)
{
    const long long N = a.N;
    if constexpr (FROM_HL) {
        float2 q[NF];
        float d[NF];
#pragma unroll
        for (int f = 0; f < NF; ++f) {
            q[f] = __ldg(a.hl + f * N + src);
            d[f] = __ldg(a.din + f * N + src);
        }
#pragma unroll
        for (int f = 0; f < NF; ++f) {
            h[f] = q[f].x;
            l[f] = q[f].y + d[f];
        }
    } else {
        double u[NF];
#pragma unroll
        for (int f = 0; f < NF; ++f) u[f] = __ldg(a.U + f * N + src);
#pragma unroll
        for (int f = 0; f < NF; ++f) split_f64(u[f], h[f], l[f]);
    }
}

// A ghost of an inflow side: the given conserved state, split.
template <int NF>
__device__ __forceinline__ void bulk_state(const double *st, float *h, float *l)
{
#pragma unroll
    for (int f = 0; f < NF; ++f) split_f64(st[f], h[f], l[f]);
}

}  // namespace wg
