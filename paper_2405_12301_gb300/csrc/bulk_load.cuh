// bulk_load.cuh -- the FP32 hi/lo state of one grid point for the 3D FP32-bulk
// kernels, read either as the split of the FP64 state U (stage 1, L(U)) or as
// the stored split of U^n plus the FP32 stage increment Delta_k (stages 2 and
// 3, see the stage-state comment of k_xy2.cu; 3D keeps it as float4 planes of
// the first four fields and float planes of E).
#pragma once
#include "weno_dev.cuh"
#include "weno_internal.h"

namespace wg {

template <int NF, bool FROM_HL>
__device__ __forceinline__ void bulk_point(const SweepArgs &a, long long src, float *h, float *l)
{
    const long long N = a.N;
    if constexpr (FROM_HL && NF == 5) {  // (only the 3D kernels read the stage state)
        // planes H4, L4 (float4: rho, m_x, m_y, m_z), then H1, L1 (E); Delta as
        // a float4 plane (din) and an E plane (din1); 32-bit cell indices on
        // 64-bit plane pointers (the host keeps N below 2^32)
        const unsigned i = (unsigned)src;
        const float4 *H4 = reinterpret_cast<const float4 *>(a.hl);
        const float *H1 = reinterpret_cast<const float *>(H4 + 2 * N);
        const float4 hq = __ldg(H4 + i), lq = __ldg(H4 + N + i);
        const float4 dq = __ldg(reinterpret_cast<const float4 *>(a.din) + i);
        const float he = __ldg(H1 + i), le = __ldg(H1 + N + i), de = __ldg(a.din1 + i);
        const float2 l01 = add2(make_float2(lq.x, lq.y), make_float2(dq.x, dq.y));
        const float2 l23 = add2(make_float2(lq.z, lq.w), make_float2(dq.z, dq.w));
        h[0] = hq.x;
        h[1] = hq.y;
        h[2] = hq.z;
        h[3] = hq.w;
        h[4] = he;
        l[0] = l01.x;
        l[1] = l01.y;
        l[2] = l23.x;
        l[3] = l23.y;
        l[4] = le + de;
    } else if constexpr (!FROM_HL) {
        double u[NF];
#pragma unroll
        for (int f = 0; f < NF; ++f) u[f] = __ldg(a.U + f * N + src);
#pragma unroll
        for (int f = 0; f < NF; ++f) split_f64(u[f], h[f], l[f]);
    }
}

// The 3D stage state written by the stage-1 epilogue: the split of U^n at one cell.
__device__ __forceinline__ void bulk_store_hl(const SweepArgs &a, long long cell, const float *h, const float *l)
{
    const long long N = a.N;
    float4 *H4 = reinterpret_cast<float4 *>(a.hl);
    float *H1 = reinterpret_cast<float *>(H4 + 2 * N);
    const unsigned i = (unsigned)cell;
    H4[i] = make_float4(h[0], h[1], h[2], h[3]);
    H4[N + i] = make_float4(l[0], l[1], l[2], l[3]);
    H1[i] = h[4];
    H1[N + i] = l[4];
}

// A ghost of an inflow side: the given conserved state, split.
template <int NF>
__device__ __forceinline__ void bulk_state(const double *st, float *h, float *l)
{
#pragma unroll
    for (int f = 0; f < NF; ++f) split_f64(st[f], h[f], l[f]);
}

}  // namespace wg
