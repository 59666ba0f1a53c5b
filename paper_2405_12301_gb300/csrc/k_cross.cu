// k_cross.cu -- pointwise WENO5-JS residual at TT-cross sample points
// (Sec. 4.2-4.3, Algorithms 1 and 2), evaluated from TT cores (Eq. TT_def).
//
// A fiber set of one instance is every sample (l, i, r): left multi-index l
// over the modes before the sweep mode m, index i of mode m, right
// multi-index r over the modes after it.  The value of field f at a sample is
// L_l G_m(i) R_r with L_l = G_0(.)..G_{m-1}(.) and R_r = G_{m+1}(.)..G_2(.).
// The residual in flux direction fd needs the 7-point stencil along fd, which
// moves the left vector (fd < m), the core index i (fd = m) or the right
// vector (fd > m).
//
// Two launches:
//   k_cross_vecs  contracts every left and right vector of every set once,
//                 the 7 shifted ones where the stencil moves that side (FP32:
//                 stored as differences from the centre vector, so rounding
//                 scales with the variation along the stencil);
//   k_cross       persistent; a work item fixes one index of the side the
//                 stencil does not move (r for fd <= m, l for fd > m).  For each
//                 chunk of samples (32 to 128, per variant) it contracts the
//                 core rows G_m(i) with that fixed vector once into shared
//                 memory; every sample (v, i) of the other side's index v
//                 then needs only 7 dot products per field, followed by the
//                 LF split fluxes at the 7 points and WENO5(+/-) at the two
//                 interfaces of the sample.
// Ghost rows (Sec. 4.5) are mapped by the boundary rule of fd.
#include "weno_dev.cuh"
#include "weno_internal.h"
#include "cross_internal.h"

namespace wg {

constexpr int XT = 256;       // threads per CTA of k_cross_vecs
constexpr int VP = 32;        // padded vector length (largest rank)
constexpr int CS = VP + 4;    // shared-memory row stride: float4 reads of 8 consecutive rows hit distinct banks
// FP32, stencil along the fiber: varying indices per block of the point-flux
// path, so that each of its phases is one pass of the CTA's threads
constexpr int fiber_vb(int threads, int chunk) { return threads / (chunk + 6) > 0 ? threads / (chunk + 6) : 1; }
constexpr int FLS = 11;       // floats per point of the fiber path's split fluxes (10, padded odd:
                              // consecutive points of a warp fall on distinct banks)
// k_cross is compiled for several (threads per CTA, samples per chunk) pairs;
// the autotuner of api_cross.cu picks one, and the persistent grid size, per
// workload class.  Until then variant 5 at 3 CTAs per SM runs: held to 80
// registers it keeps 24 warps per SM, where the unbounded builds (225
// registers) fit one CTA per SM whatever grid is asked for.
// minb > 1 asks the compiler for registers that fit minb CTAs per SM.
struct CrossVariant { int threads, chunk, minb; };
constexpr CrossVariant kCrossVariants[] = {{256, 64, 1}, {256, 32, 1}, {128, 64, 1}, {128, 32, 1},
                                           {256, 128, 1}, {256, 64, 3}, {128, 64, 6}};
constexpr int kNumCrossVariants = sizeof(kCrossVariants) / sizeof(kCrossVariants[0]);
static_assert(kCrossVariants[5].threads == 256 && kCrossVariants[5].chunk == 64 && kCrossVariants[5].minb == 3,
              "cross_default names variant 5");

template <typename T> __device__ __forceinline__ T cvtf(float x) { return (T)x; }

// Index along mode m after the boundary rule of that mode.
__device__ __forceinline__ int xmap(const CrossInst &in, int m, int c, bool &flip)
{
    return ghost_source(c, in.n[m], in.bc[m][0], in.bc[m][1], flip);
}

// Entry a of the left vector of field f for multi-index lidx (modes < mode),
// with the index of mode fd moved by s (s = 0: the centre).
template <typename T>
__device__ T left_entry(const CrossInst &in, int mode, const int *lidx, int f, int a, int fd, int s, bool &flip)
{
    flip = false;
    int i0 = lidx[0];
    if (fd == 0 && s != 0) i0 = xmap(in, 0, i0 + s, flip);
    const int r1 = in.r[0];
    if (mode == 1) return cvtf<T>(__ldg(in.core[f][0] + (long long)i0 * r1 + a));
    int i1 = lidx[1];
    if (fd == 1 && s != 0) i1 = xmap(in, 1, i1 + s, flip);
    const int r2 = in.r[1];
    const float *g0 = in.core[f][0] + (long long)i0 * r1;
    const float *g1 = in.core[f][1] + (long long)i1 * r1 * r2 + a;
    T acc = T(0);
    for (int b = 0; b < r1; ++b) acc += cvtf<T>(__ldg(g0 + b)) * cvtf<T>(__ldg(g1 + b * r2));
    return acc;
}

// Entry b of the right vector of field f for multi-index ridx (modes > mode).
template <typename T>
__device__ T right_entry(const CrossInst &in, int mode, const int *ridx, int f, int b, int fd, int s, bool &flip)
{
    flip = false;
    const int r1 = in.r[0], r2 = in.r[1];
    if (mode == 1) {
        int k = ridx[0];
        if (fd == 2 && s != 0) k = xmap(in, 2, k + s, flip);
        return cvtf<T>(__ldg(in.core[f][2] + (long long)k * r2 + b));
    }
    int j = ridx[0], k = ridx[1];
    if (fd == 1 && s != 0) j = xmap(in, 1, j + s, flip);
    if (fd == 2 && s != 0) k = xmap(in, 2, k + s, flip);
    const float *g1 = in.core[f][1] + (long long)j * r1 * r2 + (long long)b * r2;
    const float *g2 = in.core[f][2] + (long long)k * r2;
    T acc = T(0);
    for (int c = 0; c < r2; ++c) acc += cvtf<T>(__ldg(g1 + c)) * cvtf<T>(__ldg(g2 + c));
    return acc;
}

// ---------------------------------------------------------------- vectors
// Lvec of a set: [n_left][nsl][5][VP], Rvec: [n_right][nsr][5][VP]; ns = 7
// holds s = -3..3 (centre at 3), ns = 1 the centre only.  One CTA per set.
template <bool F64>
__global__ void __launch_bounds__(XT) k_cross_vecs(const CrossArgs A)
{
    using T = typename std::conditional<F64, double, float>::type;
    const CrossSet &S = A.sets[blockIdx.x];
    const CrossInst &in = A.inst[S.inst];
    const int mode = S.mode, fd = S.fd;
    T *vec = reinterpret_cast<T *>(A.vecs);
    __shared__ int bad;
    if (threadIdx.x == 0) bad = 0;
    __syncthreads();
    // index check: a bad multi-index marks the set (its samples are skipped, never read)
    for (long long u = threadIdx.x; u < S.n_left * mode; u += XT)
        if ((unsigned)S.left[u] >= (unsigned)in.n[u % mode]) bad = 1;
    for (long long u = threadIdx.x; u < S.n_right * (2 - mode); u += XT)
        if ((unsigned)S.right[u] >= (unsigned)in.n[mode + 1 + u % (2 - mode)]) bad = 1;
    __syncthreads();
    if (threadIdx.x == 0) A.bad[blockIdx.x] = bad;
    if (bad) {
        if (threadIdx.x == 0) atomicOr(A.status, ST_BADINDEX);
        return;
    }
    const int rl = mode == 0 ? 1 : in.r[mode - 1];
    const int rr = mode == 2 ? 1 : in.r[mode];
    for (int side = 0; side < 2; ++side) {
        const long long nidx = side == 0 ? S.n_left : S.n_right;
        const int ns = side == 0 ? S.nsl : S.nsr;
        const int len = side == 0 ? rl : rr;
        T *out = vec + (side == 0 ? S.lvec_off : S.rvec_off);
        const long long total = nidx * ns * 5 * VP;
        for (long long u = threadIdx.x; u < total; u += XT) {
            const int a = (int)(u % VP);
            const int f = (int)((u / VP) % 5);
            const int k = (int)((u / (5 * VP)) % ns);
            const long long idx = u / (5 * VP * ns);
            const int s = ns == 7 ? k - 3 : 0;
            T v = T(0);
            if (a < len) {
                if ((side == 0 && mode == 0) || (side == 1 && mode == 2)) {
                    v = T(1);  // empty side: the 1 x 1 identity
                } else {
                    bool fl;
                    v = side == 0 ? left_entry<T>(in, mode, S.left + idx * mode, f, a, fd, s, fl)
                                  : right_entry<T>(in, mode, S.right + idx * (2 - mode), f, a, fd, s, fl);
                    if (fl && f == 1 + fd) v = -v;  // mirrored ghost row: normal momentum negated
                    if (!F64 && s != 0) {
                        bool f0;
                        v -= side == 0 ? left_entry<T>(in, mode, S.left + idx * mode, f, a, fd, 0, f0)
                                       : right_entry<T>(in, mode, S.right + idx * (2 - mode), f, a, fd, 0, f0);
                    }
                }
            }
            out[u] = v;
        }
    }
}

// ------------------------------------------------------------------- main
template <bool F64, int XT, int CH, int MINB>
__global__ void __launch_bounds__(XT, MINB) k_cross(const CrossArgs A)
{
    using T = typename std::conditional<F64, double, float>::type;
    constexpr int CP = CH + 6;  // chunk points including the stencil halo
    extern __shared__ __align__(16) unsigned char dyn[];
    T *C = reinterpret_cast<T *>(dyn);        // [5][CP][CS] contracted core rows of the chunk
    T *Cref = C + 5 * CP * CS;                // [5][CS]     chunk reference row (FP32, fd == mode)
    T *fixv = Cref + 5 * CS;                  // [5][CS]     the work item's fixed vector
    // FP32, stencil along the fiber (role 1): per block of VB varying indices,
    // the split fluxes of every chunk point, the face fluxes and the reference values
    constexpr int VB = fiber_vb(XT, CH);
    float *FL = reinterpret_cast<float *>(fixv + 5 * CS);  // [VB][CP][FLS] f(+) then f(-), 5 fields
    float *FF = FL + VB * CP * FLS;                         // [VB][5][CH+1] face fluxes (doubled)
    float *CT = FF + VB * 5 * (CH + 1);                     // [VB][5]       reference state (row i0)
    __shared__ long long s_item;
    const T eps = T(4) * (T)A.eps;  // split fluxes are formed doubled: 4 eps gives twice the WENO5 value
    const double gm1 = A.gamma - 1.0;
    const T *vecs = reinterpret_cast<const T *>(A.vecs);

    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) s_item = (long long)atomicAdd(A.counter, 1ull);
        __syncthreads();
        const long long item = s_item;
        if (item >= A.n_work) break;
        int lo = 0, hi = A.n_sets - 1;  // the set holding this item
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (A.sets[mid].work_begin <= item) lo = mid;
            else hi = mid - 1;
        }
        if (A.bad[lo]) continue;
        const CrossSet &S = A.sets[lo];
        const CrossInst &in = A.inst[S.inst];
        const int mode = S.mode, fd = S.fd, n = S.n_mode;
        const int role = fd < mode ? 0 : (fd == mode ? 1 : 2);  // stencil moves: L / the core index / R
        const long long j = item - S.work_begin;                 // fixed index: r (role 0, 1) or l (role 2)
        const int rl = mode == 0 ? 1 : in.r[mode - 1];
        const int rr = mode == 2 ? 1 : in.r[mode];
        const int clen = role == 2 ? rr : rl;                    // length of a contracted row
        const int cl4 = (clen + 3) & ~3;
        const long long nvar = role == 2 ? S.n_right : S.n_left;
        const T *var = vecs + (role == 2 ? S.rvec_off : S.lvec_off);  // the varying side's vectors
        const int nsv = role == 2 ? S.nsr : S.nsl;
        const T alpha = (T)in.alpha;
        const T ih = (T)(0.5 / in.h[fd]);  // halves the doubled face fluxes
        {   // fixed vector (centre) of this work item
            const T *src = vecs + (role == 2 ? S.lvec_off + (j * S.nsl + (S.nsl == 7 ? 3 : 0)) * 5 * VP
                                             : S.rvec_off + (j * S.nsr + (S.nsr == 7 ? 3 : 0)) * 5 * VP);
            for (int u = threadIdx.x; u < 5 * VP; u += XT) fixv[(u / VP) * CS + u % VP] = src[u];
        }
        const long long outstride_v = role == 2 ? 1 : (long long)n * S.n_right;   // along the varying index
        const long long outbase_j = role == 2 ? j * (long long)n * S.n_right : j;  // fixed index offset
        T *out = reinterpret_cast<T *>(S.out);
        __syncthreads();

        for (int i0 = 0; i0 < n; i0 += CH) {
            const int cn = n - i0 < CH ? n - i0 : CH;             // samples in this chunk
            const int p0 = role == 1 ? i0 - 3 : i0;               // first chunk point
            const int np = role == 1 ? cn + 6 : cn;
            // chunk reference row (FP32, stencil along the fiber): G(i0) . R
            if (!F64 && role == 1) {
                for (int u = threadIdx.x; u < 5 * cl4; u += XT) {
                    const int f = u / cl4, x = u - f * cl4;
                    T acc = T(0);
                    if (x < clen) {
                        const float *g = in.core[f][mode] + ((long long)i0 * rl + x) * rr;
                        for (int y = 0; y < rr; ++y) acc += cvtf<T>(__ldg(g + y)) * fixv[f * CS + y];
                    }
                    Cref[f * CS + x] = acc;
                }
                __syncthreads();
            }
            // contracted rows: role 0/1: C[p][a] = G(p)[a][:] . R ; role 2: C[p][b] = L . G(p)[:][b]
            // (rows zero-padded to a multiple of 4 entries for the float4 reads below)
            for (int u = threadIdx.x; u < 5 * np * cl4; u += XT) {
                const int f = u / (np * cl4);
                const int rem = u - f * np * cl4;
                const int pp = rem / cl4, x = rem - pp * cl4;
                if (x >= clen) {
                    C[(f * CP + pp) * CS + x] = T(0);
                    continue;
                }
                bool flip = false;
                int c = p0 + pp;
                if (role == 1) c = xmap(in, fd, c, flip);
                const float *g = in.core[f][mode] + (long long)c * rl * rr;
                T acc = T(0);
                if (role == 2) {
                    for (int y = 0; y < rl; ++y) acc += fixv[f * CS + y] * cvtf<T>(__ldg(g + y * rr + x));
                } else if (!F64 && role == 1) {
                    const float *g0 = in.core[f][mode] + (long long)i0 * rl * rr;
                    for (int y = 0; y < rr; ++y)
                        acc += (__ldg(g + x * rr + y) - __ldg(g0 + x * rr + y)) * fixv[f * CS + y];
                } else {
                    for (int y = 0; y < rr; ++y) acc += cvtf<T>(__ldg(g + x * rr + y)) * fixv[f * CS + y];
                }
                if (flip && f == 1 + fd) acc = F64 ? -acc : -acc - T(2) * Cref[f * CS + x];
                C[(f * CP + pp) * CS + x] = acc;
            }
            __syncthreads();

            if constexpr (!F64) if (role == 1) {
                // The stencil moves along the fiber: neighbouring samples of one
                // varying index share six of their seven points and one of their two
                // faces, so each point's split flux and each face's WENO5(+/-) is
                // formed once per block of VB varying indices (the values are the
                // ones the per-sample path forms: the same dot products, split
                // fluxes relative to row i0, and weno5_pm of the same windows).
                for (long long vb0 = 0; vb0 < nvar; vb0 += VB) {
                    // reference values (row i0) of the block's varying indices
                    for (int u = threadIdx.x; u < VB * 5; u += XT) {
                        const long long v = vb0 + u / 5;
                        const int f = u % 5;
                        float racc = 0.0f;
                        if (v < nvar) {
                            const float *lv = reinterpret_cast<const float *>(var) + (v * nsv) * 5 * VP + f * VP;
                            float2 ra2 = bc2(0.0f);
                            for (int x = 0; x < cl4; x += 4) {
                                const float4 l4 = *reinterpret_cast<const float4 *>(lv + x);
                                const float4 r4 = *reinterpret_cast<const float4 *>(reinterpret_cast<const float *>(Cref) + f * CS + x);
                                ra2 = fma2(make_float2(l4.z, l4.w), make_float2(r4.z, r4.w),
                                           fma2(make_float2(l4.x, l4.y), make_float2(r4.x, r4.y), ra2));
                            }
                            racc = ra2.x + ra2.y;
                        }
                        CT[u] = racc;
                    }
                    __syncthreads();
                    // split fluxes of every chunk point
                    for (int u = threadIdx.x; u < VB * np; u += XT) {
                        const int vl = u / np, pp = u - vl * np;
                        const long long v = vb0 + vl;
                        if (v >= nvar) continue;
                        const float *lvb = reinterpret_cast<const float *>(var) + (v * nsv) * 5 * VP;
                        float dq[5];
#pragma unroll
                        for (int f = 0; f < 5; ++f) {
                            const float *lv = lvb + f * VP;
                            const float *crow = reinterpret_cast<const float *>(C) + (f * CP + pp) * CS;
                            float2 a2 = bc2(0.0f);
                            for (int x = 0; x < cl4; x += 4) {
                                const float4 l4 = *reinterpret_cast<const float4 *>(lv + x);
                                const float4 c4 = *reinterpret_cast<const float4 *>(crow + x);
                                a2 = fma2(make_float2(l4.z, l4.w), make_float2(c4.z, c4.w),
                                          fma2(make_float2(l4.x, l4.y), make_float2(c4.x, c4.y), a2));
                            }
                            dq[f] = a2.x + a2.y;
                        }
                        RefState<3> rs;
                        const float *ct = CT + vl * 5;
#pragma unroll
                        for (int f = 0; f < 5; ++f) { rs.hi[f] = ct[f]; rs.lo[f] = 0.0f; }
                        {
                            const float ir = 1.0f / ct[0];
                            float ke = 0.0f;
                            rs.rho = ct[0];
#pragma unroll
                            for (int e = 0; e < 3; ++e) {
                                rs.m[e] = ct[1 + e];
                                rs.u[e] = ct[1 + e] * ir;
                                ke += rs.m[e] * rs.u[e];
                            }
                            rs.H = ct[4] + (float)gm1 * (ct[4] - 0.5f * ke);
                        }
                        float a5[5], b5[5];
                        if (fd == 0) split_flux_diff<3, 0, true>(dq, rs, (float)alpha, (float)gm1, a5, b5);
                        else if (fd == 1) split_flux_diff<3, 1, true>(dq, rs, (float)alpha, (float)gm1, a5, b5);
                        else split_flux_diff<3, 2, true>(dq, rs, (float)alpha, (float)gm1, a5, b5);
                        float *fl = FL + (vl * CP + pp) * FLS;
#pragma unroll
                        for (int f = 0; f < 5; ++f) { fl[f] = a5[f]; fl[5 + f] = b5[f]; }
                    }
                    __syncthreads();
                    // face fluxes j = 0..cn (face j lies before sample j)
                    for (int u = threadIdx.x; u < VB * (cn + 1); u += XT) {
                        const int vl = u / (cn + 1), j = u - vl * (cn + 1);
                        if (vb0 + vl >= nvar) continue;
                        const float *fl = FL + (vl * CP + j) * FLS;
#pragma unroll
                        for (int f = 0; f < 5; ++f) {
                            const float *P = fl + f, *M = fl + 5 + f;  // point j + k at [k * FLS]
                            FF[(vl * 5 + f) * (CH + 1) + j] = weno5_pm(
                                make_float2(P[0], M[5 * FLS]), make_float2(P[FLS], M[4 * FLS]),
                                make_float2(P[2 * FLS], M[3 * FLS]), make_float2(P[3 * FLS], M[2 * FLS]),
                                make_float2(P[4 * FLS], M[FLS]), (float)eps);
                        }
                    }
                    __syncthreads();
                    for (int u = threadIdx.x; u < VB * cn; u += XT) {
                        const int vl = u / cn, ii = u - vl * cn;
                        const long long v = vb0 + vl;
                        if (v >= nvar) continue;
                        const int i = i0 + ii;
#pragma unroll
                        for (int f = 0; f < 5; ++f) {
                            const float *F = FF + (vl * 5 + f) * (CH + 1);
                            const long long o = (long long)f * S.n_left * n * S.n_right + outbase_j + v * outstride_v +
                                                (long long)i * S.n_right;
                            out[o] = -(F[ii + 1] - F[ii]) * ih;
                        }
                    }
                    // (the next block's first writes go to CT and FL, which no thread
                    // reads after the barrier above)
                }
                __syncthreads();
                continue;
            }
            // samples (v, i): 7 stencil values per field, split fluxes, two interfaces
            for (long long u = threadIdx.x; u < nvar * CH; u += XT) {
                const long long v = u / CH;
                const int ii = (int)(u - v * CH);
                if (ii >= cn) continue;
                T q7[5][7];  // FP64: values; FP32: differences from the reference state
                T ctr[5];    // FP32: reference state
#pragma unroll
                for (int f = 0; f < 5; ++f) {
                    T acc[7];
#pragma unroll
                    for (int k = 0; k < 7; ++k) acc[k] = T(0);
                    if (role == 1) {  // the same vector against the 7 rows i-3..i+3
                        const T *lv = var + (v * nsv) * 5 * VP + f * VP;
                        T racc = T(0);
                        if constexpr (F64) {
                            for (int x = 0; x < clen; ++x) {
                                const T lx = lv[x];
#pragma unroll
                                for (int k = 0; k < 7; ++k) acc[k] += lx * C[(f * CP + ii + k) * CS + x];
                            }
                        } else {
                            // f32x2: even and odd entries accumulate in the two lanes (one issue
                            // slot per two FMAs), summed at the end
                            float2 a2[7], ra2 = bc2(0.0f);
#pragma unroll
                            for (int k = 0; k < 7; ++k) a2[k] = bc2(0.0f);
                            for (int x = 0; x < cl4; x += 4) {
                                const float4 l4 = *reinterpret_cast<const float4 *>(lv + x);
                                const float2 lxy = make_float2(l4.x, l4.y), lzw = make_float2(l4.z, l4.w);
#pragma unroll
                                for (int k = 0; k < 7; ++k) {
                                    const float4 c4 = *reinterpret_cast<const float4 *>(C + (f * CP + ii + k) * CS + x);
                                    a2[k] = fma2(lzw, make_float2(c4.z, c4.w), fma2(lxy, make_float2(c4.x, c4.y), a2[k]));
                                }
                                const float4 r4 = *reinterpret_cast<const float4 *>(Cref + f * CS + x);
                                ra2 = fma2(lzw, make_float2(r4.z, r4.w), fma2(lxy, make_float2(r4.x, r4.y), ra2));
                            }
#pragma unroll
                            for (int k = 0; k < 7; ++k) acc[k] = a2[k].x + a2[k].y;
                            racc = ra2.x + ra2.y;
                        }
                        ctr[f] = racc;
#pragma unroll
                        for (int k = 0; k < 7; ++k) q7[f][k] = acc[k];
                    } else {          // the 7 shifted vectors against the row of sample i
                        const T *vv = var + (v * 7) * 5 * VP + f * VP;
                        const T *crow = C + (f * CP + ii) * CS;
                        if constexpr (F64) {
                            for (int x = 0; x < clen; ++x) {
                                const T cx = crow[x];
#pragma unroll
                                for (int k = 0; k < 7; ++k) acc[k] += vv[k * 5 * VP + x] * cx;
                            }
                        } else {  // f32x2 even / odd partial sums, as above
                            float2 a2[7];
#pragma unroll
                            for (int k = 0; k < 7; ++k) a2[k] = bc2(0.0f);
                            for (int x = 0; x < cl4; x += 4) {
                                const float4 c4 = *reinterpret_cast<const float4 *>(crow + x);
                                const float2 cxy = make_float2(c4.x, c4.y), czw = make_float2(c4.z, c4.w);
#pragma unroll
                                for (int k = 0; k < 7; ++k) {
                                    const float4 w4 = *reinterpret_cast<const float4 *>(vv + k * 5 * VP + x);
                                    a2[k] = fma2(make_float2(w4.z, w4.w), czw, fma2(make_float2(w4.x, w4.y), cxy, a2[k]));
                                }
                            }
#pragma unroll
                            for (int k = 0; k < 7; ++k) acc[k] = a2[k].x + a2[k].y;
                        }
                        ctr[f] = acc[3];
#pragma unroll
                        for (int k = 0; k < 7; ++k) q7[f][k] = (F64 || k != 3) ? acc[k] : T(0);
                    }
                }
                T fp7[5][7], fm7[5][7];
                if constexpr (F64) {
#pragma unroll
                    for (int k = 0; k < 7; ++k) {
                        double qd[5], a5[5], b5[5];
#pragma unroll
                        for (int f = 0; f < 5; ++f) qd[f] = q7[f][k];
                        if (fd == 0) split_flux_f64<3, 0, true>(qd, (double)alpha, gm1, a5, b5);
                        else if (fd == 1) split_flux_f64<3, 1, true>(qd, (double)alpha, gm1, a5, b5);
                        else split_flux_f64<3, 2, true>(qd, (double)alpha, gm1, a5, b5);
#pragma unroll
                        for (int f = 0; f < 5; ++f) { fp7[f][k] = a5[f]; fm7[f][k] = b5[f]; }
                    }
                } else {
                    RefState<3> rs;
#pragma unroll
                    for (int f = 0; f < 5; ++f) { rs.hi[f] = ctr[f]; rs.lo[f] = 0.0f; }
                    {
                        const float ir = 1.0f / ctr[0];
                        float ke = 0.0f;
                        rs.rho = ctr[0];
#pragma unroll
                        for (int e = 0; e < 3; ++e) {
                            rs.m[e] = ctr[1 + e];
                            rs.u[e] = ctr[1 + e] * ir;
                            ke += rs.m[e] * rs.u[e];
                        }
                        rs.H = ctr[4] + (float)gm1 * (ctr[4] - 0.5f * ke);
                    }
#pragma unroll
                    for (int k = 0; k < 7; ++k) {
                        float dq[5], a5[5], b5[5];
#pragma unroll
                        for (int f = 0; f < 5; ++f) dq[f] = q7[f][k];
                        if (fd == 0) split_flux_diff<3, 0, true>(dq, rs, alpha, (float)gm1, a5, b5);
                        else if (fd == 1) split_flux_diff<3, 1, true>(dq, rs, alpha, (float)gm1, a5, b5);
                        else split_flux_diff<3, 2, true>(dq, rs, alpha, (float)gm1, a5, b5);
#pragma unroll
                        for (int f = 0; f < 5; ++f) { fp7[f][k] = a5[f]; fm7[f][k] = b5[f]; }
                    }
                }
                const int i = i0 + ii;
#pragma unroll
                for (int f = 0; f < 5; ++f) {
                    const T *P = fp7[f], *M = fm7[f];
                    T Flo, Fhi;
                    if constexpr (F64) {
                        Flo = weno5<T>(P[0], P[1], P[2], P[3], P[4], eps) + weno5<T>(M[5], M[4], M[3], M[2], M[1], eps);
                        Fhi = weno5<T>(P[1], P[2], P[3], P[4], P[5], eps) + weno5<T>(M[6], M[5], M[4], M[3], M[2], eps);
                    } else {  // WENO(+) and the mirrored WENO(-) of an interface as one f32x2 pair
                        Flo = weno5_pm(make_float2(P[0], M[5]), make_float2(P[1], M[4]), make_float2(P[2], M[3]),
                                       make_float2(P[3], M[2]), make_float2(P[4], M[1]), eps);
                        Fhi = weno5_pm(make_float2(P[1], M[6]), make_float2(P[2], M[5]), make_float2(P[3], M[4]),
                                       make_float2(P[4], M[3]), make_float2(P[5], M[2]), eps);
                    }
                    // out[f][l][i][r]: role 0/1 fix r (= j) and vary l (= v); role 2 fixes l, varies r
                    const long long o = (long long)f * S.n_left * n * S.n_right + outbase_j + v * outstride_v +
                                        (long long)i * S.n_right;
                    out[o] = -(Fhi - Flo) * ih;
                }
            }
            __syncthreads();
        }
    }
}

static size_t cross_dyn_bytes(bool f64, int threads, int chunk)
{
    const size_t e = f64 ? sizeof(double) : sizeof(float);
    const int VB = fiber_vb(threads, chunk);
    const size_t fiber = f64 ? 0 : sizeof(float) * (size_t)(VB * (chunk + 6) * FLS + VB * 5 * (chunk + 1) + VB * 5);
    return e * (size_t)(5 * (chunk + 6) * CS + 2 * 5 * CS) + fiber;
}

int cross_vec_len() { return VP; }
int cross_num_variants() { return kNumCrossVariants; }
void cross_default(int *variant, int *ctas_per_sm)
{
    *variant = 5;  // {256, 64, 3}
    *ctas_per_sm = 3;
}
void cross_variant(int v, int *threads, int *chunk)
{
    *threads = kCrossVariants[v].threads;
    *chunk = kCrossVariants[v].chunk;
}

template <bool F64, int V>
static cudaError_t set_attr()
{
    constexpr int XT_ = kCrossVariants[V].threads, CH_ = kCrossVariants[V].chunk, MB_ = kCrossVariants[V].minb;
    return cudaFuncSetAttribute(k_cross<F64, XT_, CH_, MB_>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)cross_dyn_bytes(F64, XT_, CH_));
}

// Shared-memory limits of every variant, set once before any launch (and so
// never inside a stream capture).
cudaError_t cross_set_attributes()
{
    static bool done = false;
    if (done) return cudaSuccess;
    cudaError_t e = cudaSuccess, r;
#define X(V) \
    if ((r = set_attr<false, V>()) != cudaSuccess) e = r; \
    if ((r = set_attr<true, V>()) != cudaSuccess) e = r;
    X(0) X(1) X(2) X(3) X(4) X(5) X(6)
#undef X
    if (e == cudaSuccess) done = true;
    return e;
}

template <bool F64, int V>
static cudaError_t launch_main(const CrossArgs &a, long long blocks, cudaStream_t s)
{
    constexpr int XT_ = kCrossVariants[V].threads, CH_ = kCrossVariants[V].chunk, MB_ = kCrossVariants[V].minb;
    k_cross<F64, XT_, CH_, MB_><<<(unsigned)blocks, XT_, cross_dyn_bytes(F64, XT_, CH_), s>>>(a);
    return cudaGetLastError();
}

// variant: index into kCrossVariants; ctas_per_sm: persistent grid = SM count x that
// (capped by the number of work items).
cudaError_t launch_cross(const CrossArgs &a, int variant, int ctas_per_sm, cudaStream_t s)
{
    if (variant < 0 || variant >= kNumCrossVariants || ctas_per_sm < 1) return cudaErrorInvalidValue;
    cudaError_t ea = cross_set_attributes();
    if (ea != cudaSuccess) return ea;
    if (a.fp64) k_cross_vecs<true><<<a.n_sets, XT, 0, s>>>(a);
    else k_cross_vecs<false><<<a.n_sets, XT, 0, s>>>(a);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    long long blocks = (long long)sm_count() * ctas_per_sm;
    if (blocks > a.n_work) blocks = a.n_work;
    if (blocks < 1) blocks = 1;
#define X(V)                                                                             \
    if (variant == V) return a.fp64 ? launch_main<true, V>(a, blocks, s) : launch_main<false, V>(a, blocks, s);
    X(0) X(1) X(2) X(3) X(4) X(5) X(6)
#undef X
    return cudaErrorInvalidValue;
}

int cross_max_rank() { return VP; }

}  // namespace wg
