// k_maxvol.cu -- batched maxvol (the maximum-volume row selection that picks
// the cross indices of TT-cross, Sec. 3 "TT-cross Interpolation"), FP64, three
// launches per batch (phases 1 and 3 one CTA per n x r matrix, r <= 64; the
// product of phase 2 spread over many CTAs):
//   1. the r pivot rows of Gaussian elimination with partial pivoting on a
//      working copy W (largest remaining |W[i][j]| of column j, ties to the
//      smaller row);
//   2. B = A A[I]^{-1}, with A[I] inverted by Gauss-Jordan with partial
//      pivoting in shared memory;
//   3. while max |B[i][j]| > 1 + delta (ties to the first entry in row-major
//      order): row i replaces I[j] and B -= B[:, j] (B[i, :] - e_j) / B[i][j].
// W and B live in global memory (L2-resident); every pass of phases 1 and 3 is
// one block-wide argmax and one row-parallel update.
#include <climits>

#include "weno_dev.cuh"
#include "weno_internal.h"
#include "tt_internal.h"

namespace wg {

constexpr int MV_NT = 256, MV_NW = MV_NT / 32;

// |x| as an unsigned integer: for finite x its order is the order of |x|, so
// argmaxes run on the integer pipe (FP64 compares issue at the FP64 rate).
__device__ __forceinline__ unsigned long long absbits(double x)
{
    return (unsigned long long)__double_as_longlong(x) & 0x7FFFFFFFFFFFFFFFull;
}

// Block-wide argmax of (key, i): largest key, smallest i among equal keys.
__device__ __forceinline__ void block_argmax_u(unsigned long long &k, long long &i, unsigned long long *sk, long long *si)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long ok = __shfl_xor_sync(0xFFFFFFFFu, k, o);
        const long long oi = __shfl_xor_sync(0xFFFFFFFFu, i, o);
        if (ok > k || (ok == k && oi < i)) {
            k = ok;
            i = oi;
        }
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) {
        sk[warp] = k;
        si[warp] = i;
    }
    __syncthreads();
    k = sk[0];
    i = si[0];
    for (int w = 1; w < MV_NW; ++w)
        if (sk[w] > k || (sk[w] == k && si[w] < i)) {
            k = sk[w];
            i = si[w];
        }
}

size_t maxvol_smem(int r) { return sizeof(double) * (size_t)r * (2 * r + 1) + sizeof(int) * (size_t)(r + 1); }

// Phase 1 and the inverse: one CTA per matrix.
__global__ void __launch_bounds__(MV_NT) k_maxvol_pivot(const MaxvolDesc *descs)
{
    const MaxvolDesc d = descs[blockIdx.x];
    const int n = d.n, r = d.r;
    extern __shared__ double sm[];
    double *G = sm;                                  // [r][2r]: [A[I] | identity] for Gauss-Jordan
    double *row = G + (size_t)r * 2 * r;             // [r]
    int *I = reinterpret_cast<int *>(row + r);       // [r]
    __shared__ unsigned long long sk[MV_NW];
    __shared__ long long si[MV_NW];
    __shared__ int s_fail;
    __shared__ unsigned chosen[MV_NMAX / 32];  // rows already picked by the pivoting
    double *W = d.W;
    const long long nr = (long long)n * r;
    if (threadIdx.x == 0) s_fail = 0;
    for (int e = threadIdx.x; e < (n + 31) / 32; e += MV_NT) chosen[e] = 0u;
    for (long long e = threadIdx.x; e < nr; e += MV_NT) W[e] = d.A[e];
    __syncthreads();

    // 1. partial pivoting; only the columns after j are updated (earlier ones are
    // never read again)
    for (int j = 0; j < r; ++j) {
        unsigned long long kmax = 0ull;
        long long bi = LLONG_MAX;
        for (int i = threadIdx.x; i < n; i += MV_NT) {
            if ((chosen[i >> 5] >> (i & 31)) & 1u) continue;
            const unsigned long long k = absbits(W[(long long)i * r + j]) + 1ull;  // 0 marks "no row"
            if (k > kmax) {  // i grows per thread, so equal keys keep the first
                kmax = k;
                bi = i;
            }
        }
        block_argmax_u(kmax, bi, sk, si);
        const int p = (int)bi;
        if (threadIdx.x == 0) {
            I[j] = p;
            chosen[p >> 5] |= 1u << (p & 31);
        }
        __syncthreads();
        const double wp = W[(long long)p * r + j];
        if (wp != 0.0) {
            for (int i = threadIdx.x; i < n; i += MV_NT) {
                if ((chosen[i >> 5] >> (i & 31)) & 1u) continue;
                double *wi = W + (long long)i * r;
                const double f = wi[j] / wp;
                for (int c = j + 1; c < r; ++c) wi[c] = fma(-f, W[(long long)p * r + c], wi[c]);
            }
        }
        __syncthreads();
    }

    // 2. B = A A[I]^{-1}: Gauss-Jordan on [A[I] | identity]
    for (int e = threadIdx.x; e < r * 2 * r; e += MV_NT) {
        const int i = e / (2 * r), c = e - i * 2 * r;
        G[e] = c < r ? d.A[(long long)I[i] * r + c] : (c - r == i ? 1.0 : 0.0);
    }
    __syncthreads();
    for (int c = 0; c < r; ++c) {
        if (threadIdx.x == 0) {
            int p = c;
            double best = fabs(G[c * 2 * r + c]);
            for (int i = c + 1; i < r; ++i)
                if (fabs(G[i * 2 * r + c]) > best) {
                    best = fabs(G[i * 2 * r + c]);
                    p = i;
                }
            if (best == 0.0) s_fail = 1;
            if (p != c)
                for (int t = 0; t < 2 * r; ++t) {
                    const double x = G[c * 2 * r + t];
                    G[c * 2 * r + t] = G[p * 2 * r + t];
                    G[p * 2 * r + t] = x;
                }
            const double inv = best == 0.0 ? 0.0 : 1.0 / G[c * 2 * r + c];
            for (int t = 0; t < 2 * r; ++t) G[c * 2 * r + t] *= inv;
        }
        __syncthreads();
        for (int i = threadIdx.x; i < r; i += MV_NT) row[i] = G[i * 2 * r + c];  // multipliers, read before any write
        __syncthreads();
        for (int e = threadIdx.x; e < r * 2 * r; e += MV_NT) {
            const int i = e / (2 * r), t = e - i * 2 * r;
            if (i == c) continue;
            G[e] = fma(-row[i], G[c * 2 * r + t], G[e]);
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) d.status[0] = s_fail;
    if (s_fail) return;
    for (int e = threadIdx.x; e < r * r; e += MV_NT) {
        const int k = e / r, c = e - k * r;
        d.Minv[e] = G[k * 2 * r + r + c];
    }
    for (int j = threadIdx.x; j < r; j += MV_NT) d.idx[j] = I[j];
}

// B = A A[I]^{-1}: the n x r by r x r product, spread over many CTAs per matrix.
__global__ void k_maxvol_b(const MaxvolDesc *descs)
{
    const MaxvolDesc &d = descs[blockIdx.y];
    if (d.status[0]) return;
    const int r = d.r;
    const long long nr = (long long)d.n * r;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < nr; e += (long long)gridDim.x * blockDim.x) {
        const long long i = e / r;
        const int c = (int)(e - i * r);
        const double *ai = d.A + i * r;
        double acc = 0.0;
        for (int k = 0; k < r; ++k) acc = fma(ai[k], d.Minv[k * r + c], acc);
        d.B[e] = acc;
    }
}

// Phase 3, the swaps: one CTA per matrix.
__global__ void __launch_bounds__(MV_NT) k_maxvol_swap(const MaxvolDesc *descs, double delta, int max_iters)
{
    const MaxvolDesc d = descs[blockIdx.x];
    if (d.status[0]) return;
    const int n = d.n, r = d.r;
    extern __shared__ double sm[];
    double *row = sm;                                // [r]
    int *I = reinterpret_cast<int *>(row + r);       // [r]
    __shared__ unsigned long long sk[MV_NW];
    __shared__ long long si[MV_NW];
    double *B = d.B;
    const long long nr = (long long)n * r;
    for (int j = threadIdx.x; j < r; j += MV_NT) I[j] = d.idx[j];
    __syncthreads();
    // 3. swaps
    int it = 0;
    for (; it < max_iters; ++it) {
        unsigned long long kmax = 0ull;
        long long bi = LLONG_MAX;
        for (long long e = threadIdx.x; e < nr; e += MV_NT) {
            const unsigned long long k = absbits(B[e]);
            if (k > kmax || bi == LLONG_MAX) {  // e grows per thread, so equal keys keep the first
                kmax = k;
                bi = e;
            }
        }
        block_argmax_u(kmax, bi, sk, si);
        if (!(__longlong_as_double((long long)kmax) > 1.0 + delta)) break;
        const int i0 = (int)(bi / r), j0 = (int)(bi - (long long)i0 * r);
        for (int c = threadIdx.x; c < r; c += MV_NT) row[c] = B[(long long)i0 * r + c] - (c == j0 ? 1.0 : 0.0);
        __syncthreads();
        const double piv = row[j0] + 1.0;
        for (int i = threadIdx.x; i < n; i += MV_NT) {
            double *bi_ = B + (long long)i * r;
            const double f = bi_[j0] / piv;
            for (int c = 0; c < r; ++c) bi_[c] = fma(-f, row[c], bi_[c]);
        }
        if (threadIdx.x == 0) I[j0] = i0;
        __syncthreads();
    }
    for (int j = threadIdx.x; j < r; j += MV_NT) d.idx[j] = I[j];
    if (threadIdx.x == 0) {
        d.status[0] = 0;
        d.swaps[0] = it;
    }
}

cudaError_t launch_maxvol(const MaxvolDesc *d, int n, int max_r, double delta, int max_iters, cudaStream_t s)
{
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(k_maxvol_pivot, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)maxvol_smem(MV_RMAX));
        if (e != cudaSuccess) return e;
        attr = true;
    }
    k_maxvol_pivot<<<n, MV_NT, maxvol_smem(max_r), s>>>(d);
    k_maxvol_b<<<dim3(64, n), 256, 0, s>>>(d);
    k_maxvol_swap<<<n, MV_NT, sizeof(double) * max_r + sizeof(int) * (max_r + 1), s>>>(d, delta, max_iters);
    return cudaGetLastError();
}

}  // namespace wg
