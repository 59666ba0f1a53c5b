// k_maxvol.cu -- batched maxvol (the maximum-volume row selection that picks
// the cross indices of TT-cross, Sec. 3 "TT-cross Interpolation"), FP64, three
// launches per batch:
//   1. the r pivot rows I of Gaussian elimination with partial pivoting on a
//      working copy W (largest remaining |W[i][j]| of column j, ties to the
//      smaller row); the multipliers L[i][j] overwrite column j of W, and the
//      unit lower triangular L[I] is inverted;
//   2. B = A A[I]^{-1} = L L[I]^{-1} (A = P L U, so the U factor cancels; the
//      rows I get the unit vectors exactly), spread over many CTAs per matrix;
//   3. while max |B[i][j]| > 1 + delta (ties to the first entry in row-major
//      order): row i replaces I[j] and B -= B[:, j] (B[i, :] - e_j) / B[i][j].
// Forming B from L rather than from an inverse of A[I] keeps it accurate when
// A is ill-conditioned: |L| <= 1 under partial pivoting, and the scale of
// A's columns stays in U.  Phases 1 and 3 are sequences of (argmax, rank-one
// update) steps.  Each matrix gets a thread-block cluster whose CTAs own
// contiguous slices of its rows, so the FP64 work of a large matrix spreads
// over up to 16 SMs.  Per step every CTA finds the best entry of its slice and
// stashes that entry's row in a shared-memory slot; after one cluster barrier
// every CTA reduces the slots (read through distributed shared memory) to the
// same winner and copies the winner's row from its owner.  Slots alternate
// between two buffers, so the writes of step t + 1 never meet the reads of
// step t, and the stash lets the owner update the winning row in place while
// others still read it.  The working copy is column-major (W[c][i]), so a
// warp's row-parallel accesses coalesce; it stays in L2.
#include <algorithm>
#include <climits>

#include <cooperative_groups.h>

#include "weno_dev.cuh"
#include "weno_internal.h"
#include "tt_internal.h"

namespace wg {

namespace cg = cooperative_groups;

constexpr int MV_NT = 256, MV_NW = MV_NT / 32;
// A pivot |w| <= MV_RANK_TOL r max_i |A[i][j]| counts as zero: the residual
// of a column that lies in the span of the earlier ones is a few rounding
// errors of the column's own scale (a full-rank matrix reaches it only with a
// condition number near 1 / (r MV_RANK_TOL) ~ 1e13).
constexpr double MV_RANK_TOL = 4.0 * 2.220446049250313e-16;

// |x| as an unsigned integer: for finite x its order is the order of |x|, so
// argmaxes run on the integer pipe (FP64 compares issue at the FP64 rate).
__device__ __forceinline__ unsigned long long absbits(double x)
{
    return (unsigned long long)__double_as_longlong(x) & 0x7FFFFFFFFFFFFFFFull;
}

__device__ __forceinline__ bool better(unsigned long long k, long long i, unsigned long long bk, long long bi)
{
    return k > bk || (k == bk && i < bi);
}

// Block-wide argmax of (key, i): largest key, smallest i among equal keys.
__device__ __forceinline__ void block_argmax_u(unsigned long long &k, long long &i, unsigned long long *sk, long long *si)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long ok = __shfl_xor_sync(0xFFFFFFFFu, k, o);
        const long long oi = __shfl_xor_sync(0xFFFFFFFFu, i, o);
        if (better(ok, oi, k, i)) {
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
        if (better(sk[w], si[w], k, i)) {
            k = sk[w];
            i = si[w];
        }
}

// One CTA's candidate of a step: its best key, the entry's index and the
// entry's row (all r columns of W).
struct MvSlot {
    unsigned long long key;
    long long e;
    double row[MV_RMAX];
};

// Per-CTA state of a cluster-wide argmax step.
struct MvStep {
    MvSlot slot[2];
    double row[MV_RMAX];            // the winner's row, copied from its owner's slot
    unsigned long long sk[MV_NW];
    long long si[MV_NW];
    unsigned long long win_key;
    long long win_e;
    int win_rank;
};

// The cluster-wide step: publish this CTA's candidate (k, e) -- stash(slot,
// k, e) copies the candidate's row into the slot -- then agree on the winner
// (st.win_*).  Every CTA of the cluster makes the same sequence of calls (the
// barrier inside is cluster-wide); par alternates between consecutive calls.
template <class Stash>
__device__ __forceinline__ const MvSlot *cluster_argmax(cg::cluster_group &cl, MvStep &st, int par, int ncl,
                                                        unsigned long long k, long long e, Stash stash)
{
    block_argmax_u(k, e, st.sk, st.si);
    MvSlot &s = st.slot[par];
    if (threadIdx.x == 0) {
        s.key = k;
        s.e = e;
    }
    stash(s, k, e);
    cl.sync();
    if (threadIdx.x < 32) {
        const int lane = threadIdx.x;
        unsigned long long bk = 0ull;
        long long be = LLONG_MAX;
        int br = 0;
        if (lane < ncl) {
            const MvSlot *rs = cl.map_shared_rank(&s, lane);
            bk = rs->key;
            be = rs->e;
            br = lane;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const unsigned long long ok = __shfl_xor_sync(0xFFFFFFFFu, bk, o);
            const long long oe = __shfl_xor_sync(0xFFFFFFFFu, be, o);
            const int orr = __shfl_xor_sync(0xFFFFFFFFu, br, o);
            if (better(ok, oe, bk, be)) {
                bk = ok;
                be = oe;
                br = orr;
            }
        }
        if (lane == 0) {
            st.win_key = bk;
            st.win_e = be;
            st.win_rank = br;
        }
    }
    __syncthreads();
    return cl.map_shared_rank(&s, st.win_rank);  // the winner's slot
}

__device__ __forceinline__ void row_slice(int n, int rank, int ncl, int &lo, int &hi)
{
    lo = (int)((long long)rank * n / ncl);
    hi = (int)((long long)(rank + 1) * n / ncl);
}

size_t maxvol_smem(int r) { return sizeof(double) * (size_t)r * 2 * r; }

// Phase 1: pivot rows and multipliers (the whole cluster), then L[I]^{-1}
// (rank 0 alone, in dynamic shared memory).
__global__ void __launch_bounds__(MV_NT) k_maxvol_pivot(const MaxvolDesc *descs)
{
    cg::cluster_group cl = cg::this_cluster();
    const MaxvolDesc &d = descs[blockIdx.y];
    const int n = d.n, r = d.r, ncl = (int)cl.num_blocks(), rank = (int)cl.block_rank();
    int lo, hi;
    row_slice(n, rank, ncl, lo, hi);
    __shared__ MvStep st;
    __shared__ int I[MV_RMAX];
    __shared__ unsigned chosen[MV_NMAX / 8 / 32];  // rows of this slice already picked (slices have <= n/8 + 1 rows)
    __shared__ int s_fail;
    __shared__ unsigned long long cbits[MV_RMAX];  // this CTA's column maxima of |A| (bit patterns)
    __shared__ double ctol[MV_RMAX];
    double *W = d.W;
    if (threadIdx.x == 0) s_fail = 0;
    for (int e = threadIdx.x; e < (hi - lo + 31) / 32; e += MV_NT) chosen[e] = 0u;
    for (int i = lo + threadIdx.x; i < hi; i += MV_NT)  // column-major copy; a thread reads its row in order
        for (int c = 0; c < r; ++c) W[(long long)c * n + i] = d.A[(long long)i * r + c];
    // the scale of every column, max_i |A[i][c]|, over the whole cluster: a
    // pivot at or below MV_RANK_TOL of its column's scale means rank < r
    for (int c = threadIdx.x; c < r; c += MV_NT) cbits[c] = 0ull;
    __syncthreads();
    for (int c = 0; c < r; ++c) {
        unsigned long long m = 0ull;
        for (int i = lo + threadIdx.x; i < hi; i += MV_NT) m = max(m, absbits(W[(long long)c * n + i]));
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xFFFFFFFFu, m, o));
        if ((threadIdx.x & 31) == 0 && m) atomicMax(&cbits[c], m);
    }
    cl.sync();
    for (int c = threadIdx.x; c < r; c += MV_NT) {
        unsigned long long m = 0ull;
        for (int q = 0; q < ncl; ++q) m = max(m, *cl.map_shared_rank(&cbits[c], q));
        ctol[c] = MV_RANK_TOL * r * __longlong_as_double((long long)m);
    }
    __syncthreads();

    // 1. partial pivoting; only the columns after j are updated (earlier ones
    // are never read again)
    for (int j = 0; j < r; ++j) {
        unsigned long long kmax = 0ull;
        long long bi = LLONG_MAX;
        for (int i = lo + threadIdx.x; i < hi; i += MV_NT) {
            if ((chosen[(i - lo) >> 5] >> ((i - lo) & 31)) & 1u) continue;
            const unsigned long long k = absbits(W[(long long)j * n + i]) + 1ull;  // 0 marks "no row"
            if (k > kmax) {  // i grows per thread, so equal keys keep the first
                kmax = k;
                bi = i;
            }
        }
        // the slot's row: the candidate's W[j..r) (entries before j are stale)
        const MvSlot *ws = cluster_argmax(cl, st, j & 1, ncl, kmax, bi, [&](MvSlot &s, unsigned long long k, long long e) {
            if (k != 0ull)
                for (int c = j + threadIdx.x; c < r; c += MV_NT) s.row[c] = W[(long long)c * n + e];
        });
        for (int c = j + threadIdx.x; c < r; c += MV_NT) st.row[c] = ws->row[c];
        const int p = (int)st.win_e;
        if (threadIdx.x == 0) {
            I[j] = p;
            if (p >= lo && p < hi) chosen[(p - lo) >> 5] |= 1u << ((p - lo) & 31);
        }
        __syncthreads();
        const double wp = st.row[j];
        if (!(fabs(wp) > ctol[j])) {
            if (threadIdx.x == 0) s_fail = 1;  // every CTA sees the same pivot and scale
        } else {
            const double inv = 1.0 / wp;
            for (int i = lo + threadIdx.x; i < hi; i += MV_NT) {
                if ((chosen[(i - lo) >> 5] >> ((i - lo) & 31)) & 1u) continue;
                double *wj = W + (long long)j * n + i;
                const double f = *wj * inv;
                *wj = f;  // L[i][j]
                for (int c = j + 1; c < r; ++c) {
                    double *w = W + (long long)c * n + i;
                    *w = fma(-f, st.row[c], *w);
                }
            }
        }
        // the next step's argmax reads only this thread's own rows; its block
        // argmax starts with a barrier before st is written again
    }
    cl.sync();  // no CTA leaves while another may still read its slots
    if (rank != 0) return;

    // L[I]^{-1}: L[I] is unit lower triangular, row k holding the multipliers
    // of row I[k] from the steps before k (other slices' rows are read from L2:
    // they were written before the barrier above)
    extern __shared__ double G[];
    double *Lt = G;                       // [r][r]
    double *Li = G + (size_t)r * r;       // [r][r]
    for (int e = threadIdx.x; e < r * r; e += MV_NT) {
        const int k = e / r, m = e - k * r;
        Lt[e] = m < k ? __ldcg(W + (long long)m * n + I[k]) : (m == k ? 1.0 : 0.0);
    }
    __syncthreads();
    // column c of the inverse by forward substitution, one thread per column
    for (int c = threadIdx.x; c < r; c += MV_NT) {
        for (int k = 0; k < c; ++k) Li[k * r + c] = 0.0;
        Li[c * r + c] = 1.0;
        for (int k = c + 1; k < r; ++k) {
            double acc = 0.0;
            for (int m = c; m < k; ++m) acc = fma(Lt[k * r + m], Li[m * r + c], acc);
            Li[k * r + c] = -acc;
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) d.status[0] = s_fail;
    if (s_fail) return;
    for (int e = threadIdx.x; e < r * r; e += MV_NT) d.Linv[e] = Li[e];
    for (int j = threadIdx.x; j < r; j += MV_NT) d.idx[j] = I[j];
}

// B = L L[I]^{-1} (L: the multipliers in W, column-major), spread over many
// CTAs per matrix; the pivot rows get the unit vectors.
__global__ void __launch_bounds__(256) k_maxvol_b(const MaxvolDesc *descs)
{
    const MaxvolDesc &d = descs[blockIdx.y];
    if (d.status[0]) return;
    const int n = d.n, r = d.r;
    __shared__ double Li[MV_RMAX * MV_RMAX];
    __shared__ unsigned piv[MV_NMAX / 32];  // rows in I
    __shared__ int I[MV_RMAX];
    for (int e = threadIdx.x; e < r * r; e += blockDim.x) Li[e] = d.Linv[e];
    for (int w = threadIdx.x; w < (n + 31) / 32; w += blockDim.x) piv[w] = 0u;
    for (int k = threadIdx.x; k < r; k += blockDim.x) I[k] = d.idx[k];
    __syncthreads();
    for (int k = threadIdx.x; k < r; k += blockDim.x) atomicOr(&piv[I[k] >> 5], 1u << (I[k] & 31));
    __syncthreads();
    const double *W = d.W;
    const long long nr = (long long)n * r;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < nr; e += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(e / r), c = (int)(e - (long long)i * r);
        double acc = 0.0;
        if ((piv[i >> 5] >> (i & 31)) & 1u) {
            acc = I[c] == i ? 1.0 : 0.0;
        } else {
            for (int k = c; k < r; ++k) acc = fma(W[(long long)k * n + i], Li[k * r + c], acc);
        }
        d.B[e] = acc;
    }
}

// Phase 3, the swaps (the whole cluster), on a column-major copy of B in W.
__global__ void __launch_bounds__(MV_NT) k_maxvol_swap(const MaxvolDesc *descs, double delta, int max_iters)
{
    cg::cluster_group cl = cg::this_cluster();
    const MaxvolDesc &d = descs[blockIdx.y];
    if (d.status[0]) return;  // the same value for every CTA of the cluster
    const int n = d.n, r = d.r, ncl = (int)cl.num_blocks(), rank = (int)cl.block_rank();
    int lo, hi;
    row_slice(n, rank, ncl, lo, hi);
    __shared__ MvStep st;
    __shared__ int I[MV_RMAX];
    double *W = d.W;
    for (int j = threadIdx.x; j < r; j += MV_NT) I[j] = d.idx[j];
    // column-major copy of the slice, with the first argmax (e = i r + c grows
    // per thread, so equal keys keep the first)
    unsigned long long kmax = 0ull;
    long long bi = LLONG_MAX;
    for (int i = lo + threadIdx.x; i < hi; i += MV_NT)
        for (int c = 0; c < r; ++c) {
            const double b = d.B[(long long)i * r + c];
            W[(long long)c * n + i] = b;
            const unsigned long long k = absbits(b);
            if (k > kmax || bi == LLONG_MAX) {
                kmax = k;
                bi = (long long)i * r + c;
            }
        }
    __syncthreads();
    int it = 0;
    for (; it < max_iters; ++it) {
        const MvSlot *ws = cluster_argmax(cl, st, it & 1, ncl, kmax, bi, [&](MvSlot &s, unsigned long long, long long e) {
            if (e != LLONG_MAX) {
                const long long i = e / r;
                for (int c = threadIdx.x; c < r; c += MV_NT) s.row[c] = W[(long long)c * n + i];
            }
        });
        if (!(__longlong_as_double((long long)st.win_key) > 1.0 + delta)) break;  // the same decision everywhere
        const long long we = st.win_e;
        const int i0 = (int)(we / r), j0 = (int)(we - (long long)i0 * r);
        const double piv = ws->row[j0];
        for (int c = threadIdx.x; c < r; c += MV_NT) st.row[c] = (ws->row[c] - (c == j0 ? 1.0 : 0.0)) / piv;
        if (threadIdx.x == 0) I[j0] = i0;
        __syncthreads();
        // B -= B[:, j0] (row_i0 - e_j0) / piv over the slice, with the next argmax
        kmax = 0ull;
        bi = LLONG_MAX;
        for (int i = lo + threadIdx.x; i < hi; i += MV_NT) {
            const double f = W[(long long)j0 * n + i];
            for (int c = 0; c < r; ++c) {
                double *w = W + (long long)c * n + i;
                const double b = fma(-f, st.row[c], *w);
                *w = b;
                const unsigned long long k = absbits(b);
                if (k > kmax || bi == LLONG_MAX) {
                    kmax = k;
                    bi = (long long)i * r + c;
                }
            }
        }
    }
    cl.sync();  // no CTA leaves while another may still read its slots
    for (int i = lo + threadIdx.x; i < hi; i += MV_NT)
        for (int c = 0; c < r; ++c) d.B[(long long)i * r + c] = W[(long long)c * n + i];
    if (rank == 0) {
        for (int j = threadIdx.x; j < r; j += MV_NT) d.idx[j] = I[j];
        if (threadIdx.x == 0) {
            d.status[0] = 0;
            d.swaps[0] = it;
        }
    }
}

// Largest matrices first, so that their clusters start in the first wave.
void maxvol_order(MaxvolDesc *d, int n)
{
    std::stable_sort(d, d + n, [](const MaxvolDesc &a, const MaxvolDesc &b) {
        return (double)a.n * a.r * a.r > (double)b.n * b.r * b.r;
    });
}

template <class K, class... Args>
static cudaError_t launch_cluster(K kern, int ncl, int n, size_t smem, cudaStream_t s, Args... args)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(ncl, n);
    cfg.blockDim = dim3(MV_NT);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = ncl;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, args...);
}

// Cluster size: 16 CTAs where the device schedules clusters that large, else 8.
static int maxvol_cluster_size()
{
    static int ncl = 0;
    if (ncl) return ncl;
    ncl = 8;
    if (cudaFuncSetAttribute(k_maxvol_pivot, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) == cudaSuccess &&
        cudaFuncSetAttribute(k_maxvol_swap, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) == cudaSuccess) {
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(16, 1);
        cfg.blockDim = dim3(MV_NT);
        cfg.dynamicSmemBytes = maxvol_smem(MV_RMAX);
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeClusterDimension;
        at[0].val.clusterDim.x = 16;
        at[0].val.clusterDim.y = 1;
        at[0].val.clusterDim.z = 1;
        cfg.attrs = at;
        cfg.numAttrs = 1;
        int c1 = 0, c2 = 0;
        if (cudaOccupancyMaxActiveClusters(&c1, k_maxvol_pivot, &cfg) == cudaSuccess &&
            cudaOccupancyMaxActiveClusters(&c2, k_maxvol_swap, &cfg) == cudaSuccess && c1 > 0 && c2 > 0)
            ncl = 16;
    }
    cudaGetLastError();  // a refused query leaves no sticky state; clear the last error
    return ncl;
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
    const int ncl = maxvol_cluster_size();
    cudaError_t e = launch_cluster(k_maxvol_pivot, ncl, n, maxvol_smem(max_r), s, d);
    if (e != cudaSuccess) return e;
    k_maxvol_b<<<dim3(64, n), 256, 0, s>>>(d);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return launch_cluster(k_maxvol_swap, ncl, n, 0, s, d, delta, max_iters);
}

}  // namespace wg
