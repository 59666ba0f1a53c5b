// k_maxvol.cu -- batched maxvol (the maximum-volume row selection that picks
// the cross indices of TT-cross, Sec. 3 "TT-cross Interpolation"), FP64, three
// launches per batch:
//   1. the r pivot rows of Gaussian elimination with partial pivoting on a
//      working copy W (largest remaining |W[i][j]| of column j, ties to the
//      smaller row), then A[I]^{-1} by Gauss-Jordan with partial pivoting;
//   2. B = A A[I]^{-1}, spread over many CTAs per matrix;
//   3. while max |B[i][j]| > 1 + delta (ties to the first entry in row-major
//      order): row i replaces I[j] and B -= B[:, j] (B[i, :] - e_j) / B[i][j].
// Phases 1 and 3 are sequences of (argmax, rank-one update) steps.  Each matrix
// gets a thread-block cluster whose CTAs own contiguous slices of its rows, so
// the FP64 work of a large matrix spreads over up to 16 SMs.  Per step every
// CTA finds the best entry of its slice and stashes that entry's row in a
// shared-memory slot; after one cluster barrier every CTA reduces the slots
// (read through distributed shared memory) to the same winner and copies the
// winner's row from its owner.  Slots alternate between two buffers, so the
// writes of step t + 1 never meet the reads of step t, and the stash lets the
// owner update the winning row in place while others still read it.  The
// working copy is column-major (W[c][i]), so a warp's row-parallel accesses
// coalesce; it stays in L2.
#include <algorithm>
#include <climits>

#include <cooperative_groups.h>

#include "weno_dev.cuh"
#include "weno_internal.h"
#include "tt_internal.h"

namespace wg {

namespace cg = cooperative_groups;

constexpr int MV_NT = 256, MV_NW = MV_NT / 32;

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

size_t maxvol_smem(int r) { return sizeof(double) * (size_t)r * (2 * r + 1); }

// Phase 1: pivot rows (the whole cluster), then the Gauss-Jordan inverse of
// A[I] (rank 0 alone, in dynamic shared memory).
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
    double *W = d.W;
    for (int e = threadIdx.x; e < (hi - lo + 31) / 32; e += MV_NT) chosen[e] = 0u;
    for (int i = lo + threadIdx.x; i < hi; i += MV_NT)  // column-major copy; a thread reads its row in order
        for (int c = 0; c < r; ++c) W[(long long)c * n + i] = d.A[(long long)i * r + c];
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
        if (wp != 0.0 && j + 1 < r) {
            const double inv = 1.0 / wp;
            for (int i = lo + threadIdx.x; i < hi; i += MV_NT) {
                if ((chosen[(i - lo) >> 5] >> ((i - lo) & 31)) & 1u) continue;
                const double f = W[(long long)j * n + i] * inv;
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

    // A[I]^{-1}: Gauss-Jordan on [A[I] | identity], pivot search on the
    // integer pipe, row swap, scaling and elimination spread over the block
    extern __shared__ double G[];  // [r][2r]
    const int r2 = 2 * r;
    for (int e = threadIdx.x; e < r * r2; e += MV_NT) {
        const int i = e / r2, c = e - i * r2;
        G[e] = c < r ? d.A[(long long)I[i] * r + c] : (c - r == i ? 1.0 : 0.0);
    }
    if (threadIdx.x == 0) s_fail = 0;
    __shared__ int s_piv;
    __syncthreads();
    for (int c = 0; c < r; ++c) {
        if (threadIdx.x == 0) {
            int p = c;
            unsigned long long best = absbits(G[c * r2 + c]);
            for (int i = c + 1; i < r; ++i) {
                const unsigned long long k = absbits(G[i * r2 + c]);
                if (k > best) {
                    best = k;
                    p = i;
                }
            }
            if (best == 0ull) s_fail = 1;
            s_piv = p;
        }
        __syncthreads();
        const int p = s_piv;
        if (p != c)
            for (int t = c + threadIdx.x; t < r2; t += MV_NT) {
                const double x = G[c * r2 + t];
                G[c * r2 + t] = G[p * r2 + t];
                G[p * r2 + t] = x;
            }
        __syncthreads();
        const double gcc = G[c * r2 + c];
        const double inv = gcc == 0.0 ? 0.0 : 1.0 / gcc;
        __syncthreads();
        for (int t = c + threadIdx.x; t < r2; t += MV_NT) G[c * r2 + t] *= inv;
        __syncthreads();
        for (int i = threadIdx.x; i < r; i += MV_NT) st.row[i] = G[i * r2 + c];  // multipliers, read before any write
        __syncthreads();
        const int w = r2 - c;  // columns c..2r-1 (the ones before c are already unit vectors)
        for (int e = threadIdx.x; e < r * w; e += MV_NT) {
            const int i = e / w, t = c + (e - i * w);
            if (i == c) continue;
            G[i * r2 + t] = fma(-st.row[i], G[c * r2 + t], G[i * r2 + t]);
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) d.status[0] = s_fail;
    if (s_fail) return;
    for (int e = threadIdx.x; e < r * r; e += MV_NT) {
        const int k = e / r, c = e - k * r;
        d.Minv[e] = G[k * r2 + r + c];
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
