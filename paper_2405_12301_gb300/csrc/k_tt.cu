// k_tt.cu -- batched TT-rounding of 3D tensor trains in FP64 (Sec. 3
// "TT-rounding", the two-pass algorithm of Oseledets 2011, Algorithm 2), the
// rounding behind every stage of Eq. (tt-ssprk3).
//
// Building blocks, each a batched kernel over independent problems:
//   * k_qr_factor: Householder QR of a tall-skinny m x k matrix (k <= 96),
//     two-level TSQR.  A chunk of rows is factored by one CTA as a flat tree:
//     a plain Householder QR of its first b rows, then for every further
//     sub-block B of b rows the structured QR of [R; B] whose reflectors are
//     [e_j; y_j].  The chunk R factors are stacked and factored the same way
//     by a second launch.  Reflectors overwrite the matrix; taus are kept.
//   * k_qr_apply: Q [X; 0] for a k x p block X, replaying the reflectors of a
//     chunk in reverse (eight lanes per column of X, four columns per warp,
//     no block barrier inside a sub-block); writes the rows through a general row map so that results
//     land directly in TT-core layout.
//   * k_svd_jacobi: one-sided Jacobi SVD (round-robin pair ordering) of the
//     transpose of a k x q triangular factor T: T^T V = U S gives T = V S U^T;
//     picks the truncation rank from the singular values and writes V's kept
//     columns and (U S)'s kept columns.
//   * k_tt_build / k_tt_contract / k_tt_gemm_tr: the TT sum's first and last
//     unfoldings, the block-diagonal middle core times a triangular factor, and
//     a small dense product.
// All arithmetic is FP64.
#include <cfloat>

#include "weno_dev.cuh"
#include "weno_internal.h"
#include "tt_internal.h"

namespace wg {

constexpr int TT_NT = 256, TT_NW = TT_NT / 32;

__device__ __forceinline__ double warp_sum_d(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, o);
    return v;
}

// The update loops below give each column of a reflector update to a group of
// LPC lanes (CPW = 32 / LPC columns per warp, a lane every LPC-th row).  On
// this GPU every FP64 warp instruction holds the FP64 pipe however many lanes
// it serves, so the group's shuffle adds (log2 LPC per lane), the redundant
// w = tau (dot + x_j) on every lane of the group and the one-lane diagonal
// update are pure overhead on top of the 2 FMAs per row: 4 lanes keep it near
// 15% (8 lanes cost about 35%).  Sub-blocks are stored with a pitch of b + 4
// (b a multiple of 32), so a half-warp's 4 columns x 4 rows hit 16 distinct
// banks.
constexpr int LPC = 4, CPW = 32 / LPC, LDPAD = 4;
constexpr int SV_LPP = 4, SV_PPW = 32 / SV_LPP;  // Jacobi lanes per pair, pairs per warp

__device__ __forceinline__ double pair_sum_d(double v)
{
#pragma unroll
    for (int o = SV_LPP / 2; o > 0; o >>= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, o);
    return v;
}

__device__ __forceinline__ double group_sum(double v)
{
#pragma unroll
    for (int o = LPC / 2; o > 0; o >>= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, o);
    return v;
}

// Householder vector of x = (x0, y) with ||y||^2 = sig: H = I - tau v v^T,
// v = (1, y / (x0 - beta)), H x = (beta, 0).  sig == 0 gives tau = 0.
__device__ __forceinline__ void householder(double x0, double sig, double &beta, double &tau, double &scale)
{
    beta = x0;
    tau = 0.0;
    scale = 0.0;
    if (sig > 0.0) {
        beta = -copysign(sqrt(fma(x0, x0, sig)), x0);
        tau = (beta - x0) / beta;
        scale = 1.0 / (x0 - beta);
    }
}

size_t qr_factor_smem(int k, int b) { return sizeof(double) * ((size_t)k * (b + LDPAD) + (size_t)k * (k + 1) + k); }
size_t qr_apply_smem(int k, int b, int p)
{
    return sizeof(double) * ((size_t)k * (b + LDPAD) + (size_t)p * (b + LDPAD) + (size_t)p * (k + 1) + k);
}
size_t svd_smem(int pk, int q) { return sizeof(double) * ((size_t)pk * (q + 1) + (size_t)pk * (pk + 1) + 2 * pk); }

__global__ void __launch_bounds__(TT_NT) k_qr_factor(const QRDesc *descs)
{
    const QRDesc &d = descs[blockIdx.y];
    const int chunk = blockIdx.x;
    if (chunk >= d.chunks || d.m <= 0) return;
    extern __shared__ double sm[];
    const int k = d.k, b = d.b, ldb = b + LDPAD, ldr = k + 1;
    double *B = sm;                       // sub-block, column-major [k][ldb]
    double *R = B + (size_t)k * ldb;      // running R, column-major [k][ldr]
    double *ts = R + (size_t)k * ldr;     // taus of the current sub-block
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, grp = lane / LPC, sub = lane % LPC;
    const long long r0 = (long long)chunk * d.chunk_rows;
    const long long r1 = min(d.m, r0 + d.chunk_rows);

    for (int s = 0;; ++s) {
        const long long s0 = r0 + (long long)s * b;
        if (s0 >= r1) break;
        const int bs = (int)min((long long)b, r1 - s0);
        for (int e = threadIdx.x; e < bs * k; e += TT_NT) {
            const int i = e / k, c = e - i * k;
            B[c * ldb + i] = d.A[(s0 + i) * d.lda + c];
        }
        for (int j = threadIdx.x; j < k; j += TT_NT) ts[j] = 0.0;
        __syncthreads();
        if (s == 0) {
            // plain Householder QR of the first bs x k block
            const int kk = min(bs, k);
            for (int j = 0; j < kk; ++j) {
                if (warp == 0) {
                    double *x = B + j * ldb;
                    double sig = 0.0;
                    for (int i = j + 1 + lane; i < bs; i += 32) sig = fma(x[i], x[i], sig);
                    sig = warp_sum_d(sig);
                    double beta, tau, scale;
                    householder(x[j], sig, beta, tau, scale);
                    for (int i = j + 1 + lane; i < bs; i += 32) x[i] *= scale;
                    __syncwarp();  // every lane has read x[j]
                    if (lane == 0) {
                        x[j] = beta;
                        ts[j] = tau;
                    }
                }
                __syncthreads();
                const double tau = ts[j];
                if (tau != 0.0) {
                    const double *v = B + j * ldb;
                    for (int c0 = j + 1 + warp * CPW; c0 < k; c0 += TT_NW * CPW) {
                        const int c = c0 + grp;
                        const bool ok = c < k;
                        double *col = B + (ok ? c : 0) * ldb;
                        double w = 0.0;
                        if (ok)
                            for (int i = j + 1 + sub; i < bs; i += LPC) w = fma(v[i], col[i], w);
                        w = (group_sum(w) + (ok ? col[j] : 0.0)) * tau;
                        if (ok)
                            for (int i = j + 1 + sub; i < bs; i += LPC) col[i] = fma(-v[i], w, col[i]);
                        __syncwarp();
                        if (ok && sub == 0) col[j] -= w;
                    }
                }
                __syncthreads();
            }
            for (int e = threadIdx.x; e < k * k; e += TT_NT) {
                const int c = e / k, j = e - c * k;
                R[c * ldr + j] = (j <= c && j < kk) ? B[c * ldb + j] : 0.0;
            }
        } else {
            // structured QR of [R; B]: reflector j is (e_j; y_j), y_j stored in B's column j
            for (int j = 0; j < k; ++j) {
                if (warp == 0) {
                    double *y = B + j * ldb;
                    double sig = 0.0;
                    for (int i = lane; i < bs; i += 32) sig = fma(y[i], y[i], sig);
                    sig = warp_sum_d(sig);
                    double beta, tau, scale;
                    householder(R[j * ldr + j], sig, beta, tau, scale);
                    for (int i = lane; i < bs; i += 32) y[i] *= scale;
                    __syncwarp();  // every lane has read R[j][j]
                    if (lane == 0) {
                        R[j * ldr + j] = beta;
                        ts[j] = tau;
                    }
                }
                __syncthreads();
                const double tau = ts[j];
                if (tau != 0.0) {
                    const double *y = B + j * ldb;
                    for (int c0 = j + 1 + warp * CPW; c0 < k; c0 += TT_NW * CPW) {
                        const int c = c0 + grp;
                        const bool ok = c < k;
                        double *col = B + (ok ? c : 0) * ldb;
                        double w = 0.0;
                        if (ok)
                            for (int i = sub; i < bs; i += LPC) w = fma(y[i], col[i], w);
                        w = (group_sum(w) + (ok ? R[c * ldr + j] : 0.0)) * tau;
                        if (ok)
                            for (int i = sub; i < bs; i += LPC) col[i] = fma(-y[i], w, col[i]);
                        __syncwarp();
                        if (ok && sub == 0) R[c * ldr + j] -= w;
                    }
                }
                __syncthreads();
            }
        }
        for (int e = threadIdx.x; e < bs * k; e += TT_NT) {
            const int i = e / k, c = e - i * k;
            d.A[(s0 + i) * d.lda + c] = B[c * ldb + i];
        }
        for (int j = threadIdx.x; j < k; j += TT_NT) d.tau[((long long)chunk * d.sub_per_chunk + s) * k + j] = ts[j];
        __syncthreads();
    }
    for (int e = threadIdx.x; e < k * k; e += TT_NT) {
        const int j = e / k, c = e - j * k;
        d.Rout[(long long)chunk * k * k + e] = R[c * ldr + j];
    }
}

__global__ void __launch_bounds__(TT_NT) k_qr_apply(const QApplyDesc *descs)
{
    const QApplyDesc &d = descs[blockIdx.y];
    const int chunk = blockIdx.x;
    if (chunk >= d.chunks || d.m <= 0 || d.p <= 0) return;
    extern __shared__ double sm[];
    const int k = d.k, b = d.b, p = d.p, ldb = b + LDPAD, ldx = k + 1;
    double *Y = sm;                        // reflectors of a sub-block, column-major [k][ldb]
    double *Z = Y + (size_t)k * ldb;       // output block, column-major [p][ldb]
    double *X = Z + (size_t)p * ldb;       // running top rows, column-major [p][ldx]
    double *ts = X + (size_t)p * ldx;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, grp = lane / LPC, sub = lane % LPC;
    const long long r0 = (long long)chunk * d.chunk_rows;
    const long long r1 = min(d.m, r0 + d.chunk_rows);
    const int nsub = (int)((r1 - r0 + b - 1) / b);
    const int b1 = (int)min((long long)b, r1 - r0);
    const int kk = min(b1, k);  // rows of X (k unless the chunk is shorter than k)
    const double *Xin = d.X ? d.X + (long long)chunk * d.x_chunk_stride : nullptr;  // null: identity
    for (int e = threadIdx.x; e < kk * p; e += TT_NT) {
        const int j = e / p, q = e - j * p;
        X[q * ldx + j] = Xin ? Xin[(long long)j * d.ldx + q] : (j == q ? 1.0 : 0.0);
    }
    __syncthreads();
    auto store = [&](long long row0, int rows) {
        for (int e = threadIdx.x; e < rows * p; e += TT_NT) {
            const int i = e / p, q = e - i * p;
            const long long row = row0 + i;
            d.out[(row % d.P) * d.sP + (row / d.P) * d.sQ + (long long)q * d.sC] = Z[q * ldb + i];
        }
    };
    for (int s = nsub - 1; s >= 1; --s) {
        const long long s0 = r0 + (long long)s * b;
        const int bs = (int)min((long long)b, r1 - s0);
        for (int e = threadIdx.x; e < bs * k; e += TT_NT) {
            const int i = e / k, c = e - i * k;
            Y[c * ldb + i] = d.A[(s0 + i) * d.lda + c];
        }
        for (int e = threadIdx.x; e < bs * p; e += TT_NT) Z[(e / bs) * ldb + e % bs] = 0.0;
        for (int j = threadIdx.x; j < k; j += TT_NT) ts[j] = d.tau[((long long)chunk * d.sub_per_chunk + s) * k + j];
        __syncthreads();
        for (int q0 = warp * CPW; q0 < p; q0 += TT_NW * CPW) {
            const int q = q0 + grp;
            const bool ok = q < p;
            double *zq = Z + (ok ? q : 0) * ldb;
            double *xq = X + (ok ? q : 0) * ldx;
            for (int j = k - 1; j >= 0; --j) {
                const double tau = ts[j];
                if (tau == 0.0) continue;
                const double *y = Y + j * ldb;
                double w = 0.0;
                if (ok)
                    for (int i = sub; i < bs; i += LPC) w = fma(y[i], zq[i], w);
                w = (group_sum(w) + (ok ? xq[j] : 0.0)) * tau;
                if (ok)
                    for (int i = sub; i < bs; i += LPC) zq[i] = fma(-y[i], w, zq[i]);
                __syncwarp();
                if (ok && sub == 0) xq[j] -= w;
                __syncwarp();
            }
        }
        __syncthreads();
        store(s0, bs);
        __syncthreads();
    }
    // first sub-block: plain reflectors below the diagonal, acting on [X; 0]
    for (int e = threadIdx.x; e < b1 * k; e += TT_NT) {
        const int i = e / k, c = e - i * k;
        Y[c * ldb + i] = d.A[(r0 + i) * d.lda + c];
    }
    for (int e = threadIdx.x; e < b1 * p; e += TT_NT) {
        const int q = e / b1, i = e - q * b1;
        Z[q * ldb + i] = i < kk ? X[q * ldx + i] : 0.0;
    }
    for (int j = threadIdx.x; j < k; j += TT_NT) ts[j] = d.tau[(long long)chunk * d.sub_per_chunk * k + j];
    __syncthreads();
    for (int q0 = warp * CPW; q0 < p; q0 += TT_NW * CPW) {
        const int q = q0 + grp;
        const bool ok = q < p;
        double *zq = Z + (ok ? q : 0) * ldb;
        for (int j = kk - 1; j >= 0; --j) {
            const double tau = ts[j];
            if (tau == 0.0) continue;
            const double *v = Y + j * ldb;
            double w = 0.0;
            if (ok)
                for (int i = j + 1 + sub; i < b1; i += LPC) w = fma(v[i], zq[i], w);
            w = (group_sum(w) + (ok ? zq[j] : 0.0)) * tau;
            if (ok)
                for (int i = j + 1 + sub; i < b1; i += LPC) zq[i] = fma(-v[i], w, zq[i]);
            __syncwarp();
            if (ok && sub == 0) zq[j] -= w;
            __syncwarp();
        }
    }
    __syncthreads();
    store(r0, b1);
}

// One-sided Jacobi on the pk columns of M = T^T (column t = row t of T, length q).
__global__ void __launch_bounds__(TT_NT) k_svd_jacobi(const SvdDesc *descs)
{
    const SvdDesc &d = descs[blockIdx.x];
    const int pk = d.pk, q = d.q;
    if (pk <= 0) return;
    extern __shared__ double sm[];
    const int ldm = q + 1, ldv = pk + 1;
    double *M = sm;                          // [pk][ldm]
    double *V = M + (size_t)pk * ldm;        // [pk][ldv], column t = rotations applied to e_t
    double *sig = V + (size_t)pk * ldv;      // [pk]
    int *ord = reinterpret_cast<int *>(sig + pk);
    __shared__ int rotated;
    __shared__ double s_delta;
    __shared__ int s_rank;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int e = threadIdx.x; e < pk * q; e += TT_NT) {
        const int t = e / q, i = e - t * q;
        M[t * ldm + i] = d.T[(long long)t * d.ldt + i];
    }
    for (int e = threadIdx.x; e < pk * pk; e += TT_NT) {
        const int t = e / pk, i = e - t * pk;
        V[t * ldv + i] = (i == t) ? 1.0 : 0.0;
    }
    __syncthreads();
    const int n = pk + (pk & 1);  // round-robin over an even count; index pk (odd case) is a bye
    const int npairs = n / 2;
    const double tol = 8.0 * (double)max(pk, q) * DBL_EPSILON;  // cosine below which a pair counts as orthogonal
    // per round: the pairs' dot products (an SV_LPP-lane group per pair: its
    // sums cost log2 SV_LPP shuffle adds, a warp sum 5, and the columns are at
    // most 96 long), their rotations (a lane per pair: the square roots and
    // divisions run once per pair, not on every lane of a group), then the
    // rotations themselves (an SV_LPP-lane group per pair)
    __shared__ double s_a[TT_KMAX / 2], s_b[TT_KMAX / 2], s_c[TT_KMAX / 2], s_cs[TT_KMAX / 2], s_sn[TT_KMAX / 2];
    __shared__ int s_uv[TT_KMAX / 2][2];
    for (int sweep = 0; sweep < 60 && n > 1; ++sweep) {
        if (threadIdx.x == 0) rotated = 0;
        __syncthreads();
        for (int round = 0; round < n - 1; ++round) {
            auto idx = [&](int t) { return t == 0 ? 0 : 1 + (t - 1 + round) % (n - 1); };
            for (int s0 = warp * SV_PPW; s0 < npairs; s0 += TT_NW * SV_PPW) {  // the same trip count on every lane
                const int slot = s0 + lane / SV_LPP, sub = lane % SV_LPP;
                const bool ok = slot < npairs;
                const int u = ok ? idx(slot) : 0, v = ok ? idx(n - 1 - slot) : 0;
                double a = 0.0, bb = 0.0, c = 0.0;
                if (ok && u < pk && v < pk) {
                    const double *mu = M + u * ldm, *mv = M + v * ldm;
                    for (int i = sub; i < q; i += SV_LPP) {
                        a = fma(mu[i], mu[i], a);
                        bb = fma(mv[i], mv[i], bb);
                        c = fma(mu[i], mv[i], c);
                    }
                }
                a = pair_sum_d(a);
                bb = pair_sum_d(bb);
                c = pair_sum_d(c);
                if (ok && sub == 0) {
                    s_a[slot] = a;
                    s_b[slot] = bb;
                    s_c[slot] = c;
                    s_uv[slot][0] = u;
                    s_uv[slot][1] = v;
                }
            }
            __syncthreads();
            for (int slot = threadIdx.x; slot < npairs; slot += TT_NT) {
                const double a = s_a[slot], bb = s_b[slot], c = s_c[slot];
                double cs = 1.0, sn = 0.0;
                if (c != 0.0 && fabs(c) > tol * sqrt(a * bb)) {
                    const double zeta = (bb - a) / (2.0 * c);
                    const double t = copysign(1.0, zeta) / (fabs(zeta) + sqrt(fma(zeta, zeta, 1.0)));
                    cs = 1.0 / sqrt(fma(t, t, 1.0));
                    sn = cs * t;
                    rotated = 1;
                }
                s_cs[slot] = cs;
                s_sn[slot] = sn;
            }
            __syncthreads();
            for (int slot = threadIdx.x / SV_LPP; slot < npairs; slot += TT_NT / SV_LPP) {  // no shuffles: groups may leave early
                const double sn = s_sn[slot];
                if (sn == 0.0) continue;
                const double cs = s_cs[slot];
                const int u = s_uv[slot][0], v = s_uv[slot][1], sub = lane % SV_LPP;
                double *mu = M + u * ldm, *mv = M + v * ldm;
                for (int i = sub; i < q; i += SV_LPP) {
                    const double x = mu[i], y = mv[i];
                    mu[i] = cs * x - sn * y;
                    mv[i] = sn * x + cs * y;
                }
                double *vu = V + u * ldv, *vv = V + v * ldv;
                for (int i = sub; i < pk; i += SV_LPP) {
                    const double x = vu[i], y = vv[i];
                    vu[i] = cs * x - sn * y;
                    vv[i] = sn * x + cs * y;
                }
            }
            __syncthreads();
        }
        if (!rotated) break;
        __syncthreads();
    }
    // singular values, their descending order (ties by index), norm, rank
    for (int t = warp; t < pk; t += TT_NW) {
        double a = 0.0;
        for (int i = lane; i < q; i += 32) a = fma(M[t * ldm + i], M[t * ldm + i], a);
        a = warp_sum_d(a);
        if (lane == 0) sig[t] = sqrt(a);
    }
    __syncthreads();
    for (int t = threadIdx.x; t < pk; t += TT_NT) {
        int r = 0;
        for (int u = 0; u < pk; ++u) r += (sig[u] > sig[t]) || (sig[u] == sig[t] && u < t);
        ord[r] = t;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double delta;
        if (d.set_delta) {
            double s2 = 0.0;
            for (int t = pk - 1; t >= 0; --t) s2 += sig[ord[t]] * sig[ord[t]];
            delta = d.eps / sqrt(2.0) * sqrt(s2);
            d.delta[0] = delta;
            d.delta[1] = sqrt(s2);
        } else {
            delta = d.delta[0];
        }
        // smallest r >= 1 whose discarded singular values have a 2-norm <= delta
        int r = pk;
        double tail = 0.0;
        while (r > 1) {
            const double s = sig[ord[r - 1]];
            const double nt = fma(s, s, tail);
            if (sqrt(nt) > delta) break;
            tail = nt;
            --r;
        }
        if (r > d.rmax) r = d.rmax;
        s_rank = r;
        s_delta = delta;
        d.rank[0] = r;
    }
    __syncthreads();
    const int r = s_rank;
    for (int t = threadIdx.x; t < pk; t += TT_NT) d.sv[t] = sig[ord[t]];
    for (int e = threadIdx.x; e < pk * r; e += TT_NT) {
        const int i = e / r, c = e - i * r;
        d.Vsel[(long long)i * d.ld_out + c] = V[ord[c] * ldv + i];
    }
    for (int e = threadIdx.x; e < q * r; e += TT_NT) {
        const int i = e / r, c = e - i * r;
        d.Wt[(long long)i * d.ld_out + c] = M[ord[c] * ldm + i];
    }
}

// First-core unfolding C1 [n1][R1] (coefficient folded in) and transposed
// last-core unfolding MA [n3][R2] of the TT sum.
__global__ void k_tt_build(const TTSumDesc *descs)
{
    const TTSumDesc &d = descs[blockIdx.y];
    const long long e1 = (long long)d.n[0] * d.R1, e3 = (long long)d.n[2] * d.R2;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < e1 + e3;
         e += (long long)gridDim.x * blockDim.x) {
        if (e < e1) {
            const int i = (int)(e / d.R1), a = (int)(e - (long long)i * d.R1);
            int t = 0;
            while (t + 1 < d.nt && a >= d.a0[t + 1]) ++t;
            d.C1[e] = d.coef[t] * d.core[t][0][(long long)i * d.r1[t] + (a - d.a0[t])];
        } else {
            const long long f = e - e1;
            const int i = (int)(f / d.R2), bb = (int)(f - (long long)i * d.R2);
            int t = 0;
            while (t + 1 < d.nt && bb >= d.b0[t + 1]) ++t;
            d.MA[f] = d.core[t][2][(long long)i * d.r2[t] + (bb - d.b0[t])];
        }
    }
}

// MB[(j k3 + c) R1 + a] = sum_b G2_t[j][a - a0_t][b] TA[c][b0_t + b]  (t = term of a):
// the block-diagonal middle core of the sum times TA^T on its right rank,
// written as the (n2 k3) x R1 unfolding of the next QR.
__global__ void k_tt_contract(const TTSumDesc *descs)
{
    const TTSumDesc &d = descs[blockIdx.y];
    const long long tot = (long long)d.n[1] * d.k3 * d.R1;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < tot;
         e += (long long)gridDim.x * blockDim.x) {
        const int a = (int)(e % d.R1);
        const long long jc = e / d.R1;
        const int c = (int)(jc % d.k3), j = (int)(jc / d.k3);
        int t = 0;
        while (t + 1 < d.nt && a >= d.a0[t + 1]) ++t;
        const double *g = d.core[t][1] + ((long long)j * d.r1[t] + (a - d.a0[t])) * d.r2[t];
        const double *ta = d.TA + (long long)c * d.R2 + d.b0[t];
        double s = 0.0;
        for (int bb = 0; bb < d.r2[t]; ++bb) s = fma(g[bb], ta[bb], s);
        d.MB[e] = s;
    }
}

// out[i][c] = sum_a L[i][a] Rt[c][a]  (out = L Rt^T; L [rows][ka], Rt [cols][ka], row-major)
__global__ void k_tt_gemm_tr(const GemmDesc *descs)
{
    const GemmDesc &d = descs[blockIdx.y];
    const long long tot = (long long)d.rows * d.cols;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < tot;
         e += (long long)gridDim.x * blockDim.x) {
        const int c = (int)(e % d.cols);
        const long long i = e / d.cols;
        const double *l = d.L + i * d.ka;
        const double *r = d.Rt + (long long)c * d.ka;
        double s = 0.0;
        for (int a = 0; a < d.ka; ++a) s = fma(l[a], r[a], s);
        d.out[e] = s;
    }
}

static bool tt_attrs_set = false;

static cudaError_t tt_set_attributes()
{
    if (tt_attrs_set) return cudaSuccess;
    const int mx = (int)qr_apply_smem(TT_KMAX, TT_KMAX, TT_KMAX);
    cudaError_t e;
    if ((e = cudaFuncSetAttribute(k_qr_factor, cudaFuncAttributeMaxDynamicSharedMemorySize, mx)) != cudaSuccess) return e;
    if ((e = cudaFuncSetAttribute(k_qr_apply, cudaFuncAttributeMaxDynamicSharedMemorySize, mx)) != cudaSuccess) return e;
    if ((e = cudaFuncSetAttribute(k_svd_jacobi, cudaFuncAttributeMaxDynamicSharedMemorySize, mx)) != cudaSuccess) return e;
    tt_attrs_set = true;
    return cudaSuccess;
}

cudaError_t launch_qr_factor(const QRDesc *d, int n, int max_chunks, size_t smem, cudaStream_t s)
{
    cudaError_t e = tt_set_attributes();
    if (e != cudaSuccess) return e;
    k_qr_factor<<<dim3(max_chunks, n), TT_NT, smem, s>>>(d);
    return cudaGetLastError();
}

cudaError_t launch_qr_apply(const QApplyDesc *d, int n, int max_chunks, size_t smem, cudaStream_t s)
{
    cudaError_t e = tt_set_attributes();
    if (e != cudaSuccess) return e;
    k_qr_apply<<<dim3(max_chunks, n), TT_NT, smem, s>>>(d);
    return cudaGetLastError();
}

cudaError_t launch_svd_jacobi(const SvdDesc *d, int n, size_t smem, cudaStream_t s)
{
    cudaError_t e = tt_set_attributes();
    if (e != cudaSuccess) return e;
    k_svd_jacobi<<<n, TT_NT, smem, s>>>(d);
    return cudaGetLastError();
}

cudaError_t launch_tt_build(const TTSumDesc *d, int n, cudaStream_t s)
{
    k_tt_build<<<dim3(64, n), 256, 0, s>>>(d);
    return cudaGetLastError();
}

cudaError_t launch_tt_contract(const TTSumDesc *d, int n, cudaStream_t s)
{
    k_tt_contract<<<dim3((unsigned)sm_count(), n), 256, 0, s>>>(d);
    return cudaGetLastError();
}

cudaError_t launch_tt_gemm_tr(const GemmDesc *d, int n, cudaStream_t s)
{
    k_tt_gemm_tr<<<dim3(64, n), 256, 0, s>>>(d);
    return cudaGetLastError();
}

}  // namespace wg
