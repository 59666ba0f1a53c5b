// k_cross.cu -- pointwise WENO5-JS residual at TT-cross sample points
// (Sec. 4.2-4.3, Algorithms 1 and 2), evaluated from TT cores (Eq. TT_def).
//
// Work item = one fiber (instance, sweep mode, flux direction fd, left index
// l, right index r): the n_mode samples (l, i, r), i = 0..n_mode-1.  One
// persistent launch pops fibers from an atomic counter, so uneven fiber sets
// of many instances balance across the SMs.  Per fiber the CTA contracts
// the left vector L = G_0(i_0) ... (modes before `mode`) and the right
// vector R = ... G_2(i_2) (modes after it) once; per sample the value is
// L G_mode(i) R.
//   * fd == mode: the stencil runs along the fiber itself, so the fiber's
//     values are contracted once into shared memory and every interface flux
//     is reconstructed once (as in the full-grid sweep);
//   * fd != mode: the stencil shifts the left (fd < mode) or right (fd > mode)
//     multi-index; the 7 shifted vectors are contracted once per fiber and
//     each sample forms its 7-point stencil with 7 short dot products.
// Ghost rows (Sec. 4.5) are mapped by the boundary rule of fd.
//
// FP32 mode forms stencil values as differences from a reference contracted
// from core-row differences (G(i) - G(i_ref), L^(s) - L, R^(s) - R), so the
// FP32 rounding scales with the variation along the stencil; fluxes and
// reconstruction then run on those differences as in the full-grid FP32-bulk
// path.  FP64 check mode evaluates every step in FP64.
#include "weno_dev.cuh"
#include "weno_internal.h"

namespace wg {

constexpr int XT = 128;      // threads per CTA
constexpr int XRMAX = 32;    // largest TT rank
constexpr int XNFIB = 512;   // largest n_mode of the shared-memory fiber path

template <typename T> struct XBuf {
    T L[5][XRMAX];           // centre left vector per field
    T R[5][XRMAX];           // centre right vector per field
    T S[5][6][XRMAX];        // shifted vectors (FP64) or their differences (FP32), s = -3..-1, 1..3
    T ref[5];                // fiber-path reference values (FP32)
    int item;
};

template <typename T> __device__ __forceinline__ T cvt(float x) { return (T)x; }

// Row vector of core 0 at index i (r1 entries) or of core 2 (r2 entries).
template <typename T>
__device__ __forceinline__ T core_edge(const float *core, int i, int r, int a)
{
    return cvt<T>(__ldg(core + (long long)i * r + a));
}

// L_b = sum_a G0(i0)_a G1(i1)_{a b}  (mode 2 left vector), or
// R_a = sum_b G1(j)_{a b} G2(k)_b    (mode 0 right vector).
template <typename T>
__device__ __forceinline__ T two_core_left(const CrossInst &in, int f, int i0, int i1, int b)
{
    const int r1 = in.r[0], r2 = in.r[1];
    const float *g0 = in.core[f][0] + (long long)i0 * r1;
    const float *g1 = in.core[f][1] + (long long)i1 * r1 * r2;
    T s = T(0);
    for (int a = 0; a < r1; ++a) s += cvt<T>(__ldg(g0 + a)) * cvt<T>(__ldg(g1 + a * r2 + b));
    return s;
}
template <typename T>
__device__ __forceinline__ T two_core_right(const CrossInst &in, int f, int j, int k, int a)
{
    const int r1 = in.r[0], r2 = in.r[1];
    const float *g1 = in.core[f][1] + (long long)j * r1 * r2 + a * r2;
    const float *g2 = in.core[f][2] + (long long)k * r2;
    T s = T(0);
    for (int b = 0; b < r2; ++b) s += cvt<T>(__ldg(g1 + b)) * cvt<T>(__ldg(g2 + b));
    return s;
}

// Index of a stencil row along mode m after the boundary rule of fd.
__device__ __forceinline__ int xmap(const CrossInst &in, int m, int c, bool &flip)
{
    return ghost_source(c, in.n[m], in.bc[m][0], in.bc[m][1], flip);
}

// Left (mode > 0) / right (mode < 2) vector entry `a` of field f for the
// sample's multi-indices; `shift` moves the index of mode fd by s.
template <typename T>
__device__ T left_vec(const CrossInst &in, int mode, const int *lidx, int f, int a, int fd, int s, bool &flip)
{
    flip = false;
    if (mode == 1) {
        int i0 = lidx[0];
        if (fd == 0) i0 = xmap(in, 0, i0 + s, flip);
        return core_edge<T>(in.core[f][0], i0, in.r[0], a);
    }
    int i0 = lidx[0], i1 = lidx[1];
    if (fd == 0) i0 = xmap(in, 0, i0 + s, flip);
    if (fd == 1) i1 = xmap(in, 1, i1 + s, flip);
    return two_core_left<T>(in, f, i0, i1, a);
}
template <typename T>
__device__ T right_vec(const CrossInst &in, int mode, const int *ridx, int f, int a, int fd, int s, bool &flip)
{
    flip = false;
    if (mode == 1) {
        int k = ridx[0];
        if (fd == 2) k = xmap(in, 2, k + s, flip);
        return core_edge<T>(in.core[f][2], k, in.r[1], a);
    }
    int j = ridx[0], k = ridx[1];
    if (fd == 1) j = xmap(in, 1, j + s, flip);
    if (fd == 2) k = xmap(in, 2, k + s, flip);
    return two_core_right<T>(in, f, j, k, a);
}

// t = G_mode(i) R  (length r_{mode-1})  or  t = L G_mode(i)  (length r_mode),
// or the scalar L G_mode(i) R.
template <typename T>
__device__ __forceinline__ T contract_LGR(const CrossInst &in, int mode, int f, int i, const T *L, const T *R)
{
    const int rl = mode == 0 ? 1 : in.r[mode - 1];
    const int rr = mode == 2 ? 1 : in.r[mode];
    const float *g = in.core[f][mode] + (long long)i * rl * rr;
    T s = T(0);
    for (int a = 0; a < rl; ++a) {
        T row = T(0);
        for (int b = 0; b < rr; ++b) row += cvt<T>(__ldg(g + a * rr + b)) * R[b];
        s += L[a] * row;
    }
    return s;
}

template <bool F64>
__global__ void __launch_bounds__(XT) k_cross(const CrossArgs A)
{
    using T = typename std::conditional<F64, double, float>::type;
    __shared__ XBuf<T> sb;
    extern __shared__ __align__(16) unsigned char dyn[];
    T *vals = reinterpret_cast<T *>(dyn);     // [5][XNFIB]
    T *fpv = vals + 5 * XNFIB;                 // [5][XNFIB + 6]
    T *fmv = fpv + 5 * (XNFIB + 6);            // [5][XNFIB + 6]
    T *Fh = fmv + 5 * (XNFIB + 6);             // [5][XNFIB + 1]
    const T eps = (T)A.eps;
    const double gm1 = A.gamma - 1.0;

    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) sb.item = (int)atomicAdd(A.counter, 1ull);
        __syncthreads();
        const long long item = sb.item;
        if (item >= A.n_work) break;
        // locate the fiber set (binary search on work_begin)
        int lo = 0, hi = A.n_sets - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (A.sets[mid].work_begin <= item) lo = mid;
            else hi = mid - 1;
        }
        const CrossSet &S = A.sets[lo];
        const CrossInst &in = A.inst[S.inst];
        const int mode = S.mode, fd = S.fd, n = S.n_mode;
        const long long q = item - S.work_begin;
        const long long l = q / S.n_right, rr = q - l * S.n_right;
        const int *lidx = mode > 0 ? S.left + l * mode : nullptr;
        const int *ridx = mode < 2 ? S.right + rr * (2 - mode) : nullptr;
        const int rlen = mode == 0 ? 1 : in.r[mode - 1];
        const int rrlen = mode == 2 ? 1 : in.r[mode];
        // index sets live in device memory: check them here and skip a fiber
        // whose multi-indices fall outside the modes (reported, never read)
        bool badidx = false;
        for (int m = 0; m < mode; ++m) badidx |= (unsigned)lidx[m] >= (unsigned)in.n[m];
        for (int m = 0; m < 2 - mode; ++m) badidx |= (unsigned)ridx[m] >= (unsigned)in.n[mode + 1 + m];
        if (badidx) {
            if (threadIdx.x == 0) atomicOr(A.status, ST_BADINDEX);
            continue;
        }
        const T alpha = (T)in.alpha;
        const T ih = (T)(1.0 / in.h[fd]);

        // ---- fiber setup: centre and shifted left/right vectors
        for (int u = threadIdx.x; u < 5 * XRMAX; u += XT) {
            const int f = u / XRMAX, a = u - f * XRMAX;
            bool fl;
            sb.L[f][a] = (mode > 0 && a < rlen) ? left_vec<T>(in, mode, lidx, f, a, -1, 0, fl) : T(a == 0 && mode == 0);
            sb.R[f][a] = (mode < 2 && a < rrlen) ? right_vec<T>(in, mode, ridx, f, a, -1, 0, fl) : T(a == 0 && mode == 2);
        }
        const bool shiftL = fd < mode, shiftR = fd > mode;
        if (shiftL || shiftR) {
            __syncthreads();
            const int len = shiftL ? rlen : rrlen;
            for (int u = threadIdx.x; u < 5 * 6 * len; u += XT) {
                const int f = u / (6 * len), rem = u - f * 6 * len, k = rem / len, a = rem - k * len;
                const int s = k < 3 ? k - 3 : k - 2;
                bool fl;
                T v = shiftL ? left_vec<T>(in, mode, lidx, f, a, fd, s, fl) : right_vec<T>(in, mode, ridx, f, a, fd, s, fl);
                if (fl && f == 1 + fd) v = -v;  // mirrored ghost row: normal momentum negated
                if (!F64) v -= shiftL ? sb.L[f][a] : sb.R[f][a];
                sb.S[f][k][a] = v;
            }
        }
        __syncthreads();

        if (fd == mode && n <= XNFIB) {
            // ---- stencil along the fiber: values once, interfaces once
            const int iref = 0;
            for (int u = threadIdx.x; u < 5 * n; u += XT) {
                const int f = u / n, i = u - f * n;
                T v = (F64 || i == iref) ? contract_LGR<T>(in, mode, f, i, sb.L[f], sb.R[f]) : T(0);
                if (!F64) {
                    // difference from the fiber reference, from core-row differences
                    const float *g = in.core[f][mode];
                    const long long sz = (long long)rlen * rrlen;
                    T s = T(0);
                    for (int a = 0; a < rlen; ++a) {
                        T row = T(0);
                        for (int b = 0; b < rrlen; ++b)
                            row += (__ldg(g + i * sz + a * rrlen + b) - __ldg(g + iref * sz + a * rrlen + b)) * sb.R[f][b];
                        s += sb.L[f][a] * row;
                    }
                    if (i == iref) sb.ref[f] = v;
                    v = s;
                }
                vals[f * XNFIB + i] = v;
            }
            __syncthreads();
            // split point fluxes at the n + 6 points (three ghost layers per side)
            for (int p = threadIdx.x; p < n + 6; p += XT) {
                bool flip;
                const int c = xmap(in, fd, p - 3, flip);
                T q5[5], fpl[5], fml[5];
                for (int f = 0; f < 5; ++f) q5[f] = vals[f * XNFIB + c];
                if constexpr (F64) {
                    if (flip) q5[1 + fd] = -q5[1 + fd];
                    double qd[5], a5[5], b5[5];
                    for (int f = 0; f < 5; ++f) qd[f] = q5[f];
                    if (fd == 0) split_flux_f64<3, 0>(qd, (double)alpha, gm1, a5, b5);
                    else if (fd == 1) split_flux_f64<3, 1>(qd, (double)alpha, gm1, a5, b5);
                    else split_flux_f64<3, 2>(qd, (double)alpha, gm1, a5, b5);
                    for (int f = 0; f < 5; ++f) { fpl[f] = a5[f]; fml[f] = b5[f]; }
                } else {
                    if (flip) q5[1 + fd] = -q5[1 + fd] - 2.0f * sb.ref[1 + fd];  // -(ref + d) - ref
                    RefState<3> rs;
                    float rq[5];
                    for (int f = 0; f < 5; ++f) { rs.hi[f] = sb.ref[f]; rs.lo[f] = 0.0f; rq[f] = sb.ref[f]; }
                    {
                        const float ir = 1.0f / rq[0];
                        float ke = 0.0f;
                        rs.rho = rq[0];
                        for (int e = 0; e < 3; ++e) { rs.m[e] = rq[1 + e]; rs.u[e] = rq[1 + e] * ir; ke += rs.m[e] * rs.u[e]; }
                        rs.H = rq[4] + (float)gm1 * (rq[4] - 0.5f * ke);
                    }
                    float a5[5], b5[5];
                    if (fd == 0) split_flux_diff<3, 0>(q5, rs, alpha, (float)gm1, a5, b5);
                    else if (fd == 1) split_flux_diff<3, 1>(q5, rs, alpha, (float)gm1, a5, b5);
                    else split_flux_diff<3, 2>(q5, rs, alpha, (float)gm1, a5, b5);
                    for (int f = 0; f < 5; ++f) { fpl[f] = a5[f]; fml[f] = b5[f]; }
                }
                for (int f = 0; f < 5; ++f) {
                    fpv[f * (XNFIB + 6) + p] = fpl[f];
                    fmv[f * (XNFIB + 6) + p] = fml[f];
                }
            }
            __syncthreads();
            for (int u = threadIdx.x; u < 5 * (n + 1); u += XT) {
                const int f = u / (n + 1), j = u - f * (n + 1);
                const T *P = fpv + f * (XNFIB + 6);
                const T *M = fmv + f * (XNFIB + 6);
                Fh[f * (XNFIB + 1) + j] = weno5<T>(P[j], P[j + 1], P[j + 2], P[j + 3], P[j + 4], eps) +
                                          weno5<T>(M[j + 5], M[j + 4], M[j + 3], M[j + 2], M[j + 1], eps);
            }
            __syncthreads();
            for (int u = threadIdx.x; u < 5 * n; u += XT) {
                const int f = u / n, i = u - f * n;
                const T rd = -(Fh[f * (XNFIB + 1) + i + 1] - Fh[f * (XNFIB + 1) + i]) * ih;
                const long long o = (((long long)f * S.n_left + l) * n + i) * S.n_right + rr;
                reinterpret_cast<T *>(S.out)[o] = rd;
            }
            continue;
        }

        // ---- per-sample stencils (fd != mode, or fibers longer than XNFIB)
        for (int i = threadIdx.x; i < n; i += XT) {
            T q7[5][7];  // stencil values (FP64) or differences from the centre (FP32)
            T ctr[5];    // centre values
            for (int f = 0; f < 5; ++f) {
                const float *g = in.core[f][mode];
                const long long sz = (long long)rlen * rrlen;
                if (fd == mode) {
                    ctr[f] = contract_LGR<T>(in, mode, f, i, sb.L[f], sb.R[f]);
                    for (int s = -3; s <= 3; ++s) {
                        bool fl;
                        const int c = xmap(in, fd, i + s, fl);
                        T v;
                        if constexpr (F64) {
                            v = contract_LGR<T>(in, mode, f, c, sb.L[f], sb.R[f]);
                            if (fl && f == 1 + fd) v = -v;
                        } else {
                            T d = T(0);  // L (G(c) - G(i)) R
                            for (int a = 0; a < rlen; ++a) {
                                T row = T(0);
                                for (int b = 0; b < rrlen; ++b)
                                    row += (__ldg(g + c * sz + a * rrlen + b) - __ldg(g + i * sz + a * rrlen + b)) *
                                           sb.R[f][b];
                                d += sb.L[f][a] * row;
                            }
                            v = (fl && f == 1 + fd) ? -d - T(2) * ctr[f] : d;
                        }
                        q7[f][s + 3] = v;
                    }
                    continue;
                }
                // t = G(i) R (the shift moves L) or t = L G(i) (the shift moves R)
                T t[XRMAX];
                const int tl = shiftL ? rlen : rrlen;
                for (int a = 0; a < tl; ++a) t[a] = T(0);
                for (int a = 0; a < rlen; ++a)
                    for (int b = 0; b < rrlen; ++b) {
                        const T gv = cvt<T>(__ldg(g + i * sz + a * rrlen + b));
                        if (shiftL) t[a] += gv * sb.R[f][b];
                        else t[b] += sb.L[f][a] * gv;
                    }
                const T *cv = shiftL ? sb.L[f] : sb.R[f];
                T c0 = T(0);
                for (int a = 0; a < tl; ++a) c0 += cv[a] * t[a];
                ctr[f] = c0;
                q7[f][3] = F64 ? c0 : T(0);
                for (int k = 0; k < 6; ++k) {
                    T v = T(0);
                    for (int a = 0; a < tl; ++a) v += sb.S[f][k][a] * t[a];
                    q7[f][k < 3 ? k : k + 1] = v;
                }
            }
            // split fluxes at the 7 points, then interfaces i-1/2 (points 0..5) and i+1/2 (1..6)
            T fp7[5][7], fm7[5][7];
            if constexpr (F64) {
                for (int k = 0; k < 7; ++k) {
                    double qd[5], a5[5], b5[5];
                    for (int f = 0; f < 5; ++f) qd[f] = q7[f][k];
                    if (fd == 0) split_flux_f64<3, 0>(qd, (double)alpha, gm1, a5, b5);
                    else if (fd == 1) split_flux_f64<3, 1>(qd, (double)alpha, gm1, a5, b5);
                    else split_flux_f64<3, 2>(qd, (double)alpha, gm1, a5, b5);
                    for (int f = 0; f < 5; ++f) { fp7[f][k] = a5[f]; fm7[f][k] = b5[f]; }
                }
            } else {
                RefState<3> rs;
                {
                    for (int f = 0; f < 5; ++f) { rs.hi[f] = ctr[f]; rs.lo[f] = 0.0f; }
                    const float ir = 1.0f / ctr[0];
                    float ke = 0.0f;
                    rs.rho = ctr[0];
                    for (int e = 0; e < 3; ++e) { rs.m[e] = ctr[1 + e]; rs.u[e] = ctr[1 + e] * ir; ke += rs.m[e] * rs.u[e]; }
                    rs.H = ctr[4] + (float)gm1 * (ctr[4] - 0.5f * ke);
                }
                for (int k = 0; k < 7; ++k) {
                    float dq[5], a5[5], b5[5];
                    for (int f = 0; f < 5; ++f) dq[f] = q7[f][k];
                    if (fd == 0) split_flux_diff<3, 0>(dq, rs, alpha, (float)gm1, a5, b5);
                    else if (fd == 1) split_flux_diff<3, 1>(dq, rs, alpha, (float)gm1, a5, b5);
                    else split_flux_diff<3, 2>(dq, rs, alpha, (float)gm1, a5, b5);
                    for (int f = 0; f < 5; ++f) { fp7[f][k] = a5[f]; fm7[f][k] = b5[f]; }
                }
            }
            for (int f = 0; f < 5; ++f) {
                const T *P = fp7[f], *M = fm7[f];
                const T Flo = weno5<T>(P[0], P[1], P[2], P[3], P[4], eps) + weno5<T>(M[5], M[4], M[3], M[2], M[1], eps);
                const T Fhi = weno5<T>(P[1], P[2], P[3], P[4], P[5], eps) + weno5<T>(M[6], M[5], M[4], M[3], M[2], eps);
                const long long o = (((long long)f * S.n_left + l) * n + i) * S.n_right + rr;
                reinterpret_cast<T *>(S.out)[o] = -(Fhi - Flo) * ih;
            }
        }
    }
}

static size_t cross_dyn_bytes(bool f64)
{
    const size_t e = f64 ? sizeof(double) : sizeof(float);
    return e * (size_t)(5 * XNFIB + 2 * 5 * (XNFIB + 6) + 5 * (XNFIB + 1));
}

cudaError_t launch_cross(const CrossArgs &a, cudaStream_t s)
{
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(k_cross<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)cross_dyn_bytes(false));
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(k_cross<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)cross_dyn_bytes(true));
        if (e != cudaSuccess) return e;
        attr = true;
    }
    long long blocks = a.n_work < 152 * 4 ? a.n_work : 152 * 4;
    if (blocks < 1) blocks = 1;
    if (a.fp64) k_cross<true><<<(unsigned)blocks, XT, cross_dyn_bytes(true), s>>>(a);
    else k_cross<false><<<(unsigned)blocks, XT, cross_dyn_bytes(false), s>>>(a);
    return cudaGetLastError();
}

int cross_max_rank() { return XRMAX; }

}  // namespace wg
