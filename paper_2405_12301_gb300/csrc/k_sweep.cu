// k_sweep.cu -- the fused per-direction residual kernel of the WENO5-JS scheme.
//
// One launch handles one direction d of one stage.  A CTA owns a tile of W
// grid lines along d, S cells each, and runs three phases through shared
// memory:
//   A. every stencil point of the tile (S + 6 per line: three ghost layers per
//      side, Sec. 4.5) is loaded once, its ghost index mapped by the boundary
//      rule, and its Lax-Friedrichs split flux f(+/-) (Sec. 2.2) computed once;
//   B. every interface flux F^_{i+1/2} = WENO(+)(f+) + WENO(-)(f-) of the tile
//      (S + 1 per line and component) is computed once, as one work item per
//      (interface, component);
//   C. every cell forms -(F^_{i+1/2} - F^_{i-1/2}) / h_d (Sec. 4.1) and the
//      epilogue stores it, adds it to the accumulator of earlier directions,
//      writes L(U), or -- for the last direction of a stage -- applies the
//      SSP-RK3 stage combination (Eq. tt-ssprk3 without rounding) and
//      publishes the wavespeed max of the new state for the next stage's alpha.
//
// FP64 mode computes everything in FP64.  FP32-bulk mode computes phases A-C
// in FP32 on differences from a per-line reference state (exact to FP32
// relative precision of the differences), and only the final state update
// U^(k+1) = U^(k) + D is an FP64 add.
//
// The model M selects the conservation law: the Euler equations (M = 0, the
// only one with an FP32-bulk form), or one scalar field u under linear
// advection with unit velocity in every direction (M = 1, f_d(u) = u, Sec. 5.1)
// or Burgers' equation (M = 2, f_d(u) = u^2 / 2, Sec. 5.2).  The scalar laws
// run through every direction of 1D, 2D and 3D grids with this kernel.
#include <type_traits>

#include "weno_dev.cuh"
#include "weno_internal.h"

namespace wg {

constexpr int NT = 256;

template <int DIR> struct Tile { static constexpr int W = 32, S = 26; };  // y, z: 32 x-lines, 26 cells
template <> struct Tile<0> { static constexpr int W = 2, S = 122; };       // x: 2 rows, 122 cells

constexpr size_t align16(size_t x) { return (x + 15) & ~size_t(15); }

template <int M> constexpr int nfields(int D) { return M == MODEL_EULER ? D + 2 : 1; }

template <int M, int D, int DIR, bool BULK> struct Layout {
    using T = typename std::conditional<BULK, float, double>::type;
    static constexpr int NF = nfields<M>(D), W = Tile<DIR>::W, S = Tile<DIR>::S, NP = S + 6, NI = S + 1;
    static constexpr size_t fp_off = 0;
    static constexpr size_t fm_off = fp_off + sizeof(T) * NF * W * NP;
    static constexpr size_t F_off = fm_off + sizeof(T) * NF * W * NP;
    static constexpr size_t ref_off = align16(F_off + sizeof(T) * NF * W * NI);
    static constexpr size_t bytes = ref_off + (BULK ? sizeof(RefState<D>) * W : 0);
};

// Split fluxes f(+/-) = (f(u) +/- alpha u) / 2 of a scalar law (Eq. lax-friedrichs).
template <int M>
__device__ __forceinline__ void split_flux_scalar(double u, double alpha, double &fp, double &fm)
{
    const double f = M == MODEL_ADVECT ? u : 0.5 * u * u;
    fp = 0.5 * (f + alpha * u);
    fm = 0.5 * (f - alpha * u);
}

template <int M, int D, int DIR, bool BULK, int EPI>
__global__ void __launch_bounds__(NT) k_sweep(const SweepArgs a)
{
    static_assert(M == MODEL_EULER || !BULK, "the FP32-bulk form exists for the Euler equations only");
    using L = Layout<M, D, DIR, BULK>;
    using T = typename L::T;
    constexpr int NF = L::NF, W = L::W, S = L::S, NP = L::NP, NI = L::NI;
    extern __shared__ __align__(16) unsigned char smem[];
    T *sfp = reinterpret_cast<T *>(smem + L::fp_off);
    T *sfm = reinterpret_cast<T *>(smem + L::fm_off);
    T *sF = reinterpret_cast<T *>(smem + L::F_off);
    RefState<D> *sref = reinterpret_cast<RefState<D> *>(smem + L::ref_off);

    const long long dtbits = __double_as_longlong(a.ctl->dt);
    if (a.check_dt && dtbits == 0) return;  // the step is a no-op (time reached t_end)
    const double dt = __longlong_as_double(dtbits);

    const long long N = a.N;
    const int n = a.n[DIR];
    const long long st = a.stride[DIR];
    int seg, lg, other;
    if (DIR == 0) { seg = blockIdx.x; lg = blockIdx.y; other = blockIdx.z; }
    else if (DIR == 1) { lg = blockIdx.x; seg = blockIdx.y; other = blockIdx.z; }
    else { lg = blockIdx.x; other = blockIdx.y; seg = blockIdx.z; }
    const int c0 = seg * S;
    // Base offset of line w of the tile; false if the line lies outside the grid.
    auto line = [&](int w, long long &base) -> bool {
        if (DIR == 0) {
            const int y = lg * W + w;
            base = (long long)other * a.stride[2] + (long long)y * a.stride[1];
            return y < a.n[1];
        }
        const int x = lg * W + w;
        base = (long long)other * (DIR == 1 ? a.stride[2] : a.stride[1]) + x;
        return x < a.n[0];
    };

    const double alpha = a.per_dir ? __longlong_as_double((long long)a.ctl->alpha_dir[a.slot_in][DIR])
                                   : __longlong_as_double((long long)a.ctl->alpha[a.slot_in]);
    const float alpha_f = BULK ? f64_to_f32(alpha) : 0.0f;  // integer pipe: cvt issues at FP64 rate
    const double gm1 = a.gamma - 1.0;
    const T eps = BULK ? (T)a.eps_f : (T)a.eps;

    // ---- phase 0 (FP32-bulk): reference state of every line
    if constexpr (BULK) {
        for (int w = threadIdx.x; w < W; w += NT) {
            long long base;
            const bool ok = line(w, base);
            double q[NF];
            const int cr = c0 < n ? c0 : n - 1;
#pragma unroll
            for (int f = 0; f < NF; ++f)
                q[f] = ok ? a.U[f * N + base + (long long)cr * st] : (f == 0 || f == NF - 1 ? 1.0 : 0.0);
            make_ref<D>(q, a.gm1_f, sref[w]);
        }
        __syncthreads();
    }

    // ---- phase A: split point fluxes of the S + 6 stencil points of every line
    for (int u = threadIdx.x; u < W * NP; u += NT) {
        int w, p;
        if (DIR == 0) { w = u / NP; p = u - w * NP; }
        else { p = u / W; w = u - p * W; }
        long long base;
        T fpv[NF], fmv[NF];
        if (line(w, base)) {
            int c = c0 - 3 + p;
            c = c < n + 2 ? c : n + 2;
            bool flip;
            int inflow;
            const int cm = ghost_map(c, n, a.bc[DIR][0], a.bc[DIR][1], flip, inflow);
            const double *src = a.U + base + (long long)cm * st;
            double q[NF];
#pragma unroll
            for (int f = 0; f < NF; ++f) q[f] = inflow >= 0 ? a.bc_state[DIR][inflow][f] : __ldg(src + f * N);
            if (M == MODEL_EULER && flip) q[1 + DIR] = -q[1 + DIR];
            if constexpr (M != MODEL_EULER) {
                split_flux_scalar<M>(q[0], alpha, fpv[0], fmv[0]);
            } else if constexpr (BULK) {
                float dq[NF];
                diff_from_ref<D>(q, sref[w], dq);
                split_flux_diff<D, DIR>(dq, sref[w], alpha_f, a.gm1_f, fpv, fmv);
            } else {
                split_flux_f64<D, DIR>(q, alpha, gm1, fpv, fmv);
            }
        } else {
#pragma unroll
            for (int f = 0; f < NF; ++f) fpv[f] = fmv[f] = T(0);
        }
#pragma unroll
        for (int f = 0; f < NF; ++f) {
            sfp[f * W * NP + u] = fpv[f];
            sfm[f * W * NP + u] = fmv[f];
        }
    }
    __syncthreads();

    // ---- phase B: interface fluxes, one work item per (interface, component)
    for (int u = threadIdx.x; u < NF * W * NI; u += NT) {
        const int f = u / (W * NI);
        const int r = u - f * (W * NI);
        int w, j;
        if (DIR == 0) { w = r / NI; j = r - w * NI; }
        else { j = r / W; w = r - j * W; }
        if (c0 + j - 1 >= n) continue;  // right of the last cell's right face
        const T *P = sfp + f * W * NP;
        const T *M = sfm + f * W * NP;
        const int pw = DIR == 0 ? w * NP : w;
        const int ps = DIR == 0 ? 1 : W;
        // interface between local cells j-1 and j: f+ at points j..j+4, f- mirrored at j+5..j+1
        const T Fh = weno5<T>(P[pw + j * ps], P[pw + (j + 1) * ps], P[pw + (j + 2) * ps], P[pw + (j + 3) * ps],
                              P[pw + (j + 4) * ps], eps) +
                     weno5<T>(M[pw + (j + 5) * ps], M[pw + (j + 4) * ps], M[pw + (j + 3) * ps],
                              M[pw + (j + 2) * ps], M[pw + (j + 1) * ps], eps);
        sF[f * W * NI + (DIR == 0 ? w * NI + j : j * W + w)] = Fh;
    }
    __syncthreads();

    // ---- phase C: flux difference and epilogue
    const T ih = BULK ? (T)a.inv_h_f[DIR] : (T)a.inv_h[DIR];
    double cmax = 0.0;
    float cmaxf = 0.0f;
    bool bad = false;
    // stage combination coefficients (Eq. tt-ssprk3): U' = a_n U^n + b_n (U^k + dt R)
    const double an = a.stage == 0 ? 0.0 : (a.stage == 1 ? 0.75 : 1.0 / 3.0);
    const double bn = a.stage == 0 ? 1.0 : (a.stage == 1 ? 0.25 : 2.0 / 3.0);
    // FP32-bulk: a_n and b_n dt as hi + lo pairs (no systematic coefficient rounding)
    const float anf = a.stage == 0 ? 0.0f : (a.stage == 1 ? 0.75f : (float)(1.0 / 3.0));
    const float anf_lo = a.stage == 2 ? (float)(1.0 / 3.0 - (double)(float)(1.0 / 3.0)) : 0.0f;
    const float2 bdtf = BULK ? f64_to_f32x2(bn * dt) : make_float2(0.0f, 0.0f);
    for (int u = threadIdx.x; u < W * S; u += NT) {
        int w, i;
        if (DIR == 0) { w = u / S; i = u - w * S; }
        else { i = u / W; w = u - i * W; }
        long long base;
        if (!line(w, base) || c0 + i >= n) continue;
        const long long cell = base + (long long)(c0 + i) * st;
        const int jl = DIR == 0 ? w * NI + i : i * W + w;
        const int jr = DIR == 0 ? jl + 1 : jl + W;
        T rd[NF];
#pragma unroll
        for (int f = 0; f < NF; ++f) rd[f] = -(sF[f * W * NI + jr] - sF[f * W * NI + jl]) * ih;
        T *acc = reinterpret_cast<T *>(a.acc);
        if (EPI == EPI_STORE) {
#pragma unroll
            for (int f = 0; f < NF; ++f) acc[f * N + cell] = rd[f];
        } else if (EPI == EPI_ADD) {
#pragma unroll
            for (int f = 0; f < NF; ++f) acc[f * N + cell] += rd[f];
        } else {
            T r[NF];
#pragma unroll
            for (int f = 0; f < NF; ++f) r[f] = (D == 1) ? rd[f] : acc[f * N + cell] + rd[f];
            if (EPI == EPI_RHS) {
#pragma unroll
                for (int f = 0; f < NF; ++f) {
                    if constexpr (BULK) a.Rout[f * N + cell] = f32_to_f64(r[f]);
                    else a.Rout[f * N + cell] = r[f];
                }
            } else {  // EPI_STAGE
                double out[NF];
#pragma unroll
                for (int f = 0; f < NF; ++f) {
                    const double uk = a.U[f * N + cell];
                    if constexpr (BULK) {
                        float hk, lk;
                        split_f64(uk, hk, lk);
                        float dlt = fmaf(bdtf.x, r[f], bdtf.y * r[f]);
                        if (a.stage > 0) {
                            float hn, ln;
                            split_f64(a.Un[f * N + cell], hn, ln);
                            const float x = (hn - hk) + (ln - lk);
                            dlt = fmaf(anf, x, fmaf(anf_lo, x, dlt));
                        }
                        out[f] = uk + f32_to_f64(dlt);
                    } else {
                        const double s = uk + dt * r[f];
                        out[f] = a.stage == 0 ? s : an * a.Un[f * N + cell] + bn * s;
                    }
                    a.Uout[f * N + cell] = out[f];
                }
                bool b;
                if constexpr (M != MODEL_EULER) {  // |f'(u)|: 1 for advection, |u| for Burgers
                    b = !isfinite(out[0]);
                    cmax = fmax(cmax, M == MODEL_ADVECT ? 1.0 : fabs(out[0]));
                } else if constexpr (BULK) {
                    float qf[NF];
#pragma unroll
                    for (int f = 0; f < NF; ++f) qf[f] = f64_to_f32(out[f]);
                    cmaxf = fmaxf(cmaxf, wavespeed_f32<D>(qf, a.gamma_f, b));
                } else {
                    cmax = fmax(cmax, wavespeed_f64<D>(out, a.gamma, b));
                }
                bad |= b;
            }
        }
    }
    if (EPI == EPI_STAGE) {
        if (BULK) cmax = (double)cmaxf;
        block_max_publish(cmax, bad, &a.ctl->alpha[a.slot_out], &a.ctl->status);
        // 1D: |u_x| + a equals |u| + a, so the x slot takes the same maximum
        if (M == MODEL_EULER && D == 1 && a.per_dir) block_max_publish(cmax, false, &a.ctl->alpha_dir[a.slot_out][0], &a.ctl->status);
    }
}

static inline unsigned cdiv(long long a, long long b) { return (unsigned)((a + b - 1) / b); }

template <int M, int D, int DIR, bool BULK, int EPI>
static cudaError_t launch_t(const SweepArgs &a, cudaStream_t s)
{
    using L = Layout<M, D, DIR, BULK>;
    dim3 grid;
    if (DIR == 0) grid = dim3(cdiv(a.n[0], L::S), cdiv(a.n[1], L::W), (unsigned)a.n[2]);
    else if (DIR == 1) grid = dim3(cdiv(a.n[0], L::W), cdiv(a.n[1], L::S), (unsigned)a.n[2]);
    else grid = dim3(cdiv(a.n[0], L::W), (unsigned)a.n[1], cdiv(a.n[2], L::S));
    k_sweep<M, D, DIR, BULK, EPI><<<grid, NT, L::bytes, s>>>(a);
    return cudaGetLastError();
}

template <int M, int D, int DIR, bool BULK, int EPI>
static cudaError_t attr_t()
{
    using L = Layout<M, D, DIR, BULK>;
    return cudaFuncSetAttribute(k_sweep<M, D, DIR, BULK, EPI>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)L::bytes);
}

// Euler: 1D grids only (2D and 3D grids run in the fused k_xy and k_z kernels).
// Scalar laws (FP64): every direction; the first stores, the middle one of 3D
// adds, the last runs the residual or stage epilogue.
#define WG_SWEEP_TABLE(X)                                                                       \
    X(MODEL_EULER, 1, 0, false, EPI_RHS) X(MODEL_EULER, 1, 0, false, EPI_STAGE)                  \
    X(MODEL_EULER, 1, 0, true, EPI_RHS) X(MODEL_EULER, 1, 0, true, EPI_STAGE)                    \
    WG_SCALAR_ROWS(X, MODEL_ADVECT) WG_SCALAR_ROWS(X, MODEL_BURGERS)
#define WG_SCALAR_ROWS(X, M)                                                                     \
    X(M, 1, 0, false, EPI_RHS) X(M, 1, 0, false, EPI_STAGE)                                      \
    X(M, 2, 0, false, EPI_STORE) X(M, 2, 1, false, EPI_RHS) X(M, 2, 1, false, EPI_STAGE)         \
    X(M, 3, 0, false, EPI_STORE) X(M, 3, 1, false, EPI_ADD) X(M, 3, 2, false, EPI_RHS)           \
    X(M, 3, 2, false, EPI_STAGE)

cudaError_t sweep_set_attributes()
{
    cudaError_t e = cudaSuccess, r;
#define X(M, D, DIR, B, E) \
    if ((r = attr_t<M, D, DIR, B, E>()) != cudaSuccess) e = r;
    WG_SWEEP_TABLE(X)
#undef X
    return e;
}

cudaError_t launch_sweep(int model, int dim, int dir, bool bulk, int epi, const SweepArgs &a, cudaStream_t s)
{
#define X(M, D, DIR, B, E) \
    if (model == M && dim == D && dir == DIR && bulk == B && epi == E) return launch_t<M, D, DIR, B, E>(a, s);
    WG_SWEEP_TABLE(X)
#undef X
    return cudaErrorInvalidValue;
}

}  // namespace wg
