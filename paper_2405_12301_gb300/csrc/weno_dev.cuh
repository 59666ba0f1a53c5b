// weno_dev.cuh -- device building blocks of the GB300 WENO5-JS residual:
// FP64 <-> FP32 conversions on the integer pipe, ghost-index mapping,
// WENO5-JS reconstruction, point fluxes with Lax-Friedrichs splitting, and the
// device control block.
//
// On GB300 the FP64 pipe (DFMA/DADD) and the FP32<->FP64 conversion
// instructions both issue at about 1.7 per clock per SM, against about 86
// FFMA per clock per SM, so the FP32-bulk path never converts with cvt and
// keeps FP64 arithmetic to one DADD per field per stage.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace wg {

enum { BC_PERIODIC = 0, BC_TRANSMISSIVE = 1, BC_REFLECTIVE = 2, BC_INFLOW = 3 };
enum { ST_NONPHYSICAL = 1, ST_TIMEOUT = 2, ST_BADINDEX = 4 };

// Device control block of one handle: time, step size and the stage alphas.
// alpha[s] holds the bit pattern of a non-negative double so that atomicMax
// on the 64-bit integer is a max on the value (order-independent, so the
// result is bitwise deterministic).  Slot 0: alpha(U^n); slots 1..3: alpha of
// the states written by stages 1..3.
struct Ctl {
    double t;              // current time
    double t_next;         // time after the current step
    double dt;             // dt of the current step (0: the step is a no-op)
    double t_end;
    double dt_req;         // > 0: fixed dt; otherwise CFL
    double cfl_h;          // cfl * min_d h_d
    unsigned long long alpha[4];
    unsigned long long alpha_dir[4][3];  // per-direction max(|u_d| + a), same slots (per-direction mode)
    long long steps;       // steps taken since the last set_time
    long long max_steps;   // steps bound of the current run call
    int status;            // ST_* bits, latched
    int pad;
    float2 bdt[3];         // b_k dt of stage k (1, 1/4, 2/3) as FP32 pairs hi + lo, set with dt
};

// ----------------------------------------------------------------- conversions

// Splits a finite FP64 x into FP32 hi + lo: hi is x truncated to 24 significant
// bits, lo approximates x - hi (the next 23 bits), on the integer pipe plus one
// FSUB.  hi: a funnel shift lines the exponent and mantissa up with the FP32
// fields and one add rebiases the exponent by 1023 - 127.  lo: the low 29
// mantissa bits m29 are worth m29 * 2^(e-1075); 2^E (1 + (m29 >> 6) / 2^23) with
// E = e - 1046, minus 2^E, gives that value (exact, up to the 6 dropped bits).
// |x| < 2^-103 (and zero) gives hi = lo = +-0; |x| >= 2^128 is not representable
// (states that large are non-physical).
__device__ __forceinline__ void split_f64(double x, float &hi, float &lo)
{
    const unsigned xh = (unsigned)__double2hiint(x);
    const unsigned xl = (unsigned)__double2loint(x);
    const unsigned sgn = xh & 0x80000000u;
    const unsigned fs = __funnelshift_l(xl, xh, 3) + 0x40000000u;  // [e - 896 : 8][mantissa : 23]
    const unsigned hb = (fs & 0x7FFFFFFFu) | sgn;
    const unsigned eb = (fs - 0x0B800000u) & 0x7F800000u;          // exponent field of 2^(e - 1046)
    const float l = __uint_as_float(eb | ((xl >> 6) & 0x7FFFFFu)) - __uint_as_float(eb);
    const bool ok = ((xh >> 20) & 0x7FFu) >= 920u;
    hi = __uint_as_float(ok ? hb : sgn);
    lo = __uint_as_float(ok ? (__float_as_uint(l) | sgn) : sgn);
}

// FP32 -> FP64, exact for normal numbers (subnormals flush to +-0).
__device__ __forceinline__ double f32_to_f64(float f)
{
    const unsigned b = __float_as_uint(f);
    const unsigned e = (b >> 23) & 0xFFu;
    const unsigned sgn = b & 0x80000000u;
    unsigned hi = sgn | ((e + 896u) << 20) | ((b >> 3) & 0xFFFFFu);
    unsigned lo = b << 29;
    if (e == 0u) { hi = sgn; lo = 0u; }
    if (e == 255u) { hi = sgn | 0x7FF00000u | ((b >> 3) & 0xFFFFFu); }
    return __hiloint2double((int)hi, (int)lo);
}

// FP64 -> FP32 by truncation (hi part of split_f64), integer pipe only.
__device__ __forceinline__ float f64_to_f32(double x)
{
    float hi, lo;
    split_f64(x, hi, lo);
    return hi + lo;
}

// An FP64 coefficient as an unevaluated FP32 pair hi + lo (to about 2^-48
// relative): multiplying by hi alone would bias every use the same way by up
// to 2^-24, which over many time steps is a systematic error.
__device__ __forceinline__ float2 f64_to_f32x2(double x)
{
    const float hi = f64_to_f32(x);
    return make_float2(hi, f64_to_f32(x - f32_to_f64(hi)));
}

__device__ __forceinline__ float fast_rcp(float x)
{
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// ------------------------------------------------------------------ ghosts

// Interior source index of a (possibly ghost) index c in [-3, n+2] along a
// direction with n >= 3 cells (Sec. 4.5): periodic wraps, transmissive clamps,
// reflective mirrors (and the caller negates the normal momentum).
__device__ __forceinline__ int ghost_source(int c, int n, int bclo, int bchi, bool &flip)
{
    flip = false;
    if (c < 0) {
        if (bclo == BC_PERIODIC) return c + n;
        if (bclo == BC_TRANSMISSIVE) return 0;
        flip = true;
        return -1 - c;
    }
    if (c >= n) {
        if (bchi == BC_PERIODIC) return c - n;
        if (bchi == BC_TRANSMISSIVE) return n - 1;
        flip = true;
        return 2 * n - 1 - c;
    }
    return c;
}

// Full-grid ghost mapping: as ghost_source, plus inflow sides, whose ghosts
// hold a given state: *inflow is set to the side (0 low, 1 high) and a valid
// interior index is returned (the caller replaces the value); -1 otherwise.
__device__ __forceinline__ int ghost_map(int c, int n, int bclo, int bchi, bool &flip, int &inflow)
{
    inflow = -1;
    if (c < 0 && bclo == BC_INFLOW) {
        flip = false;
        inflow = 0;
        return 0;
    }
    if (c >= n && bchi == BC_INFLOW) {
        flip = false;
        inflow = 1;
        return n - 1;
    }
    return ghost_source(c, n, bclo, bchi, flip);
}

// ---------------------------------------------------------------- WENO5-JS

template <typename T> __device__ __forceinline__ T div_(T a, T b);
template <> __device__ __forceinline__ double div_<double>(double a, double b) { return a / b; }
template <> __device__ __forceinline__ float div_<float>(float a, float b) { return a * fast_rcp(b); }

// Value at x_{i+1/2} reconstructed from (a, b, c, d, e) = v_{i-2}, ..., v_{i+2}
// (Sec. 2.2): candidates v^(r), smoothness indicators beta_r, weights
// alpha_r = d_r / (beta_r + eps)^2 normalised to sum one.  Written on the
// first differences D1..D4 (D1 = b - a, ..., D4 = e - d), in which
//   beta_0 = 13/12 (D4 - D3)^2 + 1/4 (D4 - 3 D3)^2,
//   beta_1 = 13/12 (D3 - D2)^2 + 1/4 (D2 + D3)^2,
//   beta_2 = 13/12 (D2 - D1)^2 + 1/4 (3 D2 - D1)^2,
//   v^(1) = c + (D2 + 2 D3)/6,  v^(0) - v^(1) = (t1 - t0)/6,  v^(2) - v^(1) = -2 (t1 - t2)/6,
// t_r the second differences above, so with w_r = d_r g_s g_t (g = (beta + eps)^2,
// {s, t} the other two indices; w_r / sum w = omega_r)
//   sum_r omega_r v^(r) = c + [(D2 + 2 D3) sum w + w_0 (t1 - t0) - 2 w_2 (t1 - t2)] / (6 sum w),
// the same quantity with one division.
template <typename T>
__device__ __forceinline__ T weno5(T a, T b, T c, T d, T e, T eps)
{
    const T D1 = b - a, D2 = c - b, D3 = d - c, D4 = e - d;
    const T t0 = D4 - D3, t1 = D3 - D2, t2 = D2 - D1;
    const T s0 = fma(T(-3), D3, D4), s1 = D2 + D3, s2 = fma(T(3), D2, -D1);
    const T k13 = T(13.0 / 12.0), q = T(0.25);
    T g0 = fma(k13 * t0, t0, fma(q * s0, s0, eps));
    T g1 = fma(k13 * t1, t1, fma(q * s1, s1, eps));
    T g2 = fma(k13 * t2, t2, fma(q * s2, s2, eps));
    g0 *= g0;
    g1 *= g1;
    g2 *= g2;
    const T w0 = T(0.3) * (g1 * g2), w1 = T(0.6) * (g0 * g2), w2 = T(0.1) * (g0 * g1);
    const T sw = w0 + w1 + w2;
    const T num = fma(w0, t1 - t0, fma(T(-2) * w2, t1 - t2, fma(T(2), D3, D2) * sw));
    return c + div_<T>(num, T(6) * sw);
}

// WENO5 of K consecutive windows along a line, sharing what neighbouring
// windows have in common: window m is (p[m s], ..., p[(m + 4) s]) and its value
// goes to out[m os].  Moving to the next window drops the first point, so its
// first differences D1..D3, second differences t1, t2 and the 13/12 t^2 parts
// of beta_1, beta_2 are the previous window's D2..D4, t0, t1 and beta_0, beta_1
// parts; each window loads one new point and forms one new difference of each
// kind.  Every window's value is formed from its five points by the same
// operations wherever it sits in the run (the first window forms its shared
// terms directly from the same differences), so a face computed by two runs
// gets bitwise the same value.  A negative stride s walks a line backwards,
// which turns the run into the mirrored WENO(-) of the faces in reverse order.
template <typename T, int K>
__device__ __forceinline__ void weno5_slide(const T *p, int s, T eps, T *out, int os)
{
    const T k13 = T(13.0 / 12.0), q = T(0.25);
    const T v0 = *p, v1 = *(p += s);
    T c = *(p += s), d = *(p += s);
    T D1 = v1 - v0, D2 = c - v1, D3 = d - c;
    T t1 = D3 - D2, t2 = D2 - D1;
    T A1 = fma(k13 * t1, t1, eps), A2 = fma(k13 * t2, t2, eps);
#pragma unroll
    for (int m = 0; m < K; ++m) {
        const T e = *(p += s);
        const T D4 = e - d;
        const T t0 = D4 - D3;
        const T A0 = fma(k13 * t0, t0, eps);
        const T s0 = fma(T(-3), D3, D4), s1 = D2 + D3, s2 = fma(T(3), D2, -D1);
        T g0 = fma(q * s0, s0, A0), g1 = fma(q * s1, s1, A1), g2 = fma(q * s2, s2, A2);
        g0 *= g0;
        g1 *= g1;
        g2 *= g2;
        const T w0 = T(0.3) * (g1 * g2), w1 = T(0.6) * (g0 * g2), w2 = T(0.1) * (g0 * g1);
        const T sw = w0 + w1 + w2;
        const T num = fma(w0, t1 - t0, fma(T(-2) * w2, t1 - t2, fma(T(2), D3, D2) * sw));
        *out = c + div_<T>(num, T(6) * sw);
        out += os;
        D1 = D2;
        D2 = D3;
        D3 = D4;
        t2 = t1;
        t1 = t0;
        A2 = A1;
        A1 = A0;
        c = d;
        d = e;
    }
}

// ------------------------------------------------- packed FP32 pairs (f32x2)
// Two independent FP32 streams in one float2: a .f32x2 instruction takes one
// issue slot for both operations (the FMA pipe still does two), which is what
// an issue-bound kernel needs.  Each lane of a pair is rounded exactly as the
// scalar operation would round it.
__device__ __forceinline__ float2 bc2(float x) { return make_float2(x, x); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b)
{
    unsigned long long r;
    asm("sub.rn.f32x2 %0, %1, %2;"
        : "=l"(r)
        : "l"(*reinterpret_cast<const unsigned long long *>(&a)), "l"(*reinterpret_cast<const unsigned long long *>(&b)));
    return *reinterpret_cast<const float2 *>(&r);
}

// weno5 of a face's WENO(+) window (lane x) and its mirrored WENO(-) window
// (lane y) at once, returning their sum (the face flux): the same operations
// as weno5<float> on each lane; beta_2's (3 D2 - D1) is formed negated (it
// enters squared only).
__device__ __forceinline__ float weno5_pm(float2 a, float2 b, float2 c, float2 d, float2 e, float eps_)
{
    const float2 D1 = sub2(b, a), D2 = sub2(c, b), D3 = sub2(d, c), D4 = sub2(e, d);
    const float2 t0 = sub2(D4, D3), t1 = sub2(D3, D2), t2 = sub2(D2, D1);
    const float2 s0 = fma2(bc2(-3.0f), D3, D4), s1 = add2(D2, D3), s2 = fma2(bc2(-3.0f), D2, D1);
    const float2 k13 = bc2((float)(13.0 / 12.0)), q = bc2(0.25f), eps = bc2(eps_);
    float2 g0 = fma2(mul2(k13, t0), t0, fma2(mul2(q, s0), s0, eps));
    float2 g1 = fma2(mul2(k13, t1), t1, fma2(mul2(q, s1), s1, eps));
    float2 g2 = fma2(mul2(k13, t2), t2, fma2(mul2(q, s2), s2, eps));
    g0 = mul2(g0, g0);
    g1 = mul2(g1, g1);
    g2 = mul2(g2, g2);
    const float2 w0 = mul2(bc2(0.3f), mul2(g1, g2)), w1 = mul2(bc2(0.6f), mul2(g0, g2)),
                 w2 = mul2(bc2(0.1f), mul2(g0, g1));
    const float2 sw = add2(add2(w0, w1), w2);
    const float2 num =
        fma2(w0, sub2(t1, t0), fma2(mul2(bc2(-2.0f), w2), sub2(t1, t2), mul2(fma2(bc2(2.0f), D3, D2), sw)));
    const float2 den = mul2(bc2(6.0f), sw);
    const float2 v = fma2(num, make_float2(fast_rcp(den.x), fast_rcp(den.y)), c);
    return v.x + v.y;
}

// WENO5 correction of K consecutive windows along a line, from scaled first
// differences (two streams as float2 pairs).  With v the values whose
// reconstruction is wanted, D_k their first differences and t_r, s_r the
// second differences and beta parts of the weno5 comment, the correction of a
// window to its centre value c is
//   sum_r omega_r v^(r) - c = (D2 + 2 D3)/6 + (w0 (t1 - t0) - 2 w2 (t1 - t2)) / (6 sum w).
// p holds Dt = s D for a scale s, and the run returns 6 s times the correction:
//   6 s (sum_r omega_r v^(r) - c) = Ft + (w0 (tt1 - tt0) - 2 w2 (tt1 - tt2)) / sum w,
//   Ft = Dt2 + 2 Dt3,  tt = s t,
// with (13/3) tt_r^2 + st_r^2 = 4 s^2 beta_r (st = s s_r), so that
// G_r = (13/3) tt_r^2 + st_r^2 + Geps with Geps = 4 s^2 eps is 4 s^2 (beta_r + eps),
// and the weights w_r = d_r / G_r^2 up to a common factor are formed as
// (3 g1 g2, 6 g0 g2, g0 g1) with g = G^2 (d = (3, 6, 1) / 10).  Window m takes
// Dt1..Dt4 = p[m s] .. p[(m + 3) s] and writes to out[m os]; each window loads
// one new difference, and its -2 (tt1 - tt2) is twice the previous window's
// (tt1 - tt0), carried.  A mirrored window is the same run over the negated
// differences read backwards (the caller stores them negated).
template <int K>
__device__ __forceinline__ void weno5d_slide2(const float2 *p, int s, float Geps_, float2 *out, int os)
{
    const float2 k = bc2((float)(13.0 / 3.0)), Geps = bc2(Geps_);
    float2 D1 = *p, D2 = *(p += s), D3 = *(p += s);
    float2 t1 = sub2(D3, D2), t2 = sub2(D2, D1);
    float2 A1 = fma2(mul2(k, t1), t1, Geps), A2 = fma2(mul2(k, t2), t2, Geps);
    float2 h = mul2(bc2(-2.0f), sub2(t1, t2));
#pragma unroll
    for (int m = 0; m < K; ++m) {
        const float2 D4 = *(p += s);
        const float2 t0 = sub2(D4, D3);
        const float2 A0 = fma2(mul2(k, t0), t0, Geps);
        const float2 s0 = fma2(bc2(-3.0f), D3, D4), s1 = add2(D2, D3), s2 = fma2(bc2(-3.0f), D2, D1);
        float2 g0 = fma2(s0, s0, A0), g1 = fma2(s1, s1, A1), g2 = fma2(s2, s2, A2);
        g0 = mul2(g0, g0);
        g1 = mul2(g1, g1);
        g2 = mul2(g2, g2);
        const float2 w0 = mul2(g1, g2), w1 = mul2(g0, g2), w2 = mul2(g0, g1);  // times 3, 6, 1
        const float2 sw = fma2(bc2(3.0f), w0, fma2(bc2(6.0f), w1, w2));
        const float2 e0 = sub2(t1, t0);
        const float2 num = fma2(w0, mul2(bc2(3.0f), e0), mul2(w2, h));
        const float2 F = fma2(bc2(2.0f), D3, D2);
        *out = fma2(num, make_float2(fast_rcp(sw.x), fast_rcp(sw.y)), F);
        out += os;
        h = add2(e0, e0);
        D1 = D2;
        D2 = D3;
        D3 = D4;
        t2 = t1;
        t1 = t0;
        A2 = A1;
        A1 = A0;
    }
}

// The same run, emitting per cell instead of per face: with C_m the run's
// output for window m, cell m - 1 (between the faces of windows m - 1 and m)
// receives 6 D2_m + (C_m - C_{m-1}) (FWD; D2_m the window's second
// difference, the cell's own pair), or -6 D2_m + (C_{m-1} - C_m) for a run read
// backwards (!FWD), K - 1 values to out[(m - 1) os].  Those are 6 s times the
// parts of a cell's flux difference that one run contributes (k_xy2 phase C).
template <int K, bool FWD>
__device__ __forceinline__ void weno5d_cells2(const float2 *p, int s, float Geps_, float2 *out, int os)
{
    const float2 k = bc2((float)(13.0 / 3.0)), Geps = bc2(Geps_), six = bc2(FWD ? 6.0f : -6.0f);
    float2 D1 = *p, D2 = *(p += s), D3 = *(p += s);
    float2 t1 = sub2(D3, D2), t2 = sub2(D2, D1);
    float2 A1 = fma2(mul2(k, t1), t1, Geps), A2 = fma2(mul2(k, t2), t2, Geps);
    float2 h = mul2(bc2(-2.0f), sub2(t1, t2));
    float2 Cp = bc2(0.0f);
#pragma unroll
    for (int m = 0; m < K; ++m) {
        const float2 D4 = *(p += s);
        const float2 t0 = sub2(D4, D3);
        const float2 A0 = fma2(mul2(k, t0), t0, Geps);
        const float2 s0 = fma2(bc2(-3.0f), D3, D4), s1 = add2(D2, D3), s2 = fma2(bc2(-3.0f), D2, D1);
        float2 g0 = fma2(s0, s0, A0), g1 = fma2(s1, s1, A1), g2 = fma2(s2, s2, A2);
        g0 = mul2(g0, g0);
        g1 = mul2(g1, g1);
        g2 = mul2(g2, g2);
        const float2 w0 = mul2(g1, g2), w1 = mul2(g0, g2), w2 = mul2(g0, g1);
        const float2 sw = fma2(bc2(3.0f), w0, fma2(bc2(6.0f), w1, w2));
        const float2 e0 = sub2(t1, t0);
        const float2 num = fma2(w0, mul2(bc2(3.0f), e0), mul2(w2, h));
        const float2 F = fma2(bc2(2.0f), D3, D2);
        const float2 C = fma2(num, make_float2(fast_rcp(sw.x), fast_rcp(sw.y)), F);
        if (m > 0) {
            *out = fma2(six, D2, FWD ? sub2(C, Cp) : sub2(Cp, C));
            out += os;
        }
        Cp = C;
        h = add2(e0, e0);
        D1 = D2;
        D2 = D3;
        D3 = D4;
        t2 = t1;
        t1 = t0;
        A2 = A1;
        A1 = A0;
    }
}

// ----------------------------------------------------------- point fluxes

// Plain FP64 Euler flux in direction DIR (Sec. 2.1) and its LF split
// f(+/-) = (F +/- alpha U) / 2 (Sec. 2.2).
// TWICE: return 2 f(+/-) = F +/- alpha U (one FMA each, no halving); the
// caller then reconstructs with 4 eps, which gives exactly twice the WENO5
// value of f(+/-) (scaling by 2 commutes with every rounding), and halves once.
template <int D, int DIR, bool TWICE = false>
__device__ __forceinline__ void split_flux_f64(const double *q, double alpha, double gm1, double *fp, double *fm)
{
    constexpr int NF = D + 2;
    const double rho = q[0];
    const double ir = 1.0 / rho;
    double u[D];
    double ke = 0.0;
#pragma unroll
    for (int e = 0; e < D; ++e) {
        u[e] = q[1 + e] * ir;
        ke += u[e] * u[e];
    }
    const double p = gm1 * (q[D + 1] - 0.5 * rho * ke);
    double F[NF];
    F[0] = q[1 + DIR];
#pragma unroll
    for (int e = 0; e < D; ++e) F[1 + e] = q[1 + e] * u[DIR] + (e == DIR ? p : 0.0);
    F[D + 1] = u[DIR] * (q[D + 1] + p);
#pragma unroll
    for (int f = 0; f < NF; ++f) {
        if (TWICE) {
            fp[f] = fma(alpha, q[f], F[f]);
            fm[f] = fma(-alpha, q[f], F[f]);
        } else {
            fp[f] = 0.5 * (F[f] + alpha * q[f]);
            fm[f] = 0.5 * (F[f] - alpha * q[f]);
        }
    }
}

// Reference state of one tile line for the FP32-bulk path: the FP64 state
// split into hi + lo, and FP32 primitives that only ever multiply differences.
template <int D> struct RefState {
    float hi[D + 2], lo[D + 2];
    float rho, m[D], u[D], H;  // H = rho E + p
};

// The same from a state already split into FP32 hi + lo (lo may carry a stage
// increment, far above FP32 rounding, so the primitives take hi + lo).
template <int D>
__device__ __forceinline__ void make_ref_hl(const float *h, const float *l, float gm1, RefState<D> &r)
{
    float q[D + 2];
#pragma unroll
    for (int f = 0; f < D + 2; ++f) {
        r.hi[f] = h[f];
        r.lo[f] = l[f];
        q[f] = h[f] + l[f];
    }
    r.rho = q[0];
    const float ir = 1.0f / r.rho;
    float ke = 0.0f;
#pragma unroll
    for (int e = 0; e < D; ++e) {
        r.m[e] = q[1 + e];
        r.u[e] = r.m[e] * ir;
        ke += r.m[e] * r.u[e];
    }
    const float p = gm1 * (q[D + 1] - 0.5f * ke);
    r.H = q[D + 1] + p;
}

template <int D>
__device__ __forceinline__ void make_ref(const double *q, float gm1, RefState<D> &r)
{
#pragma unroll
    for (int f = 0; f < D + 2; ++f) split_f64(q[f], r.hi[f], r.lo[f]);
    r.rho = r.hi[0];
    const float ir = 1.0f / r.rho;
    float ke = 0.0f;
#pragma unroll
    for (int e = 0; e < D; ++e) {
        r.m[e] = r.hi[1 + e];
        r.u[e] = r.m[e] * ir;
        ke += r.m[e] * r.u[e];
    }
    const float p = gm1 * (r.hi[D + 1] - 0.5f * ke);
    r.H = r.hi[D + 1] + p;
}

// dq = q - ref, formed from the hi/lo splits so that it carries the full FP32
// relative precision of the difference (not of q).
template <int D>
__device__ __forceinline__ void diff_from_ref(const double *q, const RefState<D> &r, float *dq)
{
#pragma unroll
    for (int f = 0; f < D + 2; ++f) {
        float hi, lo;
        split_f64(q[f], hi, lo);
        dq[f] = (hi - r.hi[f]) + (lo - r.lo[f]);
    }
}

// Split-flux differences df(+/-) = f(+/-)(ref + dq) - f(+/-)(ref) in FP32,
// using only exact product-difference identities
//   d(ab) = da * b + a_ref * db,  du = (dm - u_ref drho) / rho,
// so every rounding error is relative to the differences, not to the state.
template <int D, int DIR, bool TWICE = false>
__device__ __forceinline__ void split_flux_diff(const float *dq, const RefState<D> &r, float alpha, float gm1,
                                                float *fp, float *fm)
{
    constexpr int NF = D + 2;
    const float rho = r.rho + dq[0];
    const float ir = fast_rcp(rho);
    float du[D], u[D];
    float dk = 0.0f;
#pragma unroll
    for (int e = 0; e < D; ++e) {
        du[e] = (dq[1 + e] - r.u[e] * dq[0]) * ir;
        u[e] = r.u[e] + du[e];
        dk += dq[1 + e] * u[e] + r.m[e] * du[e];
    }
    const float dp = gm1 * (dq[D + 1] - 0.5f * dk);
    float dF[NF];
    dF[0] = dq[1 + DIR];
#pragma unroll
    for (int e = 0; e < D; ++e) dF[1 + e] = dq[1 + e] * u[DIR] + r.m[e] * du[DIR] + (e == DIR ? dp : 0.0f);
    const float dH = dq[D + 1] + dp;
    dF[D + 1] = du[DIR] * (r.H + dH) + r.u[DIR] * dH;
#pragma unroll
    for (int f = 0; f < NF; ++f) {
        if (TWICE) {  // 2 f(+/-), see split_flux_f64
            fp[f] = fmaf(alpha, dq[f], dF[f]);
            fm[f] = fmaf(-alpha, dq[f], dF[f]);
        } else {
            fp[f] = 0.5f * (dF[f] + alpha * dq[f]);
            fm[f] = 0.5f * (dF[f] - alpha * dq[f]);
        }
    }
}

// ------------------------------------------------------------- wavespeed

// |u| + sqrt(gamma p / rho) in FP64 with the operation order of the plain
// formula (no contraction), so that alpha and dt reproduce it bit for bit.
template <int D>
__device__ __forceinline__ double wavespeed_f64(const double *q, double gamma, bool &bad)
{
    const double rho = q[0];
    double u2 = 0.0;
#pragma unroll
    for (int e = 0; e < D; ++e) {
        const double ue = __ddiv_rn(q[1 + e], rho);
        u2 = __dadd_rn(u2, __dmul_rn(ue, ue));
    }
    const double p = __dmul_rn(gamma - 1.0, __dsub_rn(q[D + 1], __dmul_rn(__dmul_rn(0.5, rho), u2)));
    bad = !(rho > 0.0) || !(p > 0.0) || !isfinite(u2) || !isfinite(q[D + 1]);
    const double a = __dsqrt_rn(__ddiv_rn(__dmul_rn(gamma, p), rho));
    return bad ? 0.0 : __dadd_rn(__dsqrt_rn(u2), a);
}

// Per-direction speeds |u_d| + a (FP64, same operation order as the plain formula).
template <int D>
__device__ __forceinline__ void dirspeeds_f64(const double *q, double gamma, double *sd)
{
    const double rho = q[0];
    double u2 = 0.0;
#pragma unroll
    for (int e = 0; e < D; ++e) {
        const double ue = __ddiv_rn(q[1 + e], rho);
        u2 = __dadd_rn(u2, __dmul_rn(ue, ue));
    }
    const double p = __dmul_rn(gamma - 1.0, __dsub_rn(q[D + 1], __dmul_rn(__dmul_rn(0.5, rho), u2)));
    const double a = __dsqrt_rn(__ddiv_rn(__dmul_rn(gamma, p), rho));
#pragma unroll
    for (int e = 0; e < D; ++e) sd[e] = __dadd_rn(fabs(__ddiv_rn(q[1 + e], rho)), a);
}

template <int D>
__device__ __forceinline__ void dirspeeds_f32(const float *q, float gamma, float *sd)
{
    const float rho = q[0];
    const float ir = 1.0f / rho;
    float u2 = 0.0f;
#pragma unroll
    for (int e = 0; e < D; ++e) {
        const float ue = q[1 + e] * ir;
        u2 += ue * ue;
    }
    const float p = (gamma - 1.0f) * (q[D + 1] - 0.5f * rho * u2);
    const float a = sqrtf(gamma * p * ir);
#pragma unroll
    for (int e = 0; e < D; ++e) sd[e] = fabsf(q[1 + e] * ir) + a;
}

// The FP32 wavespeed ||u|| + a feeds only the maximum behind alpha and dt,
// where a relative error of a few ulp is immaterial, so it takes the
// approximate reciprocal and square roots (one MUFU instruction each).
__device__ __forceinline__ float sqrt_approx(float x)
{
    float y;
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

template <int D>
__device__ __forceinline__ float wavespeed_f32(const float *q, float gamma, bool &bad)
{
    const float rho = q[0];
    const float ir = fast_rcp(rho);
    float u2 = 0.0f;
#pragma unroll
    for (int e = 0; e < D; ++e) {
        const float ue = q[1 + e] * ir;
        u2 += ue * ue;
    }
    const float p = (gamma - 1.0f) * (q[D + 1] - 0.5f * rho * u2);
    bad = !(rho > 0.0f) || !(p > 0.0f) || !isfinite(u2) || !isfinite(q[D + 1]);
    return bad ? 0.0f : sqrt_approx(u2) + sqrt_approx(gamma * p * ir);
}

// FP32 variant for the FP32-bulk kernels: the max runs on the bit patterns of
// the non-negative floats with the single-instruction warp reduction, and only
// the block's result is widened to FP64 (on the integer pipe).
__device__ __forceinline__ void block_max_publish_f32(float v, bool bad, unsigned long long *slot, int *status)
{
    __shared__ unsigned warp_max[32];
    __shared__ int any_bad;
    if (threadIdx.x == 0) any_bad = 0;
    const unsigned m = __reduce_max_sync(0xFFFFFFFFu, __float_as_uint(v));
    __syncthreads();
    if (bad) any_bad = 1;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) warp_max[wid] = m;
    __syncthreads();
    if (wid == 0) {
        const int nw = (blockDim.x + 31) >> 5;
        const unsigned mm = __reduce_max_sync(0xFFFFFFFFu, lane < nw ? warp_max[lane] : 0u);
        if (lane == 0) {
            if (mm > 0u) atomicMax(slot, (unsigned long long)__double_as_longlong(f32_to_f64(__uint_as_float(mm))));
            if (any_bad) atomicOr(status, ST_NONPHYSICAL);
        }
    }
}

// The same with one barrier: K values, each reduced per warp with the
// single-instruction reduction and combined with a shared-memory atomicMax
// into s_max[K] (with the non-physical flag into *s_bad); the caller zeroes
// s_max and *s_bad before a barrier that precedes this call.  Value 0 goes to
// *slot0, value k > 0 to slot_dir[k - 1].  Every thread of the block must call it.
template <int K>
__device__ __forceinline__ void block_max_publish_f32_1b(const float *v, bool bad, unsigned *s_max, int *s_bad,
                                                         unsigned long long *slot0, unsigned long long *slot_dir,
                                                         int *status)
{
#pragma unroll
    for (int k = 0; k < K; ++k) {
        const unsigned m = __reduce_max_sync(0xFFFFFFFFu, __float_as_uint(v[k]));
        if ((threadIdx.x & 31) == 0 && m > 0u) atomicMax(s_max + k, m);
    }
    if (bad) *s_bad = 1;
    __syncthreads();
    if (threadIdx.x < K) {
        const unsigned mm = s_max[threadIdx.x];
        unsigned long long *sl = threadIdx.x == 0 ? slot0 : slot_dir + (threadIdx.x - 1);
        if (mm > 0u) atomicMax(sl, (unsigned long long)__double_as_longlong(f32_to_f64(__uint_as_float(mm))));
    }
    if (threadIdx.x == 0 && *s_bad) atomicOr(status, ST_NONPHYSICAL);
}

// Block-wide max of a non-negative value, then one atomicMax per block on the
// 64-bit pattern of the double.  Also ORs the block's non-physical flag into
// the status word.  Every thread of the block must call it.
__device__ __forceinline__ void block_max_publish(double v, bool bad, unsigned long long *slot, int *status)
{
    __shared__ double warp_max[32];
    __shared__ int any_bad;
    if (threadIdx.x == 0) any_bad = 0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xFFFFFFFFu, v, o));
    __syncthreads();
    if (bad) any_bad = 1;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) warp_max[wid] = v;
    __syncthreads();
    if (wid == 0) {
        const int nw = (blockDim.x + 31) >> 5;
        double m = lane < nw ? warp_max[lane] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xFFFFFFFFu, m, o));
        if (lane == 0) {
            if (m > 0.0) atomicMax(slot, (unsigned long long)__double_as_longlong(m));
            if (any_bad) atomicOr(status, ST_NONPHYSICAL);
        }
    }
}

}  // namespace wg
