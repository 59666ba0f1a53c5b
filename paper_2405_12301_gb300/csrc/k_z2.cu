// k_z2.cu -- the z direction of the 3D FP32-bulk residual, in pair-difference
// form, ending the stage (the x and y directions run in k_xy<3> and leave their
// part in the FP32 accumulator).
//
// As in k_xy2 (2D), WENO5-JS needs a stencil only through its first
// differences and its centre value, and a cell's flux difference only through
// differences of interface fluxes, so the z part of a cell's residual is built
// from the split-flux differences of neighbouring points along z,
// D(a, b) = f(U_b) - f(U_a), each formed in FP32 from the two points' hi/lo
// states by exact product-difference identities (pair_diff_z), then WENO
// corrections as sliding runs over those differences (weno5d_cells2).
//
// A CTA of 256 threads owns 32 x-cells x TZ = 8 z-cells of one y-row (z-tiles
// fastest in the grid, so tiles sharing halo planes run close together), one
// cell per thread, plus three ghost planes below and above (Sec. 4.5).
//   A. own points and the 192 halo points as FP32 hi/lo into shared memory
//      (stage 1 also stores the split of U^n, the stage state);
//   F. every z pair once: each thread its own point's upper pair, threads
//      0..159 one halo pair; the five components as the f32x2 pairs (rho, m_x),
//      (m_y, m_z) and E, whose differences are stored with the E of the
//      neighbouring column so that every run works on f32x2 pairs;
//   W. 160 runs of TZ + 1 = 9 windows: (rho, m_x) and (m_y, m_z) per column
//      and sign (warps 0-3), E per column pair and sign (warp 4), each run's
//      per-cell outputs written in place over differences it has read;
//   C. -(H^_{k+1} - H^_k)/h_z plus the accumulator's x+y part, then L(U) or the
//      stage update on increments (the stage state of k_xy2.cu), and the
//      block's wavespeed maximum.
// The accumulator and Delta_k of the own cells arrive by asynchronous copies
// into the shared memory of the (then dead) points, issued after phase F.
#include "bulk_load.cuh"
#include "weno_dev.cuh"
#include "weno_internal.h"

namespace wg {

namespace z2 {
constexpr int NT = 256;
constexpr int TX = 32, TZ = 8;
constexpr int NOWN = TX * TZ;                  // 256 own points: slot z * TX + x
constexpr int ZH0 = NOWN;                      // z-halo slots [6][TX] (z = -3..-1, TZ..TZ+2)
constexpr int NPT = ZH0 + 6 * TX;              // 448 points
constexpr int NHP = 5 * TX;                    // 160 halo pairs (a = z -3, -2, -1, TZ, TZ+1)
constexpr int PZ = TZ + 5;                     // z pairs per column: a = z -3..TZ+1
constexpr int NDZ = PZ * TX;                   // one [sign][component pair] block (float2)
constexpr int NDE = PZ * TX;                   // one [sign] block of E (float; columns 2c, 2c+1 a float2)
constexpr size_t DZ_OFF = 0;
constexpr size_t DE_OFF = DZ_OFF + sizeof(float2) * 4 * NDZ;
constexpr size_t P_OFF = DE_OFF + sizeof(float) * 2 * NDE;
constexpr size_t BYTES = P_OFF + (sizeof(float4) + sizeof(float)) * 2 * NPT;
static_assert(sizeof(float) * 2 * 5 * NT <= (sizeof(float4) + sizeof(float)) * 2 * NPT,
              "the epilogue operands fit in the points' shared memory");
__device__ __forceinline__ int own_slot(int lx, int lz) { return lz * TX + lx; }
}  // namespace z2

// FP32 primitives of a point (state hi + lo); they only multiply differences.
struct Prim3 {
    float rho, u, v, w, H, mx, my, mz;
};

__device__ __forceinline__ Prim3 prim3(const float4 h4, float h1, const float4 l4, float l1, float gm1)
{
    Prim3 P;
    const float2 q01 = add2(make_float2(h4.x, h4.y), make_float2(l4.x, l4.y));
    const float2 q23 = add2(make_float2(h4.z, h4.w), make_float2(l4.z, l4.w));
    P.rho = q01.x;
    P.mx = q01.y;
    P.my = q23.x;
    P.mz = q23.y;
    const float E = __fadd_rn(h1, l1);
    const float ir = fast_rcp(P.rho);
    P.u = __fmul_rn(P.mx, ir);
    P.v = __fmul_rn(P.my, ir);
    P.w = __fmul_rn(P.mz, ir);
    const float k = __fmaf_rn(P.mz, P.w, __fmaf_rn(P.my, P.v, __fmul_rn(P.mx, P.u)));
    const float p = __fmul_rn(gm1, __fmaf_rn(-0.5f, k, E));
    P.H = __fadd_rn(E, p);
    return P;
}

// Split-flux differences of one z pair (a, b), times the exact 1/8:
// dp = (F + alpha dU) / 8, dm = -(F - alpha dU) / 8 with F the z flux
// difference (Eq. physical-fluxes: normal momentum m_z), as the pairs
// (rho, m_x), (m_y, m_z) and the scalar E; the product-difference identities
// d(xy) = dx y_b + x_a dy and du = (dm - u_a drho) / rho_b, with a's primitives.
// Every pair is formed by this one function, so a pair on a tile edge has
// bitwise the same differences in both CTAs that form it.
__device__ __forceinline__ void pair_diff_z(const float4 ha4, float ha1, const float4 la4, float la1, const Prim3 &A,
                                            const float4 hb4, float hb1, const float4 lb4, float lb1, float al,
                                            float gm1, float2 *dp, float2 *dm, float &dpE, float &dmE)
{
    const float2 d01 = add2(sub2(make_float2(hb4.x, hb4.y), make_float2(ha4.x, ha4.y)),
                            sub2(make_float2(lb4.x, lb4.y), make_float2(la4.x, la4.y)));
    const float2 d23 = add2(sub2(make_float2(hb4.z, hb4.w), make_float2(ha4.z, ha4.w)),
                            sub2(make_float2(lb4.z, lb4.w), make_float2(la4.z, la4.w)));
    const float dE = __fadd_rn(__fsub_rn(hb1, ha1), __fsub_rn(lb1, la1));
    const float dR = d01.x, dMx = d01.y, dMy = d23.x, dMz = d23.y;
    const float irb = fast_rcp(__fadd_rn(A.rho, dR));
    const float dw = __fmul_rn(__fmaf_rn(-A.w, dR, dMz), irb);   // normal velocity
    const float du = __fmul_rn(__fmaf_rn(-A.u, dR, dMx), irb);
    const float dv = __fmul_rn(__fmaf_rn(-A.v, dR, dMy), irb);
    const float wb = __fadd_rn(A.w, dw), ub = __fadd_rn(A.u, du), vb = __fadd_rn(A.v, dv);
    const float kn = __fmaf_rn(A.mz, dw, __fmul_rn(dMz, wb));                          // d(m_z w)
    const float dk = __fmaf_rn(A.my, dv, __fmaf_rn(dMy, vb, __fmaf_rn(A.mx, du, __fmaf_rn(dMx, ub, kn))));
    const float dpr = __fmul_rn(gm1, __fmaf_rn(-0.5f, dk, dE));                        // d p
    const float dH = __fadd_rn(dE, dpr);
    const float Fz = __fadd_rn(kn, dpr);                                               // d(m_z w + p)
    const float Fx = __fmaf_rn(A.mx, dw, __fmul_rn(dMx, wb));                          // d(m_x w)
    const float Fy = __fmaf_rn(A.my, dw, __fmul_rn(dMy, wb));                          // d(m_y w)
    const float FE = __fmaf_rn(A.w, dH, __fmul_rn(dw, __fadd_rn(A.H, dH)));            // d(w H)
    const float2 F01 = make_float2(dMz, Fx), F23 = make_float2(Fy, Fz);
    const float2 a2 = bc2(al), eighth = bc2(0.125f);
    dp[0] = mul2(eighth, fma2(a2, d01, F01));
    dp[1] = mul2(eighth, fma2(a2, d23, F23));
    dm[0] = mul2(eighth, fma2(a2, d01, make_float2(-F01.x, -F01.y)));
    dm[1] = mul2(eighth, fma2(a2, d23, make_float2(-F23.x, -F23.y)));
    dpE = __fmul_rn(0.125f, __fmaf_rn(al, dE, FE));
    dmE = __fmul_rn(0.125f, __fmaf_rn(al, dE, -FE));
}

__device__ __forceinline__ void cp_async4z(void *dst, const void *src)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"((unsigned)__cvta_generic_to_shared(dst)), "l"(src)
                 : "memory");
}
__device__ __forceinline__ void cp_async16z(void *dst, const void *src)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"((unsigned)__cvta_generic_to_shared(dst)), "l"(src)
                 : "memory");
}

// ST: the stage (0, 1, 2) of EPI_STAGE; EPI_RHS reads U like stage 0.
template <int EPI, bool PD, int ST>
__global__ void __launch_bounds__(z2::NT, 5) k_z2(const SweepArgs a)
{
    using namespace z2;
    constexpr int NF = 5;
    extern __shared__ __align__(16) unsigned char smem[];
    float2 *Dz = reinterpret_cast<float2 *>(smem + DZ_OFF);  // [sign][pair][PZ][TX]
    float *De = reinterpret_cast<float *>(smem + DE_OFF);    // [sign][PZ][TX]
    float4 *Ph4 = reinterpret_cast<float4 *>(smem + P_OFF);  // [NPT] hi of (rho, m_x, m_y, m_z)
    float4 *Pl4 = Ph4 + NPT;                                 // [NPT] lo
    float *Ph1 = reinterpret_cast<float *>(Pl4 + NPT);       // [NPT] hi of E
    float *Pl1 = Ph1 + NPT;                                  // [NPT] lo of E
    float *e_acc = reinterpret_cast<float *>(smem + P_OFF);  // [NF][NT] after phase F: the x+y part
    float *e_din = e_acc + NF * NT;                          // [4][NT] float4 per thread, then [NT] E

    const long long dtbits = __double_as_longlong(a.ctl->dt);
    if (a.check_dt && dtbits == 0) return;
    __shared__ float s_al;  // the z LF alpha in FP32 (converted once per block)
    __shared__ unsigned s_max[4];
    __shared__ int s_bad;
    if (threadIdx.x == 0) {
        s_max[0] = s_max[1] = s_max[2] = s_max[3] = 0u;
        s_bad = 0;
        s_al = f64_to_f32(__longlong_as_double(
            (long long)(PD ? a.ctl->alpha_dir[a.slot_in][2] : a.ctl->alpha[a.slot_in])));
    }

    const int nx = a.n[0], nz = a.n[2];
    const long long N = a.N, sz = a.stride[2];
    const int x0 = blockIdx.y * TX, z0 = blockIdx.x * TZ;
    const long long yoff = (long long)blockIdx.z * a.stride[1];
    const int tx = threadIdx.x & 31, tz = threadIdx.x >> 5;
    const int gx = x0 + tx, gz = z0 + tz;
    const bool own = gx < nx && gz < nz;
    const long long cell = yoff + (long long)(gz < nz ? gz : nz - 1) * sz + (gx < nx ? gx : nx - 1);
    constexpr bool from_hl = EPI == EPI_STAGE && ST > 0;
    if (EPI == EPI_STAGE && ST == 2) {  // U^n at the own cell, for U^{n+1} = U^n + Delta_3
#pragma unroll
        for (int f = 0; f < NF; ++f) asm volatile("prefetch.global.L2 [%0];" ::"l"(a.U + f * N + cell));
    }
    const bool interior = z0 >= 3 && z0 + TZ + 3 <= nz && x0 + TX <= nx;

    // a point's FP32 hi/lo state, boundary rule on ghost z indices
    auto load_point = [&](int lx, int lz, float *h, float *l) {
        int cx = x0 + lx, cz = z0 + lz;
        bool fz_ = false;
        if (!interior) {
            int inz;
            cx = cx < nx ? cx : nx - 1;  // columns beyond the grid only feed cells that are not written
            cz = cz < nz + 2 ? cz : nz + 2;
            cz = ghost_map(cz, nz, a.bc[2][0], a.bc[2][1], fz_, inz);
            if (inz >= 0) {  // a ghost of an inflow side holds the given state
                bulk_state<NF>(a.bc_state[2][inz], h, l);
                return;
            }
        }
        bulk_point<NF, from_hl>(a, yoff + (long long)cz * sz + cx, h, l);
        if (fz_) { h[3] = -h[3]; l[3] = -l[3]; }
    };

    // ---- phase A
    const bool halo = threadIdx.x < 6 * TX;
    const int hk = threadIdx.x >> 5, hz = hk < 3 ? hk - 3 : TZ + hk - 3;
    {
        float h[NF], l[NF], h2[NF], l2[NF];
        load_point(tx, tz, h, l);
        if (halo) load_point(tx, hz, h2, l2);
        if (EPI == EPI_STAGE && ST == 0 && own) bulk_store_hl(a, cell, h, l);  // the split of U^n
        const int so = own_slot(tx, tz);
        Ph4[so] = make_float4(h[0], h[1], h[2], h[3]);
        Pl4[so] = make_float4(l[0], l[1], l[2], l[3]);
        Ph1[so] = h[4];
        Pl1[so] = l[4];
        if (halo) {
            const int sh = ZH0 + threadIdx.x;
            Ph4[sh] = make_float4(h2[0], h2[1], h2[2], h2[3]);
            Pl4[sh] = make_float4(l2[0], l2[1], l2[2], l2[3]);
            Ph1[sh] = h2[4];
            Pl1[sh] = l2[4];
        }
    }
    __syncthreads();

    // ---- phase F: z pairs (own upper pair at index tz + 3; halo pair)
    const float gm1 = a.gm1_f, al = s_al;
    auto do_pair = [&](int sa, int sb, int idx, int col) {
        const float4 ha4 = Ph4[sa], la4 = Pl4[sa];
        const float ha1 = Ph1[sa], la1 = Pl1[sa];
        const Prim3 A = prim3(ha4, ha1, la4, la1, gm1);
        float2 dp[2], dm[2];
        float dpE, dmE;
        pair_diff_z(ha4, ha1, la4, la1, A, Ph4[sb], Ph1[sb], Pl4[sb], Pl1[sb], al, gm1, dp, dm, dpE, dmE);
        const int o = idx * TX + col;
        Dz[0 * NDZ + o] = dp[0];
        Dz[1 * NDZ + o] = dp[1];
        Dz[2 * NDZ + o] = dm[0];
        Dz[3 * NDZ + o] = dm[1];
        De[0 * NDE + o] = dpE;
        De[1 * NDE + o] = dmE;
    };
    do_pair(own_slot(tx, tz), tz + 1 < TZ ? own_slot(tx, tz + 1) : ZH0 + 3 * TX + tx, tz + 3, tx);
    if (threadIdx.x < NHP) {
        const int sa = ZH0 + threadIdx.x;
        do_pair(sa, hk == 2 ? own_slot(tx, 0) : sa + TX, hk < 3 ? hk : TZ + hk, tx);
    }
    __syncthreads();

    // the epilogue's own-cell operands into the dead points' memory: the x+y
    // part of the residual and Delta_k, their latency hidden by phase W
    if (own) {
        const float *acc = reinterpret_cast<const float *>(a.acc);
#pragma unroll
        for (int f = 0; f < NF; ++f) cp_async4z(e_acc + f * NT + threadIdx.x, acc + f * N + cell);
        if (EPI == EPI_STAGE && ST > 0) {
            cp_async16z(reinterpret_cast<float4 *>(e_din) + threadIdx.x,
                        reinterpret_cast<const float4 *>(a.din) + (unsigned)cell);
            cp_async4z(e_din + 4 * NT + threadIdx.x, a.din1 + (unsigned)cell);
        }
    }
    asm volatile("cp.async.commit_group;" ::: "memory");

    // ---- phase W: warps 0-3 run (rho, m_x) / (m_y, m_z) of column `lane`,
    // pair w & 1, sign w >> 1; warp 4 runs E of column pair lane & 15, sign
    // lane >> 4 (a runtime stride: both signs share the warp).  Cell c's output
    // goes to index c + 4 (WENO(+)) or c + 1 (WENO(-)); Geps = eps / 4 on
    // differences scaled by 1/4 (as in k_xy2).
    {
        const float Geps = 0.25f * a.eps_f;
        const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
        if (w < 4) {
            const int sg = w >> 1;
            float2 *p = Dz + w * NDZ + lane;
            if (sg) weno5d_cells2<TZ + 1, false>(p + 12 * TX, -TX, Geps, p + TZ * TX, -TX);
            else weno5d_cells2<TZ + 1, true>(p, TX, Geps, p + 4 * TX, TX);
        } else if (w == 4) {
            const int sg = lane >> 4, cp = lane & 15, st = sg ? -(TX / 2) : TX / 2;
            float2 *p = reinterpret_cast<float2 *>(De + sg * NDE) + cp;
            if (sg) weno5d_cells2<TZ + 1, false>(p + 12 * (TX / 2), st, Geps, p + TZ * (TX / 2), st);
            else weno5d_cells2<TZ + 1, true>(p, st, Geps, p + 4 * (TX / 2), st);
        }
    }
    __syncthreads();

    // ---- phase C: the z part -(H^_{k+1} - H^_k)/h_z (run sums times the factor
    // pair -(2/3)/h_z, as in k_xy2) plus the accumulator's x+y part
    asm volatile("cp.async.wait_group 0;" ::: "memory");
    float r[NF];
    {
        const float2 ih = a.ih23[2];
        const int c = tz * TX + tx;
#pragma unroll
        for (int pr = 0; pr < 2; ++pr) {
            const float2 sz2 = add2(Dz[pr * NDZ + c + 4 * TX], Dz[(2 + pr) * NDZ + c + TX]);
            const float2 rz = fma2(sz2, bc2(ih.x), mul2(sz2, bc2(ih.y)));
            r[2 * pr] = rz.x;
            r[2 * pr + 1] = rz.y;
        }
        const float se = __fadd_rn(De[c + 4 * TX], De[NDE + c + TX]);
        r[4] = __fmaf_rn(se, ih.x, __fmul_rn(se, ih.y));
    }
    if (own) {
#pragma unroll
        for (int f = 0; f < NF; ++f) r[f] = __fadd_rn(e_acc[f * NT + threadIdx.x], r[f]);
    }
    if (EPI == EPI_RHS) {
        if (own) {
#pragma unroll
            for (int f = 0; f < NF; ++f) a.Rout[f * N + cell] = f32_to_f64(r[f]);
        }
        return;
    }
    // EPI_STAGE: Delta_{k+1} = b_k (Delta_k + dt R); stage 3 ends the step with U^n + Delta_3
    float s = 0.0f, sd[3] = {0.0f, 0.0f, 0.0f};
    bool bad = false;
    if (own) {
        const float2 bdt = a.ctl->bdt[ST];
        constexpr float c_hi = ST == 1 ? 0.25f : (float)(2.0 / 3.0);
        constexpr float c_lo = ST == 1 ? 0.0f : (float)(2.0 / 3.0 - (double)(float)(2.0 / 3.0));
        float hn[NF];  // the hi part of U^n (stage 1: from the own point, already in shared memory)
        {
            const float4 *H4 = reinterpret_cast<const float4 *>(a.hl);
            const float *H1 = reinterpret_cast<const float *>(H4 + 2 * N);
            const float4 q = H4[(unsigned)cell];  // (stage 1 wrote it in phase A: a plain, coherent load)
            hn[0] = q.x;
            hn[1] = q.y;
            hn[2] = q.z;
            hn[3] = q.w;
            hn[4] = H1[(unsigned)cell];
        }
        float qn[NF], dn[NF];
#pragma unroll
        for (int f = 0; f < NF; ++f) {
            float t = bdt.y * r[f];
            if (ST > 0) {
                const float dkf = f < 4 ? e_din[4 * threadIdx.x + f] : e_din[4 * NT + threadIdx.x];
                t = fmaf(c_hi, dkf, fmaf(c_lo, dkf, t));
            }
            dn[f] = fmaf(bdt.x, r[f], t);
            if (ST == 2) a.Uout[f * N + cell] = __ldg(a.U + f * N + cell) + f32_to_f64(dn[f]);
            qn[f] = hn[f] + dn[f];
        }
        if (ST < 2) {
            reinterpret_cast<float4 *>(a.dout)[(unsigned)cell] = make_float4(dn[0], dn[1], dn[2], dn[3]);
            a.dout1[(unsigned)cell] = dn[4];
        }
        s = wavespeed_f32<3>(qn, a.gamma_f, bad);
        if (PD && !bad) dirspeeds_f32<3>(qn, a.gamma_f, sd);
    }
    const float v[4] = {s, sd[0], sd[1], sd[2]};
    block_max_publish_f32_1b<PD ? 4 : 1>(v, bad, s_max, &s_bad, &a.ctl->alpha[a.slot_out],
                                         &a.ctl->alpha_dir[a.slot_out][0], &a.ctl->status);
}

template <int EPI, bool PD, int ST>
static cudaError_t launch_z2_t(const SweepArgs &a, cudaStream_t s)
{
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(k_z2<EPI, PD, ST>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)z2::BYTES);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    dim3 grid((unsigned)((a.n[2] + z2::TZ - 1) / z2::TZ), (unsigned)((a.n[0] + z2::TX - 1) / z2::TX),
              (unsigned)a.n[1]);
    k_z2<EPI, PD, ST><<<grid, z2::NT, z2::BYTES, s>>>(a);
    return cudaGetLastError();
}

template <int EPI, bool PD>
static cudaError_t launch_z2_s(const SweepArgs &a, cudaStream_t s)
{
    if (EPI == EPI_RHS || a.stage == 0) return launch_z2_t<EPI, PD, 0>(a, s);
    if (a.stage == 1) return launch_z2_t<EPI, PD, 1>(a, s);
    return launch_z2_t<EPI, PD, 2>(a, s);
}

cudaError_t launch_z2(int epi, const SweepArgs &a, cudaStream_t s)
{
    if (a.N >= (1ll << 32)) return cudaErrorInvalidValue;  // the stage state is indexed in 32 bits
    if (epi == EPI_RHS) return a.per_dir ? launch_z2_s<EPI_RHS, true>(a, s) : launch_z2_s<EPI_RHS, false>(a, s);
    if (epi == EPI_STAGE) return a.per_dir ? launch_z2_s<EPI_STAGE, true>(a, s) : launch_z2_s<EPI_STAGE, false>(a, s);
    return cudaErrorInvalidValue;
}

}  // namespace wg
