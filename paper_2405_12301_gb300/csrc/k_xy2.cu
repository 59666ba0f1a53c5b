// k_xy2.cu -- the 2D FP32-bulk residual and SSP-RK3 stage kernel, in
// pair-difference form.
//
// WENO5-JS (Sec. 2.2) depends on a stencil only through the first differences
// of its values and its centre value, and the flux difference of a cell
// (Eq. 1d-scalar-h-pde-fd) only through differences of interface fluxes.  With
// F^_{j} = f(+)_{j-1} + c(+)_j + f(-)_j + c(-)_j (c the WENO correction to the
// upwind centre value), the x part of a cell's residual is
//   F^_{i+1} - F^_{i} = [f(+)_i - f(+)_{i-1}] + [f(-)_{i+1} - f(-)_i]
//                       + [c(+)_{i+1} - c(+)_i] + [c(-)_{i+1} - c(-)_i],
// so everything is built from the split-flux differences of neighbouring
// points, D(a, b) = f(U_b) - f(U_a) (stored scaled for weno5d_slide2, see
// pair_diff2).  Each D is formed in FP32 from the two points' FP64 states
// alone: dU = U_b - U_a from their hi/lo splits, then the exact
// product-difference identities with a's FP32 primitives (d(xy) = dx y_b +
// x_a dy, du = (dm - u_a drho) / rho_b), so it carries the FP32 relative
// precision of the difference itself.  Consequences:
//   * a face on a tile edge is formed by both CTAs that touch it from bitwise
//     the same differences by the same operations, so it is the same number in
//     both (no per-tile reference), and the periodic sums move only by the FP32
//     rounding of the per-cell terms, which scales with neighbour differences;
//   * the rounding of every WENO input scales with the difference of two
//     neighbours, not with the variation across a tile.
//
// Stage state layout (this kernel): the hi parts of a cell's four fields as one
// float4 in plane H = hl[0 .. N), their lo parts in plane L = hl[N .. 2N), and
// Delta as float [cell][4] (one float4), so a point is three loads and its lo
// part plus Delta two packed adds.  (The 3D kernels keep the same stage state
// field by field, [f][cell].)
//
// Stage state (Eq. tt-ssprk3 without rounding, written on increments): with
// U^(k) = U^n + Delta_k, Delta_1 = dt L(U^n), Delta_2 = (Delta_1 + dt L(U^1)) / 4,
// Delta_3 = 2 (Delta_2 + dt L(U^2)) / 3 and U^{n+1} = U^n + Delta_3.  Stage 1
// splits U^n into FP32 hi/lo once and stores the split (hl) with Delta_1;
// stages 2 and 3 read hl and Delta_{k-1} (FP32) instead of an FP64 state, so
// no FP64 -> FP32 split is repeated, and only stage 3 touches FP64 arithmetic
// (U^n + Delta_3, one DADD per field).
//
// A CTA of 256 threads owns a 32 x 8 tile, one cell per thread, plus the
// plus-shaped halo of three ghost layers per side (Sec. 4.5).  Phases:
//   A. every point of the tile and halo is loaded once (boundary rule on ghost
//      indices) as FP32 hi/lo into shared memory;
//   F. every neighbour pair is differenced once: each thread its own point's
//      right (x) and upper (y) pair as one f32x2 computation (x pair in lane
//      x, y pair in lane y), and one halo pair;
//   W. WENO corrections of every face as sliding runs over the differences
//      (weno5d_slide2), WENO(+) forward and the mirrored WENO(-) backward;
//   C. the cell's residual from its two pairs and four face corrections per
//      direction, then L(U) or the stage update and the block's wavespeed max.
#include "weno_dev.cuh"
#include "weno_internal.h"

namespace wg {

namespace xy2 {
constexpr int NT = 256;
constexpr int TX = 32, TY = 8;
constexpr int NOWN = TX * TY;                 // 256 own points
constexpr int YH0 = NOWN;                     // y-halo slots: [6][col] (rows -3..-1, TY..TY+2)
constexpr int XH0 = YH0 + 6 * TX;             // x-halo slots: [6][row] (cols -3..-1, TX..TX+2)
constexpr int NPT = XH0 + 6 * TY;             // 496 points; halo point k (thread k) in slot YH0 + k
constexpr int NHY = 6 * TX, NHALO = NHY + 6 * TY;  // 192 y-halo + 48 x-halo points
constexpr int PX = TX + 5;                    // x pairs per row: a = col -3..TX+1
constexpr int PXP = PX + 2;                   // their row pitch in float2 (odd: conflict-free runs)
constexpr int PY = TY + 5;                    // y pairs per column: a = row -3..TY+1
constexpr int NDX = PXP * TY;                 // one [sign][component pair] block of x differences
constexpr int NDY = PY * TX;                  // one block of y differences
constexpr int NC = TX * TY;                   // cells per block of y-run outputs
constexpr int CXP = TX + 1;                   // row pitch of the x-run outputs (float2): the
                                              // 8 rows of a warp's x runs then hit distinct banks
constexpr int NCX = CXP * TY;                 // cells per block of x-run outputs
// shared memory: differences, then the points (phases A-F) or the runs'
// per-cell outputs (W-C)
constexpr size_t DX_OFF = 0;
constexpr size_t DY_OFF = DX_OFF + sizeof(float2) * 4 * NDX;
constexpr size_t R_OFF = DY_OFF + sizeof(float2) * 4 * NDY;
constexpr size_t PTS_BYTES = sizeof(float4) * 2 * NPT;
constexpr size_t CELL_BYTES = sizeof(float2) * 4 * (NC + NCX);
constexpr size_t BYTES = R_OFF + (PTS_BYTES > CELL_BYTES ? PTS_BYTES : CELL_BYTES);

static_assert(TX == 32 && TY == 8, "the halo decode takes lane bits for TX and TY");
__device__ __forceinline__ int own_slot(int lx, int ly) { return ly * TX + lx; }
__device__ __forceinline__ int xh_slot(int lx, int ly) { return XH0 + (lx < 0 ? lx + 3 : lx - TX + 3) * TY + ly; }
__device__ __forceinline__ int yh_slot(int lx, int ly) { return YH0 + (ly < 0 ? ly + 3 : ly - TY + 3) * TX + lx; }
}  // namespace xy2

// FP32 primitives of a point (state hi + lo) that only ever multiply
// differences.  They must describe the point's current state to FP32 relative
// precision: in stages 2 and 3 the lo part carries Delta_k, which is far larger
// than FP32 rounding, so hi alone (U^n) would not do.
struct Prim2 {
    float rho, u, v, H, mx, my;
};

__device__ __forceinline__ float2 lo2(const float4 q) { return make_float2(q.x, q.y); }
__device__ __forceinline__ float2 hi2(const float4 q) { return make_float2(q.z, q.w); }
__device__ __forceinline__ float4 cat4(const float2 a, const float2 b) { return make_float4(a.x, a.y, b.x, b.y); }

__device__ __forceinline__ Prim2 prim2(const float4 h, const float4 l, float gm1)
{
    Prim2 P;
    const float2 q01 = add2(lo2(h), lo2(l)), q23 = add2(hi2(h), hi2(l));
    P.rho = q01.x;
    P.mx = q01.y;
    P.my = q23.x;
    const float E = q23.y;
    const float ir = fast_rcp(P.rho);
    P.u = __fmul_rn(P.mx, ir);
    P.v = __fmul_rn(P.my, ir);
    const float k = __fmaf_rn(P.my, P.v, __fmul_rn(P.mx, P.u));
    const float p = __fmul_rn(gm1, __fmaf_rn(-0.5f, k, E));
    P.H = __fadd_rn(E, p);
    return P;
}

// Split-flux differences of one pair (a, b) along direction DIR (0: x, 1: y),
// stored scaled by the exact factor 1/4 for the WENO runs: dp = (f(+)(U_b) -
// f(+)(U_a)) / 4 and dm = -(f(-)(U_b) - f(-)(U_a)) / 4 (the mirrored WENO(-)
// runs read the negated differences), formed as (F +/- alpha U) differences
// times 1/8, as component pairs (rho, m_x) and (m_y, E).  The hi/lo differences are taken
// on those same pairs; the identities between them are scalar.  Every pair is
// formed by this one function, so a pair shared by two CTAs (a tile edge) gets
// bitwise the same differences in both.
template <int DIR>
__device__ __forceinline__ void pair_diff1(const float4 ha, const float4 la, const Prim2 &A, const float4 hb,
                                           const float4 lb, float al, float gm1, float2 *dp_out, float2 *dm_out)
{
    const float2 d01 = add2(sub2(make_float2(hb.x, hb.y), make_float2(ha.x, ha.y)),
                            sub2(make_float2(lb.x, lb.y), make_float2(la.x, la.y)));
    const float2 d23 = add2(sub2(make_float2(hb.z, hb.w), make_float2(ha.z, ha.w)),
                            sub2(make_float2(lb.z, lb.w), make_float2(la.z, la.w)));
    const float dR = d01.x, dE = d23.y;
    const float dMn = DIR == 0 ? d01.y : d23.x, dMt = DIR == 0 ? d23.x : d01.y;
    const float una = DIR == 0 ? A.u : A.v, uta = DIR == 0 ? A.v : A.u;
    const float mna = DIR == 0 ? A.mx : A.my, mta = DIR == 0 ? A.my : A.mx;
    const float irb = fast_rcp(__fadd_rn(A.rho, dR));
    const float dun = __fmul_rn(__fmaf_rn(-una, dR, dMn), irb);  // du_n = (dm_n - u_n,a drho) / rho_b
    const float dut = __fmul_rn(__fmaf_rn(-uta, dR, dMt), irb);
    const float unb = __fadd_rn(una, dun), utb = __fadd_rn(uta, dut);
    const float kn = __fmaf_rn(mna, dun, __fmul_rn(dMn, unb));          // d(m_n u_n)
    const float dk = __fmaf_rn(mta, dut, __fmaf_rn(dMt, utb, kn));      // d(m . u)
    const float dp = __fmul_rn(gm1, __fmaf_rn(-0.5f, dk, dE));
    const float dH = __fadd_rn(dE, dp);
    const float Fn = __fadd_rn(kn, dp);
    const float Ft = __fmaf_rn(mta, dun, __fmul_rn(dMt, unb));
    const float FE = __fmaf_rn(una, dH, __fmul_rn(dun, __fadd_rn(A.H, dH)));
    // the fluxes in the component order (rho, m_x, m_y, E); (F + alpha dU) and
    // -(F - alpha dU), times the exact 1/8 (a power of two: an inexact scale such
    // as fl(1/6) would multiply every residual by the same 1 + 3e-8, a
    // systematic error that grows with the number of steps)
    const float2 F01 = make_float2(dMn, DIR == 0 ? Fn : Ft);
    const float2 F23 = make_float2(DIR == 0 ? Ft : Fn, FE);
    const float2 a2 = bc2(al), eighth = bc2(0.125f);
    dp_out[0] = mul2(eighth, fma2(a2, d01, F01));
    dp_out[1] = mul2(eighth, fma2(a2, d23, F23));
    dm_out[0] = mul2(eighth, fma2(a2, d01, make_float2(-F01.x, -F01.y)));
    dm_out[1] = mul2(eighth, fma2(a2, d23, make_float2(-F23.x, -F23.y)));
}

// A point's FP32 hi/lo state in a tile that touches the boundary: the
// boundary rule on the ghost indices (Sec. 4.5).  Kept out of line, so the
// interior tiles' straight loads are not interleaved with this code.
struct PointHL {
    float4 h, l;
};

__device__ __noinline__ PointHL load_point_bc(const double *U, const float4 *hl, const float *din, long long N,
                                              int nx, int ny, int bx0, int bx1, int by0, int by1,
                                              const double *bcs, bool from_hl, int cx, int cy)
{
    PointHL p;
    bool fx_ = false, fy_ = false;
    int inx, iny;
    cx = cx < nx + 2 ? cx : nx + 2;
    cy = cy < ny + 2 ? cy : ny + 2;
    cx = ghost_map(cx, nx, bx0, bx1, fx_, inx);
    cy = ghost_map(cy, ny, by0, by1, fy_, iny);
    if (inx >= 0 || iny >= 0) {  // a ghost of an inflow side holds the given state
        const double *st = bcs + (inx >= 0 ? inx * 5 : (2 + iny) * 5);
        split_f64(st[0], p.h.x, p.l.x);
        split_f64(st[1], p.h.y, p.l.y);
        split_f64(st[2], p.h.z, p.l.z);
        split_f64(st[3], p.h.w, p.l.w);
        return p;
    }
    const long long src = (long long)cy * nx + cx;
    if (from_hl) {
        const float4 l = hl[N + src], d = reinterpret_cast<const float4 *>(din)[src];
        p.h = hl[src];
        p.l = cat4(add2(lo2(l), lo2(d)), add2(hi2(l), hi2(d)));
    } else {
        split_f64(U[src], p.h.x, p.l.x);
        split_f64(U[N + src], p.h.y, p.l.y);
        split_f64(U[2 * N + src], p.h.z, p.l.z);
        split_f64(U[3 * N + src], p.h.w, p.l.w);
    }
    if (fx_) { p.h.y = -p.h.y; p.l.y = -p.l.y; }
    if (fy_) { p.h.z = -p.h.z; p.l.z = -p.l.z; }
    return p;
}

// ST: the stage (0, 1, 2) of EPI_STAGE; EPI_RHS reads U like stage 0.
template <int EPI, bool PD, int ST>
__global__ void __launch_bounds__(xy2::NT, 5) k_xy2(const SweepArgs a)
{
    using namespace xy2;
    constexpr int NF = 4;
    extern __shared__ __align__(16) unsigned char smem[];
    float2 *Dx = reinterpret_cast<float2 *>(smem + DX_OFF);   // [sign][pair][TY][PXP]
    float2 *Dy = reinterpret_cast<float2 *>(smem + DY_OFF);   // [sign][pair][PY][TX]
    float4 *Ph = reinterpret_cast<float4 *>(smem + R_OFF);    // [NPT] hi parts (phases A-F)
    float4 *Pl = Ph + NPT;                                    // [NPT] lo parts
    float2 *Px = reinterpret_cast<float2 *>(smem + R_OFF);    // [sign][pair][TY][CXP] (phases W-C)
    float2 *Py = Px + 4 * NCX;                                // [sign][pair][TY][TX]

    const long long dtbits = __double_as_longlong(a.ctl->dt);
    if (a.check_dt && dtbits == 0) return;
    // b_k dt comes from the control block (set with dt, an FP32 pair hi + lo) and
    // the residual factors -(2/3) / h_d from the host (SweepArgs::ih23): phase C's
    // sums are 3/2 times the flux differences (the differences are stored as 1/4
    // of themselves, and the runs return 6/4 of the corrections), and a single
    // rounded factor would bias every residual the same way
    __shared__ float2 s_al;  // the LF alpha of x and y in FP32 (converted once per block)
    __shared__ unsigned s_max[3];  // the block's wavespeed maxima (FP32 bit patterns)
    __shared__ int s_bad;
    if (threadIdx.x == 0) {
        s_max[0] = s_max[1] = s_max[2] = 0u;
        s_bad = 0;
        const double alpha = __longlong_as_double((long long)a.ctl->alpha[a.slot_in]);
        s_al = make_float2(f64_to_f32(PD ? __longlong_as_double((long long)a.ctl->alpha_dir[a.slot_in][0]) : alpha),
                           f64_to_f32(PD ? __longlong_as_double((long long)a.ctl->alpha_dir[a.slot_in][1]) : alpha));
    }

    const int nx = a.n[0], ny = a.n[1];
    const long long N = a.N;
    const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    const int gx = x0 + tx, gy = y0 + ty;
    const bool own = gx < nx && gy < ny;
    // 32-bit cell indices (the host keeps N below 2^32) on 64-bit plane pointers
    const unsigned cell = (unsigned)(gy < ny ? gy : ny - 1) * (unsigned)nx + (unsigned)(gx < nx ? gx : nx - 1);
    // stage 1 reads U^n as FP64; stages 2 and 3 read the stored split and Delta_{k-1}
    constexpr bool from_hl = EPI == EPI_STAGE && ST > 0;
    if (EPI == EPI_STAGE && ST == 2) {  // U^n at the own cell, for U^{n+1} = U^n + Delta_3
#pragma unroll
        for (int f = 0; f < NF; ++f) asm volatile("prefetch.global.L2 [%0];" ::"l"((a.U + f * N) + cell));
    }
    const bool interior = x0 >= 3 && y0 >= 3 && x0 + TX + 3 <= nx && y0 + TY + 3 <= ny;
    float4 *Hl = reinterpret_cast<float4 *>(a.hl);  // planes H and L of the stage state
    float4 *Ll = Hl + N;
    const float4 *Din = reinterpret_cast<const float4 *>(a.din);

    // ---- phase A: a point's FP32 hi/lo state, boundary rule on ghost indices
    auto load_point = [&](int lx, int ly, float4 &h, float4 &l) {
        if (!interior) {
            const PointHL p = load_point_bc(a.U, Hl, a.din, N, nx, ny, a.bc[0][0], a.bc[0][1], a.bc[1][0],
                                            a.bc[1][1], a.bcs, from_hl, x0 + lx, y0 + ly);
            h = p.h;
            l = p.l;
            return;
        }
        const unsigned src = (unsigned)(y0 + ly) * (unsigned)nx + (unsigned)(x0 + lx);
        if constexpr (from_hl) {
            const float4 lo = __ldg(Ll + src), d = __ldg(Din + src);
            h = __ldg(Hl + src);
            l = cat4(add2(lo2(lo), lo2(d)), add2(hi2(lo), hi2(d)));
        } else {
            const double *u = a.U;
            split_f64(__ldg(u + src), h.x, l.x);
            split_f64(__ldg((u += N) + src), h.y, l.y);
            split_f64(__ldg((u += N) + src), h.z, l.z);
            split_f64(__ldg((u += N) + src), h.w, l.w);
        }
    };

    // the own point and the halo point of this thread: both loads go out
    // before either is stored, so their latencies overlap
    const bool halo = threadIdx.x < NHALO;
    int hk = 0, hslot = 0, bslot = 0, hx = 0, hy = 0;
    bool hdirx = false;
    if (halo) {
        const int t = threadIdx.x;
        hslot = YH0 + t;
        if (t < NHY) {     // y halo: rows -3..-1 and TY..TY+2 of every tile column
            hx = t & 31;
            hk = t >> 5;
            hy = hk < 3 ? hk - 3 : TY + hk - 3;
            // its upper pair, except from the last row; row -1's upper point is own row 0
            bslot = hk == 2 ? own_slot(hx, 0) : hslot + TX;
        } else {           // x halo: columns -3..-1 and TX..TX+2 of every tile row
            const int u = t - NHY;
            hk = u >> 3;
            hy = u & 7;
            hx = hk < 3 ? hk - 3 : TX + hk - 3;
            hdirx = true;
            bslot = hk == 2 ? own_slot(0, hy) : hslot + TY;
        }
    }
    const bool hpair = halo && hk != 5;
    {
        float4 h, l, h2, l2;
        load_point(tx, ty, h, l);
        if (halo) load_point(hx, hy, h2, l2);
        if (EPI == EPI_STAGE && ST == 0 && own) {  // the split of U^n, read by stages 2 and 3
            Hl[cell] = h;
            Ll[cell] = l;
        }
        Ph[own_slot(tx, ty)] = h;
        Pl[own_slot(tx, ty)] = l;
        if (halo) {
            Ph[hslot] = h2;
            Pl[hslot] = l2;
        }
    }
    __syncthreads();

    // ---- phase F: neighbour-pair differences
    const float gm1 = a.gm1_f;
    const float alX = s_al.x, alY = s_al.y;
    {
        const int sa = own_slot(tx, ty);
        const int sbx = tx + 1 < TX ? own_slot(tx + 1, ty) : xh_slot(TX, ty);
        const int sby = ty + 1 < TY ? own_slot(tx, ty + 1) : yh_slot(tx, TY);
        const float4 ha = Ph[sa], la = Pl[sa];
        const Prim2 A = prim2(ha, la, gm1);
        float2 dp[2], dm[2];
        // x pair at index tx + 3 of row ty
        pair_diff1<0>(ha, la, A, Ph[sbx], Pl[sbx], alX, gm1, dp, dm);
        const int ix = ty * PXP + tx + 3;
        Dx[0 * NDX + ix] = dp[0];
        Dx[1 * NDX + ix] = dp[1];
        Dx[2 * NDX + ix] = dm[0];
        Dx[3 * NDX + ix] = dm[1];
        // y pair at index ty + 3 of column tx
        pair_diff1<1>(ha, la, A, Ph[sby], Pl[sby], alY, gm1, dp, dm);
        const int iy = (ty + 3) * TX + tx;
        Dy[0 * NDY + iy] = dp[0];
        Dy[1 * NDY + iy] = dp[1];
        Dy[2 * NDY + iy] = dm[0];
        Dy[3 * NDY + iy] = dm[1];
    }
    if (hpair) {
        const float4 ha = Ph[hslot], la = Pl[hslot], hb = Ph[bslot], lb = Pl[bslot];
        const Prim2 A = prim2(ha, la, gm1);
        float2 dp[2], dm[2];
        int o;
        float2 *Dd;
        int nd;
        if (hdirx) {
            pair_diff1<0>(ha, la, A, hb, lb, alX, gm1, dp, dm);
            o = hy * PXP + (hk < 3 ? hk : TX + hk);  // a col + 3
            Dd = Dx;
            nd = NDX;
        } else {
            pair_diff1<1>(ha, la, A, hb, lb, alY, gm1, dp, dm);
            o = (hk < 3 ? hk : TY + hk) * TX + hx;  // (a row + 3) * TX + col
            Dd = Dy;
            nd = NDY;
        }
        Dd[0 * nd + o] = dp[0];
        Dd[1 * nd + o] = dp[1];
        Dd[2 * nd + o] = dm[0];
        Dd[3 * nd + o] = dm[1];
    }
    __syncthreads();

    // the epilogue's own-cell inputs, loaded now so that phase W hides their
    // latency: Delta_k (stages 2, 3) and the hi part of U^n (its wavespeed)
    float4 dk = make_float4(0.0f, 0.0f, 0.0f, 0.0f), hn = dk;
    if (EPI == EPI_STAGE && own) {
        hn = Hl[cell];  // stage 1 wrote it in phase A (a plain, coherent load)
        if (ST > 0) dk = __ldg(Din + cell);
    }

    // ---- phase W: WENO corrections of every face (the points are dead now;
    // the runs' per-cell outputs take their place).  One run of TY + 1 = 9
    // faces per thread, pair w & 1, sign (w >> 1) & 1:
    //   warps 0-3, y: column `lane`, faces 0..8, cells 0..7;
    //   warps 4-7, x: row lane & 7, faces 8 s .. 8 s + 8, cells 8 s .. 8 s + 7
    //   for s = lane >> 3.
    // Face j's WENO(+) window takes the pairs a = j-3..j (indices j..j+3), its
    // mirrored WENO(-) window the pairs a = j+1..j-2 read backwards (indices
    // j+4..j+1).  Each run leaves a cell its pair's difference plus the change
    // of the correction across the cell (weno5d_cells2), both 6/4 of their
    // values; on differences scaled by 1/4 the smoothness indicators carry
    // 4 (1/4)^2 = 1/4 times beta, so Geps = eps / 4.
    {
        const float Geps = 0.25f * a.eps_f;
        const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, pr = w & 1, sg = (w >> 1) & 1;
        const int blk = sg * 2 + pr;
        // the strides are compile-time constants in each of the four calls, so
        // every load and store of a run takes an immediate offset
        if (w < 4) {
            const float2 *p = Dy + blk * NDY + lane;
            float2 *out = Py + blk * NC + lane;
            if (sg) weno5d_cells2<TY + 1, false>(p + 12 * TX, -TX, Geps, out + (TY - 1) * TX, -TX);
            else weno5d_cells2<TY + 1, true>(p, TX, Geps, out, TX);
        } else {
            const int ly = lane & 7, j0 = (lane >> 3) * 8;
            const float2 *p = Dx + blk * NDX + ly * PXP + j0;
            float2 *out = Px + blk * NCX + ly * CXP + j0;
            // WENO(-): differences j0+12 .. j0+1, cells j0+7 .. j0
            if (sg) weno5d_cells2<TY + 1, false>(p + 12, -1, Geps, out + (TY - 1), -1);
            else weno5d_cells2<TY + 1, true>(p, 1, Geps, out, 1);
        }
    }
    __syncthreads();

    // ---- phase C: -(F^_{i+1} - F^_i)/h_x - (G^_{j+1} - G^_j)/h_y: the sum of the
    // two runs' parts of the cell is 3/2 times each flux difference, removed by
    // the factor pairs s_ih
    float2 r[2];  // the residual, fields (rho, m_x) and (m_y, E)
    {
        const float2 ihx = a.ih23[0], ihy = a.ih23[1];
        const int c = ty * TX + tx, cx = ty * CXP + tx;
#pragma unroll
        for (int pr = 0; pr < 2; ++pr) {
            const float2 sx = add2(Px[pr * NCX + cx], Px[(2 + pr) * NCX + cx]);
            const float2 sy = add2(Py[pr * NC + c], Py[(2 + pr) * NC + c]);
            r[pr] = fma2(sy, bc2(ihy.x), fma2(sy, bc2(ihy.y), fma2(sx, bc2(ihx.x), mul2(sx, bc2(ihx.y)))));
        }
    }
    if (EPI == EPI_RHS) {
        if (own) {
            double *R = a.Rout;
            R[cell] = f32_to_f64(r[0].x);
            (R += N)[cell] = f32_to_f64(r[0].y);
            (R += N)[cell] = f32_to_f64(r[1].x);
            (R += N)[cell] = f32_to_f64(r[1].y);
        }
        return;
    }
    // EPI_STAGE: Delta_{k+1} = b_k (Delta_k + dt R); stage 3 ends the step
    float s = 0.0f, sd[2] = {0.0f, 0.0f};
    bool bad = false;
    if (own) {
        // Delta = b_k dt R + c_k Delta_k with b_k dt and c_k = 2/3 as hi + lo pairs
        // (c_k = 1/4 is exact), so the coefficients carry no systematic rounding
        const float2 bdt = a.ctl->bdt[ST];
        constexpr float c_hi = ST == 1 ? 0.25f : (float)(2.0 / 3.0);
        constexpr float c_lo = ST == 1 ? 0.0f : (float)(2.0 / 3.0 - (double)(float)(2.0 / 3.0));
        float2 dn[2], qq[2];
        const float2 dkp[2] = {lo2(dk), hi2(dk)}, hnp[2] = {lo2(hn), hi2(hn)};
#pragma unroll
        for (int pr = 0; pr < 2; ++pr) {  // field pairs, each lane rounded as the scalar form
            float2 t = mul2(bc2(bdt.y), r[pr]);
            if (ST > 0) t = fma2(bc2(c_hi), dkp[pr], fma2(bc2(c_lo), dkp[pr], t));
            dn[pr] = fma2(bc2(bdt.x), r[pr], t);
            qq[pr] = add2(hnp[pr], dn[pr]);  // the new state in FP32, for the wavespeed
        }
        if (ST == 2) {
            const float d4[NF] = {dn[0].x, dn[0].y, dn[1].x, dn[1].y};
#pragma unroll
            for (int f = 0; f < NF; ++f) (a.Uout + f * N)[cell] = __ldg((a.U + f * N) + cell) + f32_to_f64(d4[f]);
        }
        const float q[NF] = {qq[0].x, qq[0].y, qq[1].x, qq[1].y};
        if (ST < 2) reinterpret_cast<float4 *>(a.dout)[cell] = cat4(dn[0], dn[1]);
        s = wavespeed_f32<2>(q, a.gamma_f, bad);
        if (PD && !bad) dirspeeds_f32<2>(q, a.gamma_f, sd);
    }
    const float v[3] = {s, sd[0], sd[1]};
    block_max_publish_f32_1b<PD ? 3 : 1>(v, bad, s_max, &s_bad, &a.ctl->alpha[a.slot_out],
                                         &a.ctl->alpha_dir[a.slot_out][0], &a.ctl->status);
}

template <int EPI, bool PD, int ST>
static cudaError_t launch_xy2_t(const SweepArgs &a, cudaStream_t s)
{
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(k_xy2<EPI, PD, ST>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)xy2::BYTES);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    dim3 grid((unsigned)((a.n[0] + xy2::TX - 1) / xy2::TX), (unsigned)((a.n[1] + xy2::TY - 1) / xy2::TY), 1);
    k_xy2<EPI, PD, ST><<<grid, xy2::NT, xy2::BYTES, s>>>(a);
    return cudaGetLastError();
}

template <int EPI, bool PD>
static cudaError_t launch_xy2_s(const SweepArgs &a, cudaStream_t s)
{
    if (EPI == EPI_RHS || a.stage == 0) return launch_xy2_t<EPI, PD, 0>(a, s);
    if (a.stage == 1) return launch_xy2_t<EPI, PD, 1>(a, s);
    return launch_xy2_t<EPI, PD, 2>(a, s);
}

cudaError_t launch_xy2(int epi, const SweepArgs &a, cudaStream_t s)
{
    if (a.N >= (1ll << 32)) return cudaErrorInvalidValue;  // the kernel indexes cells in 32 bits
    if (epi == EPI_RHS) return a.per_dir ? launch_xy2_s<EPI_RHS, true>(a, s) : launch_xy2_s<EPI_RHS, false>(a, s);
    if (epi == EPI_STAGE) return a.per_dir ? launch_xy2_s<EPI_STAGE, true>(a, s) : launch_xy2_s<EPI_STAGE, false>(a, s);
    return cudaErrorInvalidValue;
}

}  // namespace wg
