// k_xy.cu -- fused x+y residual kernel of the WENO5-JS scheme for 2D grids in
// FP64 and for each z-plane of 3D grids (FP64 and FP32-bulk).  The 2D
// FP32-bulk kernel is k_xy2 (k_xy2.cu).
//
// A CTA (256 threads) owns a TX x TY = 32 x 8 tile of one plane, one cell per
// thread, and the plus-shaped halo around it (three ghost layers per side in x
// and in y, Sec. 4.5).  Phases, all through shared memory:
//   A+F. every point of the tile and halo is loaded once (boundary rule applied
//      to ghost indices; FP32-bulk takes its difference from the tile's
//      reference state) and its LF split fluxes f(+/-) (Sec. 2.2) are formed in
//      the directions that need them: each thread its own point in x and y, and
//      one halo point in the halo's direction;
//   W. every x- and y-interface flux of the tile is reconstructed once, WENO(+)
//      plus mirrored WENO(-): in 2D as sliding runs along tile columns and row
//      segments; in 3D planes each thread its cell's left and bottom faces for
//      every component (FP32-bulk: a face's two windows as one f32x2 pair), and
//      the tile's last column/row faces spread over the threads;
//   C. each thread forms -(dF/dx) - (dG/dy) for its cell (Sec. 4.1) and either
//      stores it (3D: the z sweep adds its part and runs the stage), writes L(U),
//      or applies the SSP-RK3 stage combination (Eq. tt-ssprk3 without rounding)
//      and publishes the wavespeed max of the new state.
// Compared with one launch per direction, each point is loaded and split once
// per stage, and in 2D the residual never leaves the SM.
#include <type_traits>

#include "bulk_load.cuh"
#include "weno_dev.cuh"
#include "weno_internal.h"

namespace wg {

namespace xy {
constexpr int NT = 256;
constexpr int TX = 32, TY = 8;
constexpr int BX = TX + 6, BY = TY + 6;     // row and column extents with halo
constexpr int BXP = BX + 3;                 // row pitch of the x-flux points (41: the sliding
                                            // runs of phase W read 8 rows x 4 components per
                                            // warp without bank conflicts)
constexpr int NXP = BXP * TY;               // x-flux points: 38 (pitch 41) x 8
constexpr int NYP = TX * BY;                // y-flux points: 32 x 14
constexpr int NXI = (TX + 1) * TY;          // x interfaces: 33 x 8
constexpr int NYI = TX * (TY + 1);          // y interfaces: 32 x 9
constexpr int NHY = 6 * TX;                 // y-halo points (rows -3..-1, TY..TY+2)
constexpr int NHALO = NHY + 6 * TY;         // plus x-halo points: 240

// 2D grids reconstruct faces with sliding runs (one thread per line segment,
// component and sign; WENO(+) and WENO(-) kept apart); 3D planes (five
// components) one thread per cell.
template <int D> constexpr bool slide() { return D == 2; }

template <int D, bool BULK> struct Layout {
    using T = typename std::conditional<BULK, float, double>::type;
    static constexpr int NF = D + 2;
    static constexpr int NS = slide<D>() ? 2 : 1;                             // face-flux copies
    static constexpr size_t F_off = 0;                                        // Fx, Fy
    static constexpr size_t fx_off = (sizeof(T) * NS * NF * (NXI + NYI) + 15) & ~size_t(15);
    static constexpr size_t fy_off = fx_off + sizeof(T) * 2 * NF * NXP;
    static constexpr size_t ref_off = (fy_off + sizeof(T) * 2 * NF * NYP + 15) & ~size_t(15);
    static constexpr size_t bytes = ref_off + sizeof(RefState<D>);
};
}  // namespace xy

// The FP32-bulk (3D plane) kernel is held to 48 registers so that 5 CTAs (40
// warps) share an SM; its shared memory allows that many.  ST (FP32-bulk): the
// stage, which selects where the stencil state comes from -- the split of U
// (stage 1, L(U)) or the stored split of U^n plus Delta_k (stages 2 and 3, the
// stage state of k_xy2.cu).
template <int D, bool BULK, int EPI, bool PD, int ST = 0>
__global__ void __launch_bounds__(xy::NT, BULK ? 5 : 1) k_xy(const SweepArgs a)
{
    using namespace xy;
    using L = Layout<D, BULK>;
    static_assert(!BULK || (D == 3 && EPI == EPI_STORE), "2D FP32-bulk runs in k_xy2");
    using T = typename L::T;
    constexpr int NF = L::NF;
    extern __shared__ __align__(16) unsigned char smem[];
    T *Fx = reinterpret_cast<T *>(smem + L::F_off);        // [NS][NF][TY][TX+1]
    T *Fy = Fx + L::NS * NF * NXI;                         // [NS][NF][TY+1][TX]
    T *fx = reinterpret_cast<T *>(smem + L::fx_off);       // [2][NF][TY][BXP]
    T *fy = reinterpret_cast<T *>(smem + L::fy_off);       // [2][NF][BY][TX]
    RefState<D> &ref = *reinterpret_cast<RefState<D> *>(smem + L::ref_off);

    // dt and alpha come from the control block; the FP32 path converts them on
    // the integer pipe (a cvt issues at FP64 rate on this GPU)
    const long long dtbits = __double_as_longlong(a.ctl->dt);
    if (a.check_dt && dtbits == 0) return;
    const double dt = __longlong_as_double(dtbits);
    const double alpha = __longlong_as_double((long long)a.ctl->alpha[a.slot_in]);
    // LF constants of the x and y splittings: the global alpha, or per direction
    const double alx = PD ? __longlong_as_double((long long)a.ctl->alpha_dir[a.slot_in][0]) : alpha;
    const double aly = PD ? __longlong_as_double((long long)a.ctl->alpha_dir[a.slot_in][1]) : alpha;

    const int nx = a.n[0], ny = a.n[1];
    const long long N = a.N;
    const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
    const long long zoff = (long long)blockIdx.z * a.stride[2];
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    const int gx = x0 + tx, gy = y0 + ty;
    const bool own = gx < nx && gy < ny;
    const long long cell = zoff + (long long)(gy < ny ? gy : ny - 1) * nx + (gx < nx ? gx : nx - 1);

    // the stage combination needs U^n at this thread's cell: issue the loads now
    double un[NF];
    if (!BULK && EPI == EPI_STAGE && a.stage > 0) {
#pragma unroll
        for (int f = 0; f < NF; ++f) un[f] = __ldg(a.Un + f * N + cell);
    }

    // interior tiles (halo inside the grid) skip the boundary rule
    const bool interior = x0 >= 3 && y0 >= 3 && x0 + TX + 3 <= nx && y0 + TY + 3 <= ny;

    auto load_point = [&](int lx, int ly, double *q) {
        int cx = x0 + lx, cy = y0 + ly;
        bool fx_ = false, fy_ = false;
        if (!interior) {
            int inx, iny;
            cx = cx < nx + 2 ? cx : nx + 2;
            cy = cy < ny + 2 ? cy : ny + 2;
            cx = ghost_map(cx, nx, a.bc[0][0], a.bc[0][1], fx_, inx);
            cy = ghost_map(cy, ny, a.bc[1][0], a.bc[1][1], fy_, iny);
            if (inx >= 0 || iny >= 0) {  // a ghost of an inflow side holds the given state
                const double *st = inx >= 0 ? a.bc_state[0][inx] : a.bc_state[1][iny];
#pragma unroll
                for (int f = 0; f < NF; ++f) q[f] = st[f];
                return;
            }
        }
        const double *src = a.U + zoff + (long long)cy * nx + cx;
#pragma unroll
        for (int f = 0; f < NF; ++f) q[f] = __ldg(src + f * N);
        if (fx_) q[1] = -q[1];
        if (fy_) q[2] = -q[2];
    };

    // FP32-bulk: a point's hi/lo state (boundary rule on ghost indices)
    auto load_point_b = [&](int lx, int ly, float *h, float *l) {
        int cx = x0 + lx, cy = y0 + ly;
        bool fx_ = false, fy_ = false;
        if (!interior) {
            int inx, iny;
            cx = cx < nx + 2 ? cx : nx + 2;
            cy = cy < ny + 2 ? cy : ny + 2;
            cx = ghost_map(cx, nx, a.bc[0][0], a.bc[0][1], fx_, inx);
            cy = ghost_map(cy, ny, a.bc[1][0], a.bc[1][1], fy_, iny);
            if (inx >= 0 || iny >= 0) {
                bulk_state<NF>(inx >= 0 ? a.bc_state[0][inx] : a.bc_state[1][iny], h, l);
                return;
            }
        }
        bulk_point<NF, (ST > 0)>(a, zoff + (long long)cy * nx + cx, h, l);
        if (fx_) { h[1] = -h[1]; l[1] = -l[1]; }
        if (fy_) { h[2] = -h[2]; l[2] = -l[2]; }
    };

    // ---- phase A+F: own point (x and y fluxes) and one halo point per thread;
    // their loads go out before the reference state's barrier, so their latency
    // overlaps warp 0's work on the reference
    double uk[NF];                // U^(k) at the own cell (FP64), kept for the stage combination
    float hq[NF], lq[NF];         // the own point's hi/lo (FP32-bulk)
    if constexpr (BULK) load_point_b(tx, ty, hq, lq);
    else load_point(tx, ty, uk);
    const bool halo = threadIdx.x < NHALO;
    int hx = 0, hy = 0;
    bool hdirx = false;
    double qd[NF];
    float hh[NF], lh[NF];
    if (halo) {
        int t = threadIdx.x;
        if (t < NHY) {     // y halo: rows -3..-1 and TY..TY+2 of every tile column
            hx = t & 31;
            const int k = t >> 5;
            hy = k < 3 ? k - 3 : TY + k - 3;
        } else {           // x halo: columns -3..-1 and TX..TX+2 of every tile row
            t -= NHY;
            hy = t / 6;
            const int k = t - hy * 6;
            hx = k < 3 ? k - 3 : TX + k - 3;
            hdirx = true;
        }
        if constexpr (BULK) load_point_b(hx, hy, hh, lh);
        else load_point(hx, hy, qd);
    }

    // ---- reference state of the tile (FP32-bulk): its first cell; the LF
    // constants in FP32, converted once per block
    __shared__ float2 s_al;
    if (BULK) {
        if (threadIdx.x < 32) {  // the tile's first cell is inside the grid
            float h0[NF], l0[NF];
            load_point_b(0, 0, h0, l0);
            RefState<D> r;
            make_ref_hl<D>(h0, l0, a.gm1_f, r);
            if (threadIdx.x == 0) {
                ref = r;
                const float ax = f64_to_f32(alx);
                s_al = make_float2(ax, PD ? f64_to_f32(aly) : ax);
            }
        }
        __syncthreads();
    }
    const T alX = BULK ? (T)s_al.x : (T)alx;
    const T alY = BULK ? (T)s_al.y : (T)aly;
    const double gm1 = a.gamma - 1.0;

    // split fluxes of a point in one direction, stored at its slot of fx / fy
    auto split_store = [&](const T *fp, const T *fm, bool dirx, int lx, int ly) {
        if (dirx) {
            const int o = ly * BXP + (lx + 3);
#pragma unroll
            for (int f = 0; f < NF; ++f) {
                fx[f * NXP + o] = fp[f];
                fx[(NF + f) * NXP + o] = fm[f];
            }
        } else {
            const int o = (ly + 3) * TX + lx;
#pragma unroll
            for (int f = 0; f < NF; ++f) {
                fy[f * NYP + o] = fp[f];
                fy[(NF + f) * NYP + o] = fm[f];
            }
        }
    };
    // split flux of a point in direction DIR, stored at its slot of fx / fy
    auto flux_store = [&](const T *q, bool dirx, int lx, int ly) {
        T fp[NF], fm[NF];
        if constexpr (BULK) {
            if (dirx) split_flux_diff<D, 0, true>(q, ref, alX, a.gm1_f, fp, fm);
            else split_flux_diff<D, 1, true>(q, ref, alY, a.gm1_f, fp, fm);
        } else {
            if (dirx) split_flux_f64<D, 0, true>(q, alX, gm1, fp, fm);
            else split_flux_f64<D, 1, true>(q, alY, gm1, fp, fm);
        }
        split_store(fp, fm, dirx, lx, ly);
    };

    {
        T q[NF];
        if constexpr (BULK) {
#pragma unroll
            for (int f = 0; f < NF; ++f) q[f] = (hq[f] - ref.hi[f]) + (lq[f] - ref.lo[f]);
        } else {
#pragma unroll
            for (int f = 0; f < NF; ++f) q[f] = uk[f];
        }
        flux_store(q, true, tx, ty);
        flux_store(q, false, tx, ty);
    }
    if (halo) {
        T q[NF];
        if constexpr (BULK) {
#pragma unroll
            for (int f = 0; f < NF; ++f) q[f] = (hh[f] - ref.hi[f]) + (lh[f] - ref.lo[f]);
        } else {
#pragma unroll
            for (int f = 0; f < NF; ++f) q[f] = qd[f];
        }
        flux_store(q, hdirx, hx, hy);
    }
    __syncthreads();

    // ---- phase W: own left x face and bottom y face for every component, plus
    // one of the remaining faces (top of the tile's top row, right of its last column)
    // the shared arrays hold 2 f(+/-): reconstruct with 4 eps (twice the WENO5 value)
    const T eps = T(4) * (BULK ? (T)a.eps_f : (T)a.eps);
    // (FP32: WENO(+) and the mirrored WENO(-) of a face as one f32x2 pair)
    auto face_x = [&](int f, int ly, int j) -> T {  // between local columns j-1 and j of row ly
        const T *P = fx + f * NXP + ly * BXP;
        const T *M = fx + (NF + f) * NXP + ly * BXP;
        if constexpr (BULK)
            return weno5_pm(make_float2(P[j], M[j + 5]), make_float2(P[j + 1], M[j + 4]),
                            make_float2(P[j + 2], M[j + 3]), make_float2(P[j + 3], M[j + 2]),
                            make_float2(P[j + 4], M[j + 1]), eps);
        else
            return weno5<T>(P[j], P[j + 1], P[j + 2], P[j + 3], P[j + 4], eps) +
                   weno5<T>(M[j + 5], M[j + 4], M[j + 3], M[j + 2], M[j + 1], eps);
    };
    auto face_y = [&](int f, int lx, int j) -> T {  // between local rows j-1 and j of column lx
        const T *P = fy + f * NYP + lx;
        const T *M = fy + (NF + f) * NYP + lx;
        if constexpr (BULK)
            return weno5_pm(make_float2(P[j * TX], M[(j + 5) * TX]), make_float2(P[(j + 1) * TX], M[(j + 4) * TX]),
                            make_float2(P[(j + 2) * TX], M[(j + 3) * TX]), make_float2(P[(j + 3) * TX], M[(j + 2) * TX]),
                            make_float2(P[(j + 4) * TX], M[(j + 1) * TX]), eps);
        else
            return weno5<T>(P[j * TX], P[(j + 1) * TX], P[(j + 2) * TX], P[(j + 3) * TX], P[(j + 4) * TX], eps) +
                   weno5<T>(M[(j + 5) * TX], M[(j + 4) * TX], M[(j + 3) * TX], M[(j + 2) * TX], M[(j + 1) * TX], eps);
    };
    T fxl[NF], fyb[NF];
    if constexpr (slide<D>()) {
        // Two runs of TY + 1 = 9 windows per thread, one code path (a single
        // unrolled copy keeps the kernel inside the instruction cache):
        //   y: column `lane`, component w & 3, sign w >> 2, faces 0..8;
        //   x: row lane & 7, component lane >> 3, sign w >> 2, faces 8 s .. 8 s + 8
        //      for s = w & 3 -- neighbouring segments share one face and write it
        //      with the same value (each window is formed from its own five points).
        const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, sg = w >> 2;
#pragma unroll 1
        for (int item = 0; item < 2; ++item) {
            const T *p;
            T *out;
            int st, os;
            if (item == 0) {
                const int f = w & 3;
                p = fy + (sg * NF + f) * NYP + lane;
                out = Fy + (sg * NF + f) * NYI + lane;
                st = TX;
                os = TX;
            } else {
                const int ly = lane & 7, f = lane >> 3, j0 = (w & 3) * 8;
                p = fx + (sg * NF + f) * NXP + ly * BXP + j0;
                out = Fx + (sg * NF + f) * NXI + ly * (TX + 1) + j0;
                st = 1;
                os = 1;
            }
            if (sg) {  // WENO(-): the same run read backwards from the far end
                p += (TY + 5) * st;
                out += TY * os;
                st = -st;
                os = -os;
            }
            weno5_slide<T, TY + 1>(p, st, eps, out, os);
        }
    } else {
#pragma unroll
        for (int f = 0; f < NF; ++f) {
            fxl[f] = face_x(f, ty, tx);
            Fx[f * NXI + ty * (TX + 1) + tx] = fxl[f];
            fyb[f] = face_y(f, tx, ty);
            Fy[f * NYI + ty * TX + tx] = fyb[f];
        }
        if (threadIdx.x < NF * (TX + TY)) {
            const int t = threadIdx.x;
            if (t < NF * TX) {
                const int f = t >> 5, lx = t & 31;
                Fy[f * NYI + TY * TX + lx] = face_y(f, lx, TY);
            } else {
                const int u = t - NF * TX;
                const int f = u >> 3, ly = u & 7;
                Fx[f * NXI + ly * (TX + 1) + TX] = face_x(f, ly, TX);
            }
        }
    }
    __syncthreads();

    // ---- phase C: the cell's residual -(dF/dx) - (dG/dy) and the epilogue
    // face fluxes are twice F^: the halving rides on 1/h
    const T ihx = T(0.5) * (BULK ? (T)a.inv_h_f[0] : (T)a.inv_h[0]);
    const T ihy = T(0.5) * (BULK ? (T)a.inv_h_f[1] : (T)a.inv_h[1]);
    T r[NF];
#pragma unroll
    for (int f = 0; f < NF; ++f) {
        T dx, dy;
        if constexpr (slide<D>()) {  // F^ = WENO(+) + WENO(-) at the right/top and left/bottom faces
            const int ox = f * NXI + ty * (TX + 1) + tx, oy = f * NYI + ty * TX + tx;
            const T *FxM = Fx + NF * NXI, *FyM = Fy + NF * NYI;
            dx = (Fx[ox + 1] + FxM[ox + 1]) - (Fx[ox] + FxM[ox]);
            dy = (Fy[oy + TX] + FyM[oy + TX]) - (Fy[oy] + FyM[oy]);
        } else {
            dx = Fx[f * NXI + ty * (TX + 1) + tx + 1] - fxl[f];
            dy = Fy[f * NYI + (ty + 1) * TX + tx] - fyb[f];
        }
        r[f] = -dx * ihx - dy * ihy;
    }
    if (EPI == EPI_STORE) {
        if (own) {
            T *acc = reinterpret_cast<T *>(a.acc);
#pragma unroll
            for (int f = 0; f < NF; ++f) acc[f * N + cell] = r[f];
        }
        return;
    }
    if (EPI == EPI_RHS) {
        if (own) {
#pragma unroll
            for (int f = 0; f < NF; ++f) {
                if constexpr (BULK) a.Rout[f * N + cell] = f32_to_f64(r[f]);
                else a.Rout[f * N + cell] = r[f];
            }
        }
        return;
    }
    // EPI_STAGE (FP64): U' = a_n U^n + b_n (U^k + dt R)
    if constexpr (!BULK) {
        double cmax = 0.0, sd[D];
#pragma unroll
        for (int e = 0; e < D; ++e) sd[e] = 0.0;
        bool bad = false;
        if (own) {
            const double an = a.stage == 0 ? 0.0 : (a.stage == 1 ? 0.75 : 1.0 / 3.0);
            const double bn = a.stage == 0 ? 1.0 : (a.stage == 1 ? 0.25 : 2.0 / 3.0);
            double out[NF];
#pragma unroll
            for (int f = 0; f < NF; ++f) {
                const double sf = uk[f] + dt * r[f];
                out[f] = a.stage == 0 ? sf : an * un[f] + bn * sf;
                a.Uout[f * N + cell] = out[f];
            }
            cmax = wavespeed_f64<D>(out, a.gamma, bad);
            if (PD && !bad) dirspeeds_f64<D>(out, a.gamma, sd);
        }
        block_max_publish(cmax, bad, &a.ctl->alpha[a.slot_out], &a.ctl->status);
        if constexpr (PD) {
#pragma unroll
            for (int e = 0; e < D; ++e) block_max_publish(sd[e], false, &a.ctl->alpha_dir[a.slot_out][e], &a.ctl->status);
        }
    }
}

template <int D, bool BULK, int EPI, bool PD, int ST>
static cudaError_t launch_xy_st(const SweepArgs &a, cudaStream_t s)
{
    using L = xy::Layout<D, BULK>;
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(k_xy<D, BULK, EPI, PD, ST>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)L::bytes);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    dim3 grid((unsigned)((a.n[0] + xy::TX - 1) / xy::TX), (unsigned)((a.n[1] + xy::TY - 1) / xy::TY),
              (unsigned)a.n[2]);
    k_xy<D, BULK, EPI, PD, ST><<<grid, xy::NT, L::bytes, s>>>(a);
    return cudaGetLastError();
}

// FP32-bulk: the stage selects the stencil-state source (a handle's stage
// state exists only inside a step; L(U) reads U like stage 1)
template <int D, bool BULK, int EPI, bool PD>
static cudaError_t launch_xy_t(const SweepArgs &a, cudaStream_t s)
{
    if (!BULK || a.hl == nullptr || a.stage == 0) return launch_xy_st<D, BULK, EPI, PD, 0>(a, s);
    if (a.stage == 1) return launch_xy_st<D, BULK, EPI, PD, 1>(a, s);
    return launch_xy_st<D, BULK, EPI, PD, 2>(a, s);
}

cudaError_t launch_xy(int dim, bool bulk, int epi, const SweepArgs &a, cudaStream_t s)
{
    if (bulk && a.N >= (1ll << 32)) return cudaErrorInvalidValue;  // the stage state is indexed in 32 bits
#define X(D, B, E)                                            \
    if (dim == D && bulk == B && epi == E)                    \
        return a.per_dir ? launch_xy_t<D, B, E, true>(a, s)   \
                         : launch_xy_t<D, B, E, false>(a, s);
    X(2, false, EPI_RHS) X(2, false, EPI_STAGE) X(3, false, EPI_STORE) X(3, true, EPI_STORE)
#undef X
    return cudaErrorInvalidValue;
}

}  // namespace wg
