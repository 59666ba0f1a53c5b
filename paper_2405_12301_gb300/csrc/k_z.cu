// k_z.cu -- z direction of the WENO5-JS residual for 3D grids, ending the
// residual of a stage (the x and y directions run in k_xy.cu).
#include <type_traits>

#include "bulk_load.cuh"
#include "weno_dev.cuh"
#include "weno_internal.h"

namespace wg {

// ---------------------------------------------------------------------------
// z direction of a 3D grid, ending the residual: a CTA owns 32 x-cells x TZ = 8
// z-cells of one y-row, one cell per thread, plus the 3 + 3 halo z-planes of
// its 32 columns.  Same phases as above for one direction; the epilogue adds
// the x+y part left in the accumulator by k_xy<3, ..., EPI_STORE>, then writes
// L(U) or applies the SSP-RK3 stage combination and publishes the wavespeed max.
// FP32-bulk runs the stages on increments (the stage state of k_xy2.cu): stage
// 1 stores the hi/lo split of U^n and Delta_1, stages 2 and 3 read them, and
// only stage 3 touches FP64 (U^{n+1} = U^n + Delta_3); ST is the stage.
namespace zs {
constexpr int NT = 256;
constexpr int TX = 32, TZ = 8;
constexpr int BZ = TZ + 6;                  // column extent with halo
constexpr int NZP = TX * BZ;                // z-flux points: 32 x 14
constexpr int NZI = TX * (TZ + 1);          // z interfaces: 32 x 9
constexpr int NHALO = 6 * TX;               // 192 halo points

template <bool BULK> struct Layout {
    using T = typename std::conditional<BULK, float, double>::type;
    static constexpr int NF = 5;
    static constexpr size_t F_off = 0;
    static constexpr size_t fz_off = (sizeof(T) * NF * NZI + 15) & ~size_t(15);
    static constexpr size_t ref_off = (fz_off + sizeof(T) * 2 * NF * NZP + 15) & ~size_t(15);
    // FP32-bulk: the epilogue's own-cell operands, copied asynchronously at the
    // start (the x+y residual, Delta_k, and in stage 3 U^n): [NF][NT] each
    static constexpr size_t e_off = (ref_off + sizeof(RefState<3>) + 15) & ~size_t(15);
    static constexpr size_t bytes = BULK ? e_off + 2 * sizeof(float) * NF * NT : ref_off + sizeof(RefState<3>);
    // (e_din holds a float4 per thread, the first four fields, then a float, E)
    static constexpr size_t bytes_un = BULK ? bytes + sizeof(double) * NF * NT : bytes;  // stage 3
};

__device__ __forceinline__ void cp_async4(void *dst, const void *src)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"((unsigned)__cvta_generic_to_shared(dst)), "l"(src)
                 : "memory");
}
__device__ __forceinline__ void cp_async16(void *dst, const void *src)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"((unsigned)__cvta_generic_to_shared(dst)), "l"(src)
                 : "memory");
}
__device__ __forceinline__ void cp_async8(void *dst, const void *src)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"((unsigned)__cvta_generic_to_shared(dst)), "l"(src)
                 : "memory");
}
}  // namespace zs

template <bool BULK, int EPI, bool PD, int ST = 0>
__global__ void __launch_bounds__(zs::NT, BULK ? 5 : 1) k_z(const SweepArgs a)
{
    using namespace zs;
    using L = Layout<BULK>;
    using T = typename L::T;
    constexpr int NF = 5;
    extern __shared__ __align__(16) unsigned char smem[];
    T *Fz = reinterpret_cast<T *>(smem + L::F_off);        // [NF][TZ+1][TX]
    T *fz = reinterpret_cast<T *>(smem + L::fz_off);       // [2][NF][BZ][TX]
    RefState<3> &ref = *reinterpret_cast<RefState<3> *>(smem + L::ref_off);

    const long long dtbits = __double_as_longlong(a.ctl->dt);
    if (a.check_dt && dtbits == 0) return;
    const double dt = __longlong_as_double(dtbits);
    const double alpha = PD ? __longlong_as_double((long long)a.ctl->alpha_dir[a.slot_in][2])
                                   : __longlong_as_double((long long)a.ctl->alpha[a.slot_in]);
    // FP32-bulk: alpha converted once per block (b_k dt comes from the control
    // block as an FP32 pair, set with dt)
    __shared__ float s_al;
    if (BULK && threadIdx.x == 0) s_al = f64_to_f32(alpha);

    const int nx = a.n[0], nz = a.n[2];
    const long long N = a.N, sz = a.stride[2];
    // z-tiles are the fastest grid index, so that tiles sharing halo planes run
    // close together and find those planes in L2
    const int x0 = blockIdx.y * TX, z0 = blockIdx.x * TZ;
    const long long yoff = (long long)blockIdx.z * a.stride[1];
    const int tx = threadIdx.x & 31, tz = threadIdx.x >> 5;
    const int gx = x0 + tx, gz = z0 + tz;
    const bool own = gx < nx && gz < nz;
    const long long cell = yoff + (long long)(gz < nz ? gz : nz - 1) * sz + (gx < nx ? gx : nx - 1);

    double un[NF];
    if (!BULK && EPI == EPI_STAGE && a.stage > 0) {
#pragma unroll
        for (int f = 0; f < NF; ++f) un[f] = __ldg(a.Un + f * N + cell);
    }
    // FP32-bulk: the epilogue's operands go out now as asynchronous copies into
    // shared memory, so their latency hides behind the whole residual
    float *e_acc = reinterpret_cast<float *>(smem + L::e_off);  // [NF][NT]
    float *e_din = e_acc + NF * NT;                             // [NF][NT]
    double *e_un = reinterpret_cast<double *>(e_din + NF * NT); // [NF][NT] (stage 3)
    if (BULK && own) {
        const float *acc = reinterpret_cast<const float *>(a.acc);
#pragma unroll
        for (int f = 0; f < NF; ++f) {
            cp_async4(e_acc + f * NT + threadIdx.x, acc + f * N + cell);
            if (EPI == EPI_STAGE && ST == 2) cp_async8(e_un + f * NT + threadIdx.x, a.U + f * N + cell);
        }
        if (EPI == EPI_STAGE && ST > 0) {  // Delta_k: the float4 plane of the first four fields, then E
            cp_async16(reinterpret_cast<float4 *>(e_din) + threadIdx.x, reinterpret_cast<const float4 *>(a.din) + cell);
            cp_async4(e_din + 4 * NT + threadIdx.x, a.din1 + cell);
        }
    }
    if (BULK) asm volatile("cp.async.commit_group;" ::: "memory");
    const double gm1 = a.gamma - 1.0;
    const bool interior = z0 >= 3 && z0 + TZ + 3 <= nz && x0 + TX <= nx;

    auto load_point = [&](int lx, int lz, double *q) {
        int cx = x0 + lx, cz = z0 + lz;
        bool fz_ = false;
        if (!interior) {
            int inz;
            cx = cx < nx ? cx : nx - 1;  // columns beyond the grid only feed cells that are not written
            cz = cz < nz + 2 ? cz : nz + 2;
            cz = ghost_map(cz, nz, a.bc[2][0], a.bc[2][1], fz_, inz);
            if (inz >= 0) {  // a ghost of an inflow side holds the given state
#pragma unroll
                for (int f = 0; f < NF; ++f) q[f] = a.bc_state[2][inz][f];
                return;
            }
        }
        const double *src = a.U + yoff + (long long)cz * sz + cx;
#pragma unroll
        for (int f = 0; f < NF; ++f) q[f] = __ldg(src + f * N);
        if (fz_) q[3] = -q[3];
    };
    // FP32-bulk: a point's hi/lo state (boundary rule on ghost indices)
    auto load_point_b = [&](int lx, int lz, float *h, float *l) {
        int cx = x0 + lx, cz = z0 + lz;
        bool fz_ = false;
        if (!interior) {
            int inz;
            cx = cx < nx ? cx : nx - 1;
            cz = cz < nz + 2 ? cz : nz + 2;
            cz = ghost_map(cz, nz, a.bc[2][0], a.bc[2][1], fz_, inz);
            if (inz >= 0) {
                bulk_state<NF>(a.bc_state[2][inz], h, l);
                return;
            }
        }
        bulk_point<NF, (ST > 0)>(a, yoff + (long long)cz * sz + cx, h, l);
        if (fz_) { h[3] = -h[3]; l[3] = -l[3]; }
    };
    auto flux_store = [&](const T *q, int lx, int lz) {
        T fp[NF], fm[NF];
        const T al = BULK ? (T)s_al : (T)alpha;  // (s_al is read after the reference state's barrier)
        if constexpr (BULK) split_flux_diff<3, 2, true>(q, ref, al, a.gm1_f, fp, fm);
        else split_flux_f64<3, 2, true>(q, al, gm1, fp, fm);
        const int o = (lz + 3) * TX + lx;
#pragma unroll
        for (int f = 0; f < NF; ++f) {
            fz[f * NZP + o] = fp[f];
            fz[(NF + f) * NZP + o] = fm[f];
        }
    };

    // own and halo loads go out before the reference state's barrier, so their
    // latency overlaps warp 0's work on the reference
    double uk[NF];
    float hk[NF], lk[NF];  // FP32-bulk: the own point's hi/lo
    if constexpr (BULK) load_point_b(tx, tz, hk, lk);
    else load_point(tx, tz, uk);
    const bool halo = threadIdx.x < NHALO;
    const int hx = threadIdx.x & 31, hz = (threadIdx.x >> 5) < 3 ? (threadIdx.x >> 5) - 3 : TZ + (threadIdx.x >> 5) - 3;
    double qd[NF];
    float hh[NF], lh[NF];
    if (halo) {
        if constexpr (BULK) load_point_b(hx, hz, hh, lh);
        else load_point(hx, hz, qd);
    }
    if (BULK && EPI == EPI_STAGE && ST == 0 && own) {  // the split of U^n, read by stages 2 and 3
#pragma unroll
        bulk_store_hl(a, cell, hk, lk);
    }
    if (BULK) {
        if (threadIdx.x < 32) {  // the tile's first cell is inside the grid
            float h0[NF], l0[NF];
            load_point_b(0, 0, h0, l0);
            RefState<3> r;
            make_ref_hl<3>(h0, l0, a.gm1_f, r);
            if (threadIdx.x == 0) ref = r;
        }
        __syncthreads();
    }
    {
        T q[NF];
        if constexpr (BULK) {
#pragma unroll
            for (int f = 0; f < NF; ++f) q[f] = (hk[f] - ref.hi[f]) + (lk[f] - ref.lo[f]);
        } else {
#pragma unroll
            for (int f = 0; f < NF; ++f) q[f] = uk[f];
        }
        flux_store(q, tx, tz);
    }
    if (halo) {
        const int lx = hx, lz = hz;
        T q[NF];
        if constexpr (BULK) {
#pragma unroll
            for (int f = 0; f < NF; ++f) q[f] = (hh[f] - ref.hi[f]) + (lh[f] - ref.lo[f]);
        } else {
#pragma unroll
            for (int f = 0; f < NF; ++f) q[f] = qd[f];
        }
        flux_store(q, lx, lz);
    }
    __syncthreads();

    // the shared arrays hold 2 f(+/-): reconstruct with 4 eps (twice the WENO5 value)
    const T eps = T(4) * (BULK ? (T)a.eps_f : (T)a.eps);
    // (FP32: WENO(+) and the mirrored WENO(-) of a face as one f32x2 pair)
    auto face_z = [&](int f, int lx, int j) -> T {  // between local planes j-1 and j of column lx
        const T *P = fz + f * NZP + lx;
        const T *M = fz + (NF + f) * NZP + lx;
        if constexpr (BULK)
            return weno5_pm(make_float2(P[j * TX], M[(j + 5) * TX]), make_float2(P[(j + 1) * TX], M[(j + 4) * TX]),
                            make_float2(P[(j + 2) * TX], M[(j + 3) * TX]), make_float2(P[(j + 3) * TX], M[(j + 2) * TX]),
                            make_float2(P[(j + 4) * TX], M[(j + 1) * TX]), eps);
        else
            return weno5<T>(P[j * TX], P[(j + 1) * TX], P[(j + 2) * TX], P[(j + 3) * TX], P[(j + 4) * TX], eps) +
                   weno5<T>(M[(j + 5) * TX], M[(j + 4) * TX], M[(j + 3) * TX], M[(j + 2) * TX], M[(j + 1) * TX], eps);
    };
    T fzb[NF];
#pragma unroll
    for (int f = 0; f < NF; ++f) {
        fzb[f] = face_z(f, tx, tz);
        Fz[f * NZI + tz * TX + tx] = fzb[f];
    }
    if (threadIdx.x < NF * TX) {
        const int f = threadIdx.x >> 5, lx = threadIdx.x & 31;
        Fz[f * NZI + TZ * TX + lx] = face_z(f, lx, TZ);
    }
    __syncthreads();

    const T ihz = T(0.5) * (BULK ? (T)a.inv_h_f[2] : (T)a.inv_h[2]);  // face fluxes are twice F^
    const T *acc = reinterpret_cast<const T *>(a.acc);
    if (BULK) asm volatile("cp.async.wait_group 0;" ::: "memory");  // this thread's own copies
    T r[NF];
#pragma unroll
    for (int f = 0; f < NF; ++f) {
        const T dz = Fz[f * NZI + (tz + 1) * TX + tx] - fzb[f];
        if constexpr (BULK) r[f] = e_acc[f * NT + threadIdx.x] + (-dz * ihz);
        else r[f] = acc[f * N + cell] + (-dz * ihz);
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
    if constexpr (BULK) {
        // Delta_{k+1} = b_k (Delta_k + dt R); stage 3 ends the step with U^n + Delta_3
        float s = 0.0f, sd[3] = {0.0f, 0.0f, 0.0f};
        bool bad = false;
        if (own) {
            // b_k dt and c_k = 2/3 as hi + lo pairs: no systematic coefficient rounding
            const float2 bdt = a.ctl->bdt[ST];
            constexpr float c_hi = ST == 1 ? 0.25f : (float)(2.0 / 3.0);
            constexpr float c_lo = ST == 1 ? 0.0f : (float)(2.0 / 3.0 - (double)(float)(2.0 / 3.0));
            float qn[NF], dn[NF];
#pragma unroll
            for (int f = 0; f < NF; ++f) {
                float t = bdt.y * r[f];
                if (ST > 0) {
                    const float dkf = f < 4 ? e_din[4 * threadIdx.x + f] : e_din[4 * NT + threadIdx.x];
                    t = fmaf(c_hi, dkf, fmaf(c_lo, dkf, t));
                }
                const float d = fmaf(bdt.x, r[f], t);
                if (ST < 2) dn[f] = d;
                else a.Uout[f * N + cell] = e_un[f * NT + threadIdx.x] + f32_to_f64(d);
                qn[f] = hk[f] + d;  // the new state in FP32 (hk is the hi part of U^n)
            }
            if (ST < 2) {  // Delta_{k+1}: the float4 plane of the first four fields, then E
                reinterpret_cast<float4 *>(a.dout)[(unsigned)cell] = make_float4(dn[0], dn[1], dn[2], dn[3]);
                a.dout1[(unsigned)cell] = dn[4];
            }
            s = wavespeed_f32<3>(qn, a.gamma_f, bad);
            if (PD && !bad) dirspeeds_f32<3>(qn, a.gamma_f, sd);
        }
        block_max_publish_f32(s, bad, &a.ctl->alpha[a.slot_out], &a.ctl->status);
        if constexpr (PD) {
#pragma unroll
            for (int e = 0; e < 3; ++e) block_max_publish_f32(sd[e], false, &a.ctl->alpha_dir[a.slot_out][e], &a.ctl->status);
        }
    } else {
        double cmax = 0.0, sd[3] = {0.0, 0.0, 0.0};
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
            cmax = wavespeed_f64<3>(out, a.gamma, bad);
            if (PD && !bad) dirspeeds_f64<3>(out, a.gamma, sd);
        }
        block_max_publish(cmax, bad, &a.ctl->alpha[a.slot_out], &a.ctl->status);
        if constexpr (PD) {
#pragma unroll
            for (int e = 0; e < 3; ++e) block_max_publish(sd[e], false, &a.ctl->alpha_dir[a.slot_out][e], &a.ctl->status);
        }
    }
}

template <bool BULK, int EPI, bool PD, int ST>
static cudaError_t launch_z_st(const SweepArgs &a, cudaStream_t s)
{
    using L = zs::Layout<BULK>;
    constexpr size_t bytes = (BULK && EPI == EPI_STAGE && ST == 2) ? L::bytes_un : L::bytes;
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(k_z<BULK, EPI, PD, ST>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)bytes);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    dim3 grid((unsigned)((a.n[2] + zs::TZ - 1) / zs::TZ), (unsigned)((a.n[0] + zs::TX - 1) / zs::TX), (unsigned)a.n[1]);
    k_z<BULK, EPI, PD, ST><<<grid, zs::NT, bytes, s>>>(a);
    return cudaGetLastError();
}

template <bool BULK, int EPI, bool PD>
static cudaError_t launch_z_t(const SweepArgs &a, cudaStream_t s)
{
    if (!BULK || EPI != EPI_STAGE || a.stage == 0) return launch_z_st<BULK, EPI, PD, 0>(a, s);
    if (a.stage == 1) return launch_z_st<BULK, EPI, PD, 1>(a, s);
    return launch_z_st<BULK, EPI, PD, 2>(a, s);
}

cudaError_t launch_z(bool bulk, int epi, const SweepArgs &a, cudaStream_t s)
{
    if (bulk && a.N >= (1ll << 32)) return cudaErrorInvalidValue;  // the stage state is indexed in 32 bits
#define X(B, E, P) \
    if (bulk == B && epi == E && (a.per_dir != 0) == P) return launch_z_t<B, E, P>(a, s);
    X(false, EPI_RHS, false) X(false, EPI_STAGE, false) X(true, EPI_RHS, false) X(true, EPI_STAGE, false)
    X(false, EPI_RHS, true) X(false, EPI_STAGE, true) X(true, EPI_RHS, true) X(true, EPI_STAGE, true)
#undef X
    return cudaErrorInvalidValue;
}

}  // namespace wg
