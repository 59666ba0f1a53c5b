// k_aux.cu -- small kernels around the residual sweeps: the global
// wavespeed max (LF alpha, Sec. 4.3), the device-side time-step control
// (dt = lambda h / alpha with the last step shortened to land on t_end,
// Eq. cfl-other), and the fixed-order FP64 conservation sums.
#include "weno_dev.cuh"
#include "weno_internal.h"

namespace wg {

template <int D, bool BULK>
__global__ void __launch_bounds__(256) k_alpha(const double *__restrict__ U, long long N, double gamma, Ctl *ctl,
                                               int slot, int per_dir)
{
    constexpr int NF = D + 2;
    double m = 0.0, md[D];
    float mf = 0.0f, mdf[D];
#pragma unroll
    for (int e = 0; e < D; ++e) { md[e] = 0.0; mdf[e] = 0.0f; }
    bool bad = false;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
        double q[NF];
#pragma unroll
        for (int f = 0; f < NF; ++f) q[f] = __ldg(U + f * N + i);
        bool b;
        if (BULK) {
            float qf[NF];
#pragma unroll
            for (int f = 0; f < NF; ++f) qf[f] = f64_to_f32(q[f]);
            mf = fmaxf(mf, wavespeed_f32<D>(qf, (float)gamma, b));
            if (per_dir) {
                float sd[D];
                dirspeeds_f32<D>(qf, (float)gamma, sd);
#pragma unroll
                for (int e = 0; e < D; ++e) mdf[e] = fmaxf(mdf[e], b ? 0.0f : sd[e]);
            }
        } else {
            m = fmax(m, wavespeed_f64<D>(q, gamma, b));
            if (per_dir) {
                double sd[D];
                dirspeeds_f64<D>(q, gamma, sd);
#pragma unroll
                for (int e = 0; e < D; ++e) md[e] = fmax(md[e], b ? 0.0 : sd[e]);
            }
        }
        bad |= b;
    }
    if (BULK) {
        m = (double)mf;
#pragma unroll
        for (int e = 0; e < D; ++e) md[e] = (double)mdf[e];
    }
    block_max_publish(m, bad, &ctl->alpha[slot], &ctl->status);
    if (per_dir) {
#pragma unroll
        for (int e = 0; e < D; ++e) block_max_publish(md[e], false, &ctl->alpha_dir[slot][e], &ctl->status);
    }
}

// Scalar laws: alpha = max |f'(u)| (1 for advection, |u| for Burgers).
template <int M>
__global__ void __launch_bounds__(256) k_alpha_scalar(const double *__restrict__ U, long long N, Ctl *ctl, int slot)
{
    double m = 0.0;
    bool bad = false;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
        const double u = __ldg(U + i);
        bad |= !isfinite(u);
        m = fmax(m, M == MODEL_ADVECT ? 1.0 : fabs(u));
    }
    block_max_publish(m, bad, &ctl->alpha[slot], &ctl->status);
}

__global__ void k_reset_slot(Ctl *ctl, int slot)
{
    ctl->alpha[slot] = 0ull;
    for (int e = 0; e < 3; ++e) ctl->alpha_dir[slot][e] = 0ull;
}

__global__ void k_copy_alpha(const Ctl *ctl, int slot, double *out)
{
    out[0] = __longlong_as_double((long long)ctl->alpha[slot]);
}

// Start of a step: dt from alpha(U^n) (or the fixed dt), shortened so that the
// time lands exactly on t_end; zero when the time is up or the step budget of
// the current call is spent.  Clears the stage alpha slots 1..3.
__global__ void k_step_begin(Ctl *c)
{
    const double t = c->t, te = c->t_end;
    const double alpha = __longlong_as_double((long long)c->alpha[0]);
    double dt = c->dt_req > 0.0 ? c->dt_req : c->cfl_h / alpha;
    double tn = t + dt;
    if (!(dt > 0.0) || !isfinite(dt)) {
        if (t < te && c->steps < c->max_steps) atomicOr(&c->status, ST_NONPHYSICAL);
        dt = 0.0;
        tn = t;
    } else if (!(t < te) || c->steps >= c->max_steps) {
        dt = 0.0;
        tn = t;
    } else if (tn >= te) {
        dt = te - t;
        tn = te;
    }
    c->dt = dt;
    c->t_next = tn;
    c->bdt[0] = f64_to_f32x2(dt);
    c->bdt[1] = f64_to_f32x2(0.25 * dt);
    c->bdt[2] = f64_to_f32x2(2.0 / 3.0 * dt);
    for (int k = 1; k < 4; ++k) {
        c->alpha[k] = 0ull;
        for (int e = 0; e < 3; ++e) c->alpha_dir[k][e] = 0ull;
    }
}

// End of a step: advance the time and carry alpha(U^{n+1}) into slot 0.
__global__ void k_step_end(Ctl *c)
{
    if (c->dt > 0.0) {
        c->t = c->t_next;
        c->steps += 1;
        c->alpha[0] = c->alpha[3];
        for (int e = 0; e < 3; ++e) c->alpha_dir[0][e] = c->alpha_dir[3][e];
    }
}

// Two-level fixed-order sums: block b reduces a fixed contiguous chunk of
// cells with a fixed tree; one block then reduces the partials in order.
constexpr int SUM_NT = 256;

__device__ __forceinline__ double block_sum_fixed(double v, double *sh)
{
    sh[threadIdx.x] = v;
    __syncthreads();
    for (int o = SUM_NT / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
        __syncthreads();
    }
    const double r = sh[0];
    __syncthreads();
    return r;
}

__global__ void __launch_bounds__(SUM_NT) k_sums_partial(const double *__restrict__ U, int nf, long long N,
                                                         long long chunk, double *partials)
{
    __shared__ double sh[SUM_NT];
    const long long b0 = (long long)blockIdx.x * chunk;
    const long long b1 = b0 + chunk < N ? b0 + chunk : N;
    for (int f = 0; f < nf; ++f) {
        double s = 0.0;
        for (long long i = b0 + threadIdx.x; i < b1; i += SUM_NT) s += U[f * N + i];
        s = block_sum_fixed(s, sh);
        if (threadIdx.x == 0) partials[(long long)blockIdx.x * nf + f] = s;
    }
}

__global__ void __launch_bounds__(SUM_NT) k_sums_final(const double *partials, int nblocks, int nf, double *out)
{
    __shared__ double sh[SUM_NT];
    for (int f = 0; f < nf; ++f) {
        double s = 0.0;
        for (int b = threadIdx.x; b < nblocks; b += SUM_NT) s += partials[(long long)b * nf + f];
        s = block_sum_fixed(s, sh);
        if (threadIdx.x == 0) out[f] = s;
    }
}

int sums_blocks(long long N)
{
    const long long b = (N + 4095) / 4096;
    return (int)(b < 1024 ? (b < 1 ? 1 : b) : 1024);
}

cudaError_t launch_sums(const double *U, int nf, long long N, double *partials, int nblocks, double *out,
                        cudaStream_t s)
{
    const long long chunk = (N + nblocks - 1) / nblocks;
    k_sums_partial<<<nblocks, SUM_NT, 0, s>>>(U, nf, N, chunk, partials);
    k_sums_final<<<1, SUM_NT, 0, s>>>(partials, nblocks, nf, out);
    return cudaGetLastError();
}

int sm_count()
{
    static int cache[64] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 152;
    if (cache[dev] == 0) {
        int n = 0;
        if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n < 1) return 152;
        cache[dev] = n;
    }
    return cache[dev];
}

cudaError_t launch_alpha(int model, int dim, bool bulk, const double *U, long long N, double gamma, Ctl *ctl,
                         int slot, int per_dir, cudaStream_t s)
{
    int blocks = (int)((N + 255) / 256);
    if (blocks > sm_count() * 8) blocks = sm_count() * 8;
    if (blocks < 1) blocks = 1;
    if (model == MODEL_ADVECT) k_alpha_scalar<MODEL_ADVECT><<<blocks, 256, 0, s>>>(U, N, ctl, slot);
    if (model == MODEL_BURGERS) k_alpha_scalar<MODEL_BURGERS><<<blocks, 256, 0, s>>>(U, N, ctl, slot);
    if (model != MODEL_EULER) return cudaGetLastError();
#define X(D, B) \
    if (dim == D && bulk == B) k_alpha<D, B><<<blocks, 256, 0, s>>>(U, N, gamma, ctl, slot, per_dir);
    X(1, false) X(2, false) X(3, false) X(1, true) X(2, true) X(3, true)
#undef X
    return cudaGetLastError();
}

cudaError_t launch_reset_slot(Ctl *ctl, int slot, cudaStream_t s)
{
    k_reset_slot<<<1, 1, 0, s>>>(ctl, slot);
    return cudaGetLastError();
}

cudaError_t launch_copy_alpha(const Ctl *ctl, int slot, double *out, cudaStream_t s)
{
    k_copy_alpha<<<1, 1, 0, s>>>(ctl, slot, out);
    return cudaGetLastError();
}

cudaError_t launch_step_begin(Ctl *ctl, cudaStream_t s)
{
    k_step_begin<<<1, 1, 0, s>>>(ctl);
    return cudaGetLastError();
}

cudaError_t launch_step_end(Ctl *ctl, cudaStream_t s)
{
    k_step_end<<<1, 1, 0, s>>>(ctl);
    return cudaGetLastError();
}

}  // namespace wg
