// tc_contract.cu -- A/B of the rank contraction of the cross evaluation on the
// 5th-generation tensor cores against the FP32 FMA pipe.
//
// The contraction of k_cross, with the stencil across the fiber, is per field a
// product D = A B^T with A the varying side's shifted vectors ((varying index,
// shift) rows, K = rank entries each) and B the chunk's contracted core rows
// (one row per sample).  This probe times that product alone on tiles of the
// shape a tensor-core path of k_cross would use: M = 128 rows of A (18 varying
// indices x 7 shifts, padded), N = 16 or 64 rows of B, K = 32 (the largest rank).
//
//   k_tc:   A and B are split into TF32 hi + lo (round to nearest) and staged in
//           shared memory in the canonical K-major layout without swizzle (core
//           matrices of 8 rows x 16 bytes); one thread issues, per 8-wide K step,
//           tcgen05.mma kind::tf32 for hi*hi, hi*lo and lo*hi (the 3-term split:
//           TF32 alone is too coarse for FP32 results), accumulating in TMEM;
//           tcgen05.commit signals an mbarrier; the four warps read D back with
//           tcgen05.ld (warp w owns TMEM lanes 32w..32w+31) and store it.
//   k_simt: each thread forms its row's N dot products on the FMA pipe, in f32x2
//           even/odd pairs as k_cross does, B staged in shared memory.
//
// Both read the same pool of tiles and write D to global memory; the host
// checks both against FP64 products and times them with CUDA events.  Every
// wait on the mbarrier is bounded: past the limit the kernel records a timeout,
// still waits (bounded) for its MMAs, frees its TMEM and returns.
// Output: one JSON line per configuration.
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <vector>
#include <cuda_runtime.h>

constexpr int M = 128, K = 32;
constexpr int NT = 128;                 // four warps: the 128 TMEM lanes of D
constexpr int LBO = 128;                // bytes between core matrices adjacent in K
constexpr int SBO = (K / 4) * 128;      // bytes between core matrices adjacent in M / N (8-row groups)

__device__ int g_timeout;

__device__ __forceinline__ unsigned smem_u32(const void *p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ unsigned tf32_rna(float x)
{
    unsigned r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return r;
}

// Shared-memory matrix descriptor: start address, leading (K) and stride (M/N)
// byte offsets, descriptor version 1, no swizzle.
__device__ __forceinline__ unsigned long long smem_desc(const void *p)
{
    const unsigned long long a = (smem_u32(p) & 0x3FFFFu) >> 4;
    return a | ((unsigned long long)(LBO >> 4) << 16) | ((unsigned long long)(SBO >> 4) << 32) | (1ull << 46);
}

// Instruction descriptor of kind::tf32: D in FP32, A and B TF32, both K-major,
// N >> 3 in bits 17-22, M >> 4 in bits 24-28.
__host__ __device__ constexpr unsigned instr_desc(int m, int n)
{
    return (1u << 4) | (2u << 7) | (2u << 10) | ((unsigned)(n >> 3) << 17) | ((unsigned)(m >> 4) << 24);
}

// element (r, k) of an R x K operand in the canonical K-major layout
__device__ __forceinline__ int kmajor_off(int r, int k) { return (r >> 3) * SBO + (k >> 2) * LBO + (r & 7) * 16 + (k & 3) * 4; }

__device__ __forceinline__ bool mbar_wait(unsigned bar, unsigned parity, long long limit)
{
    for (long long i = 0; i < limit; ++i) {
        unsigned ok;
        asm volatile(
            "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}"
            : "=r"(ok)
            : "r"(bar), "r"(parity)
            : "memory");
        if (ok) return true;
    }
    return false;
}

template <int N>
__global__ void __launch_bounds__(NT) k_tc(const float *__restrict__ A, const float *__restrict__ B, float *D,
                                            int tiles, int iters)
{
    constexpr int TMEM_COLS = N < 32 ? 32 : N;
    extern __shared__ __align__(1024) unsigned char sm[];
    unsigned char *Ahi = sm, *Alo = Ahi + M * K * 4, *Bhi = Alo + M * K * 4, *Blo = Bhi + N * K * 4;
    __shared__ __align__(8) unsigned long long bar;
    __shared__ unsigned tmem_base;
    const int t = threadIdx.x, w = t >> 5;
    if (w == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base)),
                     "r"(TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (t == 0) asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&bar)) : "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const unsigned tmem = tmem_base;
    const unsigned idesc = instr_desc(M, N);
    bool failed = false;
    int issued = 0;  // MMA groups committed (each completes one mbarrier phase)
    for (int it = 0; it < iters; ++it) {
        const int tile = (blockIdx.x + it * gridDim.x) % tiles;
        // stage A (row t) and B (rows t, t + 128, ...) as TF32 hi / lo
        {
            const float4 *a = reinterpret_cast<const float4 *>(A + ((size_t)tile * M + t) * K);
#pragma unroll
            for (int q = 0; q < K / 4; ++q) {
                const float4 v = __ldg(a + q);
                const uint4 h = make_uint4(tf32_rna(v.x), tf32_rna(v.y), tf32_rna(v.z), tf32_rna(v.w));
                const uint4 l = make_uint4(tf32_rna(v.x - __uint_as_float(h.x)), tf32_rna(v.y - __uint_as_float(h.y)),
                                           tf32_rna(v.z - __uint_as_float(h.z)), tf32_rna(v.w - __uint_as_float(h.w)));
                *reinterpret_cast<uint4 *>(Ahi + kmajor_off(t, 4 * q)) = h;
                *reinterpret_cast<uint4 *>(Alo + kmajor_off(t, 4 * q)) = l;
            }
            for (int u = t; u < N * K / 4; u += NT) {
                const int r = u / (K / 4), q = u % (K / 4);
                const float4 v = __ldg(reinterpret_cast<const float4 *>(B + ((size_t)tile * N + r) * K) + q);
                const uint4 h = make_uint4(tf32_rna(v.x), tf32_rna(v.y), tf32_rna(v.z), tf32_rna(v.w));
                const uint4 l = make_uint4(tf32_rna(v.x - __uint_as_float(h.x)), tf32_rna(v.y - __uint_as_float(h.y)),
                                           tf32_rna(v.z - __uint_as_float(h.z)), tf32_rna(v.w - __uint_as_float(h.w)));
                *reinterpret_cast<uint4 *>(Bhi + kmajor_off(r, 4 * q)) = h;
                *reinterpret_cast<uint4 *>(Blo + kmajor_off(r, 4 * q)) = l;
            }
        }
        // the operands are read by the tensor cores through the async proxy
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();
        if (t == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll
            for (int ks = 0; ks < K / 8; ++ks) {  // 8 TF32 per K step: two core matrices
                const unsigned long long ah = smem_desc(Ahi + ks * 2 * LBO), al = smem_desc(Alo + ks * 2 * LBO);
                const unsigned long long bh = smem_desc(Bhi + ks * 2 * LBO), bl = smem_desc(Blo + ks * 2 * LBO);
                const unsigned acc0 = ks > 0 ? 1u : 0u;  // the first product of a tile starts D afresh
                asm volatile(
                    "{\n.reg .pred p, q;\nsetp.ne.b32 p, %6, 0;\nsetp.eq.b32 q, %6, %6;\n"
                    "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %3, %5, p;\n"
                    "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %4, %5, q;\n"
                    "tcgen05.mma.cta_group::1.kind::tf32 [%0], %2, %3, %5, q;\n}" ::"r"(tmem),
                    "l"(ah), "l"(al), "l"(bh), "l"(bl), "r"(idesc), "r"(acc0)
                    : "memory");
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                             smem_u32(&bar))
                         : "memory");
        }
        ++issued;
        const bool ok = mbar_wait(smem_u32(&bar), (unsigned)((issued - 1) & 1), 1ll << 20);
        failed = __syncthreads_or(!ok) != 0;  // one decision for the whole block
        if (failed) break;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        // D rows 32 w .. 32 w + 31 (this warp's TMEM lanes), 16 columns per load
#pragma unroll
        for (int c0 = 0; c0 < N; c0 += 16) {
            unsigned r[16];
            const unsigned taddr = tmem + ((unsigned)(32 * w) << 16) + (unsigned)c0;
            asm volatile(
                "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, "
                "%14, %15}, [%16];"
                : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                  "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
                : "r"(taddr)
                : "memory");
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
            float4 *o = reinterpret_cast<float4 *>(D + ((size_t)tile * M + t) * N + c0);
#pragma unroll
            for (int q = 0; q < 4; ++q)
                o[q] = make_float4(__uint_as_float(r[4 * q]), __uint_as_float(r[4 * q + 1]), __uint_as_float(r[4 * q + 2]),
                                   __uint_as_float(r[4 * q + 3]));
        }
        // every lane's reads of D end before the next tile's MMAs overwrite it
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();
    }
    if (failed) {
        if (t == 0) atomicExch(&g_timeout, 1);
        mbar_wait(smem_u32(&bar), (unsigned)((issued - 1) & 1), 1ll << 20);  // the MMAs in flight, bounded
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (w == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS) : "memory");
    }
}

template <int N>
__global__ void __launch_bounds__(NT) k_simt(const float *__restrict__ A, const float *__restrict__ B, float *D,
                                              int tiles, int iters)
{
    __shared__ __align__(16) float Bs[N * K];
    const int t = threadIdx.x;
    for (int it = 0; it < iters; ++it) {
        const int tile = (blockIdx.x + it * gridDim.x) % tiles;
        __syncthreads();
        for (int u = t; u < N * K / 4; u += NT)
            reinterpret_cast<float4 *>(Bs)[u] = __ldg(reinterpret_cast<const float4 *>(B + (size_t)tile * N * K) + u);
        __syncthreads();
        const float4 *a = reinterpret_cast<const float4 *>(A + ((size_t)tile * M + t) * K);
        float4 av[K / 4];
#pragma unroll
        for (int q = 0; q < K / 4; ++q) av[q] = __ldg(a + q);
#pragma unroll 4
        for (int n = 0; n < N; ++n) {
            const float4 *b = reinterpret_cast<const float4 *>(Bs + n * K);
            float2 s = make_float2(0.0f, 0.0f);
#pragma unroll
            for (int q = 0; q < K / 4; ++q) {
                const float4 bv = b[q];
                s = __ffma2_rn(make_float2(av[q].z, av[q].w), make_float2(bv.z, bv.w),
                               __ffma2_rn(make_float2(av[q].x, av[q].y), make_float2(bv.x, bv.y), s));
            }
            D[((size_t)tile * M + t) * N + n] = s.x + s.y;
        }
    }
}

static void ck(cudaError_t e, const char *what)
{
    if (e != cudaSuccess) {
        fprintf(stderr, "%s: %s\n", what, cudaGetErrorString(e));
        exit(1);
    }
}

// worst |D - D64| / sum_k |a_k b_k| over a sample of tiles
static double check(const std::vector<float> &A, const std::vector<float> &B, const std::vector<float> &D, int N,
                    int tiles, int sample)
{
    double worst = 0.0;
    for (int tl = 0; tl < tiles; tl += tiles / sample) {
        for (int m = 0; m < M; ++m)
            for (int n = 0; n < N; ++n) {
                double s = 0.0, sa = 0.0;
                for (int k = 0; k < K; ++k) {
                    const double p = (double)A[((size_t)tl * M + m) * K + k] * (double)B[((size_t)tl * N + n) * K + k];
                    s += p;
                    sa += std::fabs(p);
                }
                const double e = std::fabs((double)D[((size_t)tl * M + m) * N + n] - s) / (sa > 0 ? sa : 1.0);
                worst = e > worst ? e : worst;
            }
    }
    return worst;
}

template <int N>
static void run(int sms)
{
    const int tiles = 4096, blocks = sms * 4, iters = 32;
    std::vector<float> hA((size_t)tiles * M * K), hB((size_t)tiles * N * K);
    unsigned s = 12301u;
    auto rnd = [&]() {
        s = s * 1664525u + 1013904223u;
        return (float)((s >> 8) * (1.0 / 16777216.0)) * 2.0f - 1.0f;
    };
    for (auto &x : hA) x = rnd();
    for (auto &x : hB) x = rnd();
    float *dA, *dB, *dD1, *dD2;
    ck(cudaMalloc(&dA, hA.size() * 4), "malloc");
    ck(cudaMalloc(&dB, hB.size() * 4), "malloc");
    ck(cudaMalloc(&dD1, (size_t)tiles * M * N * 4), "malloc");
    ck(cudaMalloc(&dD2, (size_t)tiles * M * N * 4), "malloc");
    ck(cudaMemcpy(dA, hA.data(), hA.size() * 4, cudaMemcpyHostToDevice), "copy");
    ck(cudaMemcpy(dB, hB.data(), hB.size() * 4, cudaMemcpyHostToDevice), "copy");
    const size_t smem = (size_t)(2 * M * K + 2 * N * K) * 4;
    ck(cudaFuncSetAttribute(k_tc<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem), "attr");
    int zero = 0;
    ck(cudaMemcpyToSymbol(g_timeout, &zero, sizeof(int)), "symbol");
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    float ms_tc = 0.0f, ms_simt = 0.0f;
    for (int rep = 0; rep < 3; ++rep) {  // the last of three runs is timed
        cudaEventRecord(e0);
        k_tc<N><<<blocks, NT, smem>>>(dA, dB, dD1, tiles, iters);
        cudaEventRecord(e1);
        ck(cudaEventSynchronize(e1), "k_tc");
        cudaEventElapsedTime(&ms_tc, e0, e1);
        cudaEventRecord(e0);
        k_simt<N><<<blocks, NT>>>(dA, dB, dD2, tiles, iters);
        cudaEventRecord(e1);
        ck(cudaEventSynchronize(e1), "k_simt");
        cudaEventElapsedTime(&ms_simt, e0, e1);
    }
    ck(cudaGetLastError(), "launch");
    int timeout = 0;
    ck(cudaMemcpyFromSymbol(&timeout, g_timeout, sizeof(int)), "symbol");
    std::vector<float> D1((size_t)tiles * M * N), D2((size_t)tiles * M * N);
    ck(cudaMemcpy(D1.data(), dD1, D1.size() * 4, cudaMemcpyDeviceToHost), "copy");
    ck(cudaMemcpy(D2.data(), dD2, D2.size() * 4, cudaMemcpyDeviceToHost), "copy");
    const double e_tc = check(hA, hB, D1, N, tiles, 16), e_simt = check(hA, hB, D2, N, tiles, 16);
    const double products = (double)blocks * iters;
    printf("{\"probe\": \"tc_contract\", \"M\": %d, \"N\": %d, \"K\": %d, \"tiles_timed\": %.0f, \"tc_ms\": %.4f, "
           "\"simt_ms\": %.4f, \"tc_ns_per_tile\": %.3f, \"simt_ns_per_tile\": %.3f, \"tc_rel_err\": %.3e, "
           "\"simt_rel_err\": %.3e, \"tc_timeout\": %d}\n",
           M, N, K, products, ms_tc, ms_simt, ms_tc * 1e6 / products, ms_simt * 1e6 / products, e_tc, e_simt, timeout);
    cudaFree(dA);
    cudaFree(dB);
    cudaFree(dD1);
    cudaFree(dD2);
}

int main()
{
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    run<16>(sms);
    run<64>(sms);
    return 0;
}
