// pipe_peaks.cu -- throughput of the GB300 arithmetic pipes the roofline of
// this library's kernels is stated against: FP32 FFMA, packed FFMA2 (f32x2),
// FP64 DFMA and the FP64 <-> FP32 conversions.
//
// Each kernel runs long dependency-free streams of one instruction kind (8
// independent accumulators per thread) on every SM, launched as exactly one
// wave (as many CTAs per SM as can be resident, at most 8), and every CTA reads
// the SM clock around its loop, so the result is in operations per clock per
// SM, independent of the clock the GPU ran at.  The host also times the whole
// launch with CUDA events, which gives operations per second.  Output: one
// JSON line per pipe.
#include <cstdio>
#include <cstdlib>
#include <cuda_runtime.h>

constexpr int NT = 256;
constexpr int ACC = 8;

__device__ unsigned long long g_cycles[4096];

template <int KIND>
__global__ void __launch_bounds__(NT) k_pipe(int iters, float seed, float *sink)
{
    float a[ACC];
    float2 p[ACC];
    double d[ACC];
#pragma unroll
    for (int k = 0; k < ACC; ++k) {
        a[k] = seed + 0.001f * (threadIdx.x + k);
        p[k] = make_float2(a[k], a[k] + 0.5f);
        d[k] = (double)a[k];
    }
    const float m = 0.9999f, c = 1e-4f;
    const float2 m2 = make_float2(m, m), c2 = make_float2(c, c);
    __syncthreads();
    const unsigned long long t0 = clock64();
#pragma unroll 1
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int u = 0; u < 4; ++u) {
#pragma unroll
            for (int k = 0; k < ACC; ++k) {
                if (KIND == 0) a[k] = fmaf(a[k], m, c);
                if (KIND == 1) p[k] = __ffma2_rn(p[k], m2, c2);
                if (KIND == 2) d[k] = fma(d[k], 0.9999, 1e-4);
                if (KIND == 4) a[k] = __double2float_rn((double)a[k] * 0.9999);
            }
        }
    }
    __syncthreads();
    const unsigned long long t1 = clock64();
    if (threadIdx.x == 0) g_cycles[blockIdx.x] = t1 - t0;
    float s = 0.0f;
#pragma unroll
    for (int k = 0; k < ACC; ++k) s += a[k] + p[k].x + p[k].y + (float)d[k];
    if (s == 12345.678f) sink[threadIdx.x] = s;  // keeps the streams live
}

template <int KIND>
static void run(const char *name, int ops_per_inst, int blocks_per_sm, int iters)
{
    int dev = 0, sms = 0, resident = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&resident, k_pipe<KIND>, NT, 0);
    if (resident < blocks_per_sm) blocks_per_sm = resident;
    if (blocks_per_sm < 1) return;
    const int blocks = sms * blocks_per_sm;
    if (blocks > 4096) return;
    float *sink = nullptr;
    cudaMalloc(&sink, NT * sizeof(float));
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    k_pipe<KIND><<<blocks, NT>>>(iters / 10, 1.0f, sink);  // warm-up
    cudaEventRecord(e0);
    k_pipe<KIND><<<blocks, NT>>>(iters, 1.0f, sink);
    cudaEventRecord(e1);
    cudaEventSynchronize(e1);
    float ms = 0.0f;
    cudaEventElapsedTime(&ms, e0, e1);
    unsigned long long cyc[4096];
    cudaMemcpyFromSymbol(cyc, g_cycles, sizeof(unsigned long long) * blocks);
    double cmax = 0.0, csum = 0.0;
    for (int b = 0; b < blocks; ++b) {
        csum += (double)cyc[b];
        cmax = cyc[b] > cmax ? (double)cyc[b] : cmax;
    }
    const double insts = (double)blocks * NT * iters * 4 * ACC;  // thread-instructions
    const double per_sm = insts / sms;
    const cudaError_t err = cudaGetLastError();
    printf("{\"pipe\": \"%s\", \"thread_ops_per_clk_per_sm\": %.2f, \"flop_per_op\": %d, "
           "\"tops_per_s\": %.3f, \"ms\": %.3f, \"sms\": %d, \"ctas_per_sm\": %d, \"clock_mhz_implied\": %.0f, "
           "\"status\": \"%s\"}\n",
           name, per_sm / cmax, ops_per_inst, insts / (ms * 1e-3) / 1e12, ms, sms, blocks_per_sm,
           cmax / (ms * 1e-3) / 1e6, cudaGetErrorString(err));
    cudaFree(sink);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
}

int main()
{
    run<0>("ffma_f32", 2, 8, 4096);
    run<1>("ffma2_f32x2 (one instruction, two FMAs)", 4, 8, 4096);
    run<2>("dfma_f64", 2, 8, 512);
    run<4>("cvt f32->f64, DMUL, cvt f64->f32 (one op = the three)", 1, 8, 256);
    return 0;
}
