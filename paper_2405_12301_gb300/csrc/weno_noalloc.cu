// weno_noalloc.cu -- conservation sums without any device allocation.
//
// weno_sums needs a handle, and a handle owns cudaMalloc'ed scratch.  This
// entry point runs the same two fixed-order reduction kernels, but keeps their
// per-block partial sums in a file-scope device array that is part of the
// loaded library, so the call itself never allocates.
#include <mutex>
#include <string>

#include "../../include/weno_gb300.h"
#include "weno_internal.h"

namespace wg {
void set_thread_error(const std::string &msg);
}

namespace {

constexpr int kMaxFields = 5;
constexpr int kMaxBlocks = 1024;  // the reduction never uses more blocks (sums_blocks caps it)

// 1024 blocks x 5 fields x 8 bytes = 40 KiB, resident on every device that
// loads the library until the process exits.  Every slot a call reads is
// written earlier in the same call, so nothing needs clearing between calls.
static __device__ __align__(256) double g_partials[kMaxBlocks * kMaxFields];

constexpr int kMaxDevices = 64;
double *g_partials_addr[kMaxDevices] = {};
std::mutex g_setup_mutex;

int reject(int code, const char *msg)
{
    wg::set_thread_error(msg);
    return code;
}

}  // namespace

extern "C" int weno_sums_noalloc(const double *U, int32_t nf, int64_t ncells, double *sums_dev, void *cuda_stream)
{
    if (!U || !sums_dev) return reject(WENO_ERR_ARG, "weno_sums_noalloc: null U or sums_dev");
    if (nf < 1 || nf > kMaxFields)
        return reject(WENO_ERR_ARG, "weno_sums_noalloc: nf must be 1..5 (scratch holds 1024 x 5 partial sums)");
    if (ncells < 1 || ncells > (int64_t(1) << 40))
        return reject(WENO_ERR_ARG, "weno_sums_noalloc: ncells must be 1..2^40");
    const int nblocks = wg::sums_blocks(ncells);
    if (nblocks > kMaxBlocks) return reject(WENO_ERR_ARG, "weno_sums_noalloc: too many partial sums for the scratch");
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return reject(WENO_ERR_CUDA, "weno_sums_noalloc: cudaGetDevice failed");
    if (dev < 0 || dev >= kMaxDevices) return reject(WENO_ERR_UNSUPPORTED, "weno_sums_noalloc: device index above 63");
    double *partials = nullptr;
    {
        // one-time set-up per device, with that device current: the device
        // address of the scratch array (its host-side name is not one)
        std::lock_guard<std::mutex> lock(g_setup_mutex);
        if (!g_partials_addr[dev]) {
            void *p = nullptr;
            const cudaError_t e = cudaGetSymbolAddress(&p, g_partials);
            if (e != cudaSuccess)
                return reject(WENO_ERR_CUDA,
                              (std::string("weno_sums_noalloc: cudaGetSymbolAddress: ") + cudaGetErrorString(e)).c_str());
            g_partials_addr[dev] = static_cast<double *>(p);
        }
        partials = g_partials_addr[dev];
    }
    const cudaError_t e =
        wg::launch_sums(U, nf, (long long)ncells, partials, nblocks, sums_dev, (cudaStream_t)cuda_stream);
    if (e != cudaSuccess)
        return reject(WENO_ERR_CUDA, (std::string("weno_sums_noalloc: launch: ") + cudaGetErrorString(e)).c_str());
    return WENO_OK;
}
