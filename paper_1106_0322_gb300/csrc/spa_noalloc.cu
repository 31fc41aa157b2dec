// spa_noalloc.cu -- systematic resampling for callers that cannot allocate device memory.
//
// spa_resample_systematic() allocates its device buffers on every call. Some callers
// cannot do that: a process whose device memory is all held by another allocator (a
// framework's caching pool that has reserved the GPU), code on a latency-critical path
// where cudaMalloc / cudaFree would synchronise the device, and services that must not
// grow their device footprint after start-up. spa_resample_systematic_noalloc() is for
// them. The caller passes device buffers for the weights and the ancestor indices. The
// only scratch the kernel needs -- the blocked cumulative sum of the weights and one
// carry per 256-block -- lives in the fixed file-scope device array below, so the call
// allocates nothing.
#include <mutex>

#include "../../include/spa.h"
#include "spa_device.cuh"
#include "spa_internal.h"

namespace {

constexpr int64_t MAX_N = SPA_NOALLOC_RESAMPLE_MAX_N;
constexpr int64_t SCRATCH_DOUBLES = MAX_N + (MAX_N + 255) / 256 + 1;

// Shared by every call on a device; each GPU that loads the library holds it until exit.
static __device__ __align__(256) double g_resample_scratch[SCRATCH_DOUBLES];

constexpr int MAX_DEVICES = 64;
std::mutex g_mu;
double* g_scratch[MAX_DEVICES] = {nullptr};

}  // namespace

extern "C" int spa_resample_systematic_noalloc(const double* W_device, int64_t N, double u, int32_t* idx_device,
                                               void* stream)
{
    if (!W_device || !idx_device) {
        spa::set_thread_error("spa_resample_systematic_noalloc: NULL device buffer");
        return SPA_EINVAL;
    }
    if (N < 1 || N > MAX_N) {
        spa::set_thread_error("spa_resample_systematic_noalloc: N must be in [1, SPA_NOALLOC_RESAMPLE_MAX_N]; got N = ",
                              N);
        return SPA_EINVAL;
    }
    if (!(u >= 0.0 && u < 1.0)) {
        spa::set_thread_error("spa_resample_systematic_noalloc: u must be in [0, 1)");
        return SPA_EINVAL;
    }
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= MAX_DEVICES) {
        spa::set_thread_error("spa_resample_systematic_noalloc: no usable current device");
        return SPA_ECUDA;
    }
    double* scratch = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_mu);
        if (!g_scratch[dev]) {
            // First call on this device (which is current): the array's name is only a host
            // stand-in, so resolve its device address once and keep it.
            void* p = nullptr;
            if (cudaGetSymbolAddress(&p, g_resample_scratch) != cudaSuccess || !p) {
                spa::set_thread_error("spa_resample_systematic_noalloc: cudaGetSymbolAddress failed");
                return SPA_ECUDA;
            }
            g_scratch[dev] = static_cast<double*>(p);
        }
        scratch = g_scratch[dev];
    }
    // The kernel writes every scratch entry it later reads, so nothing needs clearing.
    const cudaError_t e = spa::launch_resample_index(W_device, N, scratch, idx_device, nullptr, 0, nullptr, u,
                                                     static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) {
        spa::set_thread_error("spa_resample_systematic_noalloc: kernel launch failed");
        return SPA_ECUDA;
    }
    return SPA_OK;
}
