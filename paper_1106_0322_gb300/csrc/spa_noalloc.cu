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
#include <cstdio>
#include <mutex>

#include "../../include/spa.h"
#include "spa_device.cuh"
#include "spa_internal.h"

namespace {

constexpr int64_t MAX_N = SPA_NOALLOC_RESAMPLE_MAX_N;
constexpr int64_t SCRATCH_DOUBLES = MAX_N + (MAX_N + 255) / 256 + 1;

// Shared by every call on a device; each GPU that loads the library holds it until exit.
static __device__ __align__(256) double g_resample_scratch[SCRATCH_DOUBLES];

// The array's device address per device, resolved at the first call on that device (with
// it current). The address belongs to the CUDA context that loaded the module, so each
// entry also records that context's unique ID: after a cudaDeviceReset the primary context
// is a new one with a new ID, and the address is resolved again instead of reused.
constexpr int MAX_DEVICES = 64;
struct ScratchSlot {
    unsigned long long ctx_id = 0;
    double* ptr = nullptr;
};
std::mutex g_mu;
ScratchSlot g_scratch[MAX_DEVICES];

typedef CUresult (*CtxGetCurrentFn)(CUcontext*);
typedef CUresult (*CtxGetIdFn)(CUcontext, unsigned long long*);

// The unique ID of the calling thread's current context (0 if it cannot be read). The
// driver entry points are looked up through the runtime, so the library needs no -lcuda.
unsigned long long current_context_id()
{
    static CtxGetCurrentFn get_current = nullptr;
    static CtxGetIdFn get_id = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_current = reinterpret_cast<CtxGetCurrentFn>(p);
        p = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_id = reinterpret_cast<CtxGetIdFn>(p);
    });
    if (!get_current || !get_id) return 0;
    CUcontext ctx = nullptr;
    unsigned long long id = 0;
    if (get_current(&ctx) != CUDA_SUCCESS || !ctx || get_id(ctx, &id) != CUDA_SUCCESS) return 0;
    return id;
}

int cuda_error(const char* what, cudaError_t e)
{
    char msg[256];
    std::snprintf(msg, sizeof(msg), "spa_resample_systematic_noalloc: %s: %s", what, cudaGetErrorString(e));
    spa::set_thread_error(msg);
    return SPA_ECUDA;
}

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
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_error("cudaGetDevice", e);
    if (dev < 0 || dev >= MAX_DEVICES) {
        spa::set_thread_error("spa_resample_systematic_noalloc: device ordinal out of range: ", dev);
        return SPA_ECUDA;
    }
    int major = 0;
    e = cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev);
    if (e != cudaSuccess) return cuda_error("cudaDeviceGetAttribute", e);
    if (major != 10) {
        spa::set_thread_error("spa_resample_systematic_noalloc: the library is built for sm_103a (compute capability "
                              "10.x); this device has major version ",
                              major);
        return SPA_EUNSUPPORTED;
    }
    double* scratch = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_mu);
        const unsigned long long id = current_context_id();
        ScratchSlot& s = g_scratch[dev];
        if (!s.ptr || id == 0 || s.ctx_id != id) {
            // First call on this device in this context: the array's name is only a host
            // stand-in, so resolve its device address (a lookup, not an allocation).
            void* p = nullptr;
            e = cudaGetSymbolAddress(&p, g_resample_scratch);
            if (e != cudaSuccess || !p) return cuda_error("cudaGetSymbolAddress", e);
            s.ptr = static_cast<double*>(p);
            s.ctx_id = id;
        }
        scratch = s.ptr;
    }
    // The kernel writes every scratch entry it later reads, so nothing needs clearing.
    e = spa::launch_resample_index(W_device, N, scratch, idx_device, nullptr, 0, nullptr, u,
                                   static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return cuda_error("kernel launch", e);
    return SPA_OK;
}
