// Allocation-free FP64 moment sums (cdf_moment_sums_static).
//
// Some callers cannot call cudaMalloc once they are running: real-time loops
// that forbid allocation after start-up, plug-ins inside a host application
// that owns all device memory through its own pool, and processes under a
// fixed device-memory quota where a late allocation can fail or fragment the
// pool.  For them this entry point runs the same two-pass reduction as
// cdf_lb_mass with its block partials in a file-scope device array instead of
// handle-owned scratch; the caller passes the input fields and the output.
// The first call on each device (and again after that device's context was
// torn down and recreated) does a set-up that may load kernel code, which can
// allocate: make it at start-up, before the allocation-free phase and before
// any stream capture.
#include <cuda_runtime.h>

#include <mutex>

#include "../../include/cdf_lb.h"
#include "lb_internal.h"

namespace cdflb {
namespace {

// Block partials: kReduceBlocks blocks x at most 3 * kMaxM + 5 sums, i.e.
// 304 x 17 doubles = 41,344 bytes.  Every GPU that loads the library holds this
// array until the process exits.  Every call writes each slot it later reads,
// so nothing has to be cleared between calls; calls that overlap on the GPU
// (two streams, or two threads) share it and race.
constexpr int kStaticSlots = kReduceBlocks * (3 * kMaxM + 5);
static __device__ __align__(256) double g_static_partials[kStaticSlots];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mu;
// Per device: the array's device address and the context it was looked up in.
// A context that was torn down and recreated (cudaDeviceReset, or a primary
// context released and retained again) has a new id, so the set-up runs again.
struct Setup {
    unsigned long long ctx_id;
    double *partials;
};
Setup g_setup[kMaxDevices] = {};

// The driver's cuCtxGetCurrent and cuCtxGetId, looked up once through the
// runtime (no link-time dependency on libcuda).
typedef int (*CtxGetCurrentFn)(void **);
typedef int (*CtxGetIdFn)(void *, unsigned long long *);
CtxGetCurrentFn g_ctx_get_current = nullptr;
CtxGetIdFn g_ctx_get_id = nullptr;
std::once_flag g_driver_once;

void find_driver_entry_points() {
    void *f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
        g_ctx_get_current = reinterpret_cast<CtxGetCurrentFn>(f);
    f = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
        g_ctx_get_id = reinterpret_cast<CtxGetIdFn>(f);
}

// Id of the calling thread's current context; 0 if there is none yet.
unsigned long long current_context_id() {
    std::call_once(g_driver_once, find_driver_entry_points);
    void *ctx = nullptr;
    unsigned long long id = 0;
    if (!g_ctx_get_current || !g_ctx_get_id || g_ctx_get_current(&ctx) != 0 || !ctx) return 0;
    if (g_ctx_get_id(ctx, &id) != 0) return 0;
    return id;
}

}  // namespace
}  // namespace cdflb

using namespace cdflb;

extern "C" cdf_status cdf_moment_sums_static(const float *dev_fields, const float *dev_fields_old, int nx,
                                             int ny, int m, double *dev_out, void *stream) {
    if (!dev_fields || !dev_out) return report_error(CDF_EINVAL, "dev_fields and dev_out must not be NULL");
    if (nx < 1 || ny < 1) return report_error(CDF_EINVAL, "grid must be at least 1 x 1");
    if ((long long)nx * ny >= (1LL << 31)) return report_error(CDF_EINVAL, "grid too large: nx * ny must be below 2^31");
    if (m < 1 || m > CDF_MAX_M)
        return report_error(CDF_EINVAL, "m must be in [1, 4]: the static scratch holds 17 sums per block");
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) return report_error(CDF_ECUDA, "no current CUDA device");
    if (dev < 0 || dev >= kMaxDevices) return report_error(CDF_EINVAL, "device index above 63");
    double *partials = nullptr;
    {
        // Set-up, once per device and context, with that device current: the
        // array's name is a host-side stand-in, so its device address is looked
        // up here; the reduction kernels' code is loaded here too, so that no
        // later call loads (and allocates) it lazily.
        std::lock_guard<std::mutex> lk(g_setup_mu);
        const unsigned long long ctx = current_context_id();
        if (!g_setup[dev].partials || ctx == 0 || ctx != g_setup[dev].ctx_id) {
            void *p = nullptr;
            cudaError_t e = cudaGetSymbolAddress(&p, g_static_partials);
            if (e != cudaSuccess || !p)
                return report_error(CDF_ECUDA, "cudaGetSymbolAddress of the static scratch failed");
            e = preload_reduce_kernels();
            if (e != cudaSuccess) return report_error(CDF_ECUDA, "loading the reduction kernels failed");
            g_setup[dev].partials = static_cast<double *>(p);
            g_setup[dev].ctx_id = current_context_id();  // the look-up made a context current
        }
        partials = g_setup[dev].partials;
    }
    cudaError_t e = launch_reduce(dev_fields, dev_fields_old, nx, ny, nx, (long long)nx * ny, m, partials,
                                  dev_out, static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return report_error(CDF_ECUDA, "reduction launch failed");
    return CDF_OK;
}
