// planc_sqnorm_noalloc: ||X||^2 without any device allocation.
//
// Some callers cannot allocate device memory at the moment they need this
// reduction: code that runs while a CUDA stream is being captured into a graph
// (allocation calls are not allowed there), runtimes that hand out every byte
// of device memory from their own fixed pool, and latency-critical loops that
// must not enter the allocator.  They also cannot create a planc context,
// whose workspace is allocated in planc_init.  This entry point gives them the
// same two-kernel reduction as planc_sqnorm, with its per-block partial sums
// kept in a statically sized device array that is part of the library image.
#include <mutex>

#include "internal.h"

namespace {

// Per-block FP64 partial sums.  The array exists once per device that loads
// the library and lives until the process exits.
constexpr int kMaxPartials = 1024;  // 8 KiB
static __device__ __align__(256) double g_sqnorm_partials[kMaxPartials];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
// the array's device address per device, with the CUDA context it was looked
// up in: a context that is torn down and created again (cudaDeviceReset, a
// primary-context reset) loads the library's module anew, and the array may
// then sit elsewhere, so an address is reused only inside its own context
struct Cached {
  void* ctx;
  double* addr;
};
Cached g_cache[kMaxDevices] = {};

// cuCtxGetCurrent through the runtime's driver entry point (no link-time
// dependency on the driver library)
using CtxGetCurrentFn = int (*)(void**);
CtxGetCurrentFn ctx_get_current() {
  static CtxGetCurrentFn fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<CtxGetCurrentFn>(f);
  });
  return fn;
}

// Device address of the array in the current device's current context,
// looked up with that device current the first time it is needed there.
cudaError_t partials_on_current_device(double** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  CtxGetCurrentFn get = ctx_get_current();
  void* ctx = nullptr;
  if (get == nullptr || get(&ctx) != 0) return cudaErrorInitializationError;
  std::lock_guard<std::mutex> lock(g_mu);
  if (ctx == nullptr || g_cache[dev].addr == nullptr || g_cache[dev].ctx != ctx) {
    void* p = nullptr;
    // (with no context current on this thread yet, the lookup makes the
    // device's primary context current, and the handle is read after it)
    e = cudaGetSymbolAddress(&p, g_sqnorm_partials);
    if (e != cudaSuccess) return e;
    if (ctx == nullptr && (get(&ctx) != 0 || ctx == nullptr)) return cudaErrorInitializationError;
    g_cache[dev].ctx = ctx;
    g_cache[dev].addr = static_cast<double*>(p);
  }
  *out = g_cache[dev].addr;
  return cudaSuccess;
}

}  // namespace

extern "C" planc_status_t planc_sqnorm_noalloc(planc_dtype_t x_dtype, const void* X, int64_t n,
                                               double* alpha, void* cuda_stream) {
  if (!X || !alpha) return PLANC_E_INVALID;
  if ((int)x_dtype < 0 || (int)x_dtype > 3) return PLANC_E_DTYPE;
  if (n < 1 || n > (1LL << 40)) return PLANC_E_SHAPE;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return PLANC_E_CUDA;
  const int nblk = planc::sqnorm_blocks(n, sms);
  if (nblk > kMaxPartials) return PLANC_E_SHAPE;  // more partials than the array holds
  double* part = nullptr;
  if (partials_on_current_device(&part) != cudaSuccess) return PLANC_E_CUDA;
  // every block overwrites its own partial before the final sum reads it,
  // so the array needs no clearing between calls
  cudaError_t e = planc::launch_sqnorm(x_dtype, X, n, part, nblk, alpha,
                                       static_cast<cudaStream_t>(cuda_stream));
  return e == cudaSuccess ? PLANC_OK : PLANC_E_CUDA;
}
