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
double* g_partials_addr[kMaxDevices] = {};

// Device address of the array on the current device, looked up once per
// device with that device current.
cudaError_t partials_on_current_device(double** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_mu);
  if (g_partials_addr[dev] == nullptr) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_sqnorm_partials);
    if (e != cudaSuccess) return e;
    g_partials_addr[dev] = static_cast<double*>(p);
  }
  *out = g_partials_addr[dev];
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
