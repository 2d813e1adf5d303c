// Partial MTTKRP on the tcgen05 tensor cores (placeholder until the tensor
// core path is enabled: every shape is routed to the CUDA-core kernels).
#include "internal.h"

namespace planc {

bool pm_tc_eligible(planc_dtype_t, bool, int64_t, int64_t, int) { return false; }

size_t pm_tc_workspace_bytes(planc_dtype_t, bool, int64_t, int64_t, int, int) { return 0; }

cudaError_t launch_pm_tc(planc_dtype_t, const void*, int64_t, int64_t, bool, const KrpHost&, int,
                         void*, bool, void*, size_t, int*, int, cudaStream_t) {
  return cudaErrorNotSupported;
}

}  // namespace planc
