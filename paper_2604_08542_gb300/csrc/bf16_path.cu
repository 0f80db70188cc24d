// BF16 tensor-core path (tcgen05 + TMA) of the test-time-training layer.
#include "ttt_internal.h"

namespace scal3r {

bool bf16_shape_supported(int D, int F) { return D == 64 && F == 128; }

cudaError_t launch_bf16_sweep(const Params&, const WorkItem*, int, int, const void*, cudaStream_t) {
  return cudaErrorNotSupported;
}

cudaError_t launch_bf16_bsweep(const Params&, const WorkItem*, int, int, const void*, cudaStream_t) {
  return cudaErrorNotSupported;
}

}  // namespace scal3r
