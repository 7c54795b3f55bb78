// Tensor-core bound path (placeholder until the tcgen05 kernel lands).
#include "internal.cuh"

namespace isx {

bool bf16_supported(isx_inr) { return false; }

isx_status bound_bf16(isx_inr, const CellSource&, int64_t, isx_bound_mode, int, float*, float*, cudaStream_t) {
  set_error("BF16 tensor-core propagation is not built yet");
  return ISX_ERR_UNSUPPORTED;
}

}  // namespace isx
