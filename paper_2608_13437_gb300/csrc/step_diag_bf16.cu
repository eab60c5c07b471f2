// Diagnostic variant of the fused step for __nv_bfloat16 population storage.
#include "step_diag.cuh"

namespace lbm {
cudaError_t launch_step_diag_bf16(const DomainConst& P, int parity, void* pop, const float* ghost,
                                  unsigned* flag, float* ufield, float* rec, int block_x,
                                  cudaStream_t s) {
  return launch_step_diag_t<__nv_bfloat16>(P, parity, pop, ghost, flag, ufield, rec, block_x, s);
}
}  // namespace lbm
