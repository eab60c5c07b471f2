// Shared-memory-staged variants of the fused step for __nv_bfloat16 population storage.
#include "step_staged.cuh"

namespace lbm {
cudaError_t staged_prepare_bf16(const DomainConst& P, int variant, int* grid) {
  return staged_prepare_t<__nv_bfloat16>(P, variant, grid);
}
cudaError_t launch_step_staged_bf16(const DomainConst& P, int parity, void* pop, unsigned* flag,
                                    int variant, int grid, int skip_first, cudaStream_t s) {
  return staged_launch_t<__nv_bfloat16>(P, parity, pop, flag, variant, grid, skip_first, s);
}
}  // namespace lbm
