// Shared-memory-staged variants of the fused step for float population storage.
#include "step_staged.cuh"

namespace lbm {
cudaError_t staged_prepare_f32(const DomainConst& P, int variant, int* grid) {
  return staged_prepare_t<float>(P, variant, grid);
}
cudaError_t launch_step_staged_f32(const DomainConst& P, int parity, void* pop, unsigned* flag,
                                   int variant, int grid, int skip_first, cudaStream_t s) {
  return staged_launch_t<float>(P, parity, pop, flag, variant, grid, skip_first, s);
}
}  // namespace lbm
