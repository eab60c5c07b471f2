// Fused step kernels for __half population storage.
#include "step_impl.cuh"

namespace lbm {
cudaError_t launch_step_f16(const DomainConst& P, int parity, void* pop, const float* ghost,
                          unsigned* flag, int block_x, int variant, cudaStream_t s) {
  return launch_step_t<__half>(P, parity, pop, ghost, flag, block_x, variant, s);
}
}  // namespace lbm
