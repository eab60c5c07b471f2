// The fused per-time-step kernel: load 98 populations through the AA index map of
// the step's parity, collide in registers, store 98 populations in place.
#pragma once

#include "lbm_internal.h"

namespace lbm {

template <int PARITY, typename S, bool HELD>
__global__ void __launch_bounds__(256) k_step(const DomainConst P, S* __restrict__ pop,
                                              const float* __restrict__ ghost,
                                              unsigned* __restrict__ flag) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  if (x >= P.nx) return;
  const CellIndex c = make_index(P, x, blockIdx.y, blockIdx.z);
  float d[kF][kQ];
  load_cell<PARITY, HELD, S>(P, pop, ghost, c, d);
  if (P.collide) {
    const float probe = collide_cell<false>(P, d, nullptr);
    if (!isfinite(probe)) atomicOr(flag, 1u);
  }
#pragma unroll
  for (int k = 0; k < kF; ++k) store_field<PARITY, S>(P, pop, c, k, d[k]);
}

template <typename S>
cudaError_t launch_step_t(const DomainConst& P, int parity, void* pop, const float* ghost,
                          unsigned* flag, int block_x, cudaStream_t s) {
  const dim3 block(block_x);
  const dim3 grid((P.nx + block_x - 1) / block_x, P.ny, P.nz);
  S* p = static_cast<S*>(pop);
  if (P.bc_x) {
    if (parity) k_step<1, S, true><<<grid, block, 0, s>>>(P, p, ghost, flag);
    else k_step<0, S, true><<<grid, block, 0, s>>>(P, p, ghost, flag);
  } else {
    if (parity) k_step<1, S, false><<<grid, block, 0, s>>>(P, p, ghost, flag);
    else k_step<0, S, false><<<grid, block, 0, s>>>(P, p, ghost, flag);
  }
  return cudaGetLastError();
}

}  // namespace lbm
