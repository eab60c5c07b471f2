// The fused per-time-step kernel: load 98 populations through the AA index map of
// the step's parity, collide in registers, store 98 populations in place.
#pragma once

#include "lbm_internal.h"

namespace lbm {

// MINB = resident 128-thread blocks per SM the register budget is sized for:
// 3 -> at most 170 registers (no spills), 4 -> at most 128 (a few spilled words).
template <int PARITY, typename S, bool HELD, int MINB>
__global__ void __launch_bounds__(128, MINB) k_step(const DomainConst P, S* __restrict__ pop,
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
  store_cell<PARITY, S>(P, pop, c, d);
}

template <typename S, int MINB>
void launch_variant(const DomainConst& P, int parity, S* p, const float* ghost, unsigned* flag,
                    dim3 grid, dim3 block, cudaStream_t s) {
  if (P.bc_x) {
    if (parity) k_step<1, S, true, MINB><<<grid, block, 0, s>>>(P, p, ghost, flag);
    else k_step<0, S, true, MINB><<<grid, block, 0, s>>>(P, p, ghost, flag);
  } else {
    if (parity) k_step<1, S, false, MINB><<<grid, block, 0, s>>>(P, p, ghost, flag);
    else k_step<0, S, false, MINB><<<grid, block, 0, s>>>(P, p, ghost, flag);
  }
}

// variant 0: register budget for 3 blocks of 128 per SM; 1: for 4 blocks.
template <typename S>
cudaError_t launch_step_t(const DomainConst& P, int parity, void* pop, const float* ghost,
                          unsigned* flag, int block_x, int variant, cudaStream_t s) {
  if (block_x < 32 || block_x > 128 || (block_x & 31)) return cudaErrorInvalidConfiguration;
  const dim3 block(block_x);
  const dim3 grid((P.nx + block_x - 1) / block_x, P.ny, P.nz);
  S* p = static_cast<S*>(pop);
  if (variant) launch_variant<S, 4>(P, parity, p, ghost, flag, grid, block, s);
  else launch_variant<S, 3>(P, parity, p, ghost, flag, grid, block, s);
  return cudaGetLastError();
}

}  // namespace lbm
