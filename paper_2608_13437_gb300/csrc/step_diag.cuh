// The fused step with the diagnostics of the state it reads (Sec. 3.2, Eq. 7): the
// same cell update as k_step, and from the same registers, one diagnostic record per
// warp (sums, extrema, non-finite count of its 32 cells) plus u and mu_local into a
// 4-float-per-cell field for the velocity-gradient pass. No separate pass over the
// populations is needed.
#pragma once

#include "diag_device.cuh"
#include "lbm_internal.h"
#include "step_impl.cuh"

namespace lbm {

static_assert(kDiagRecFloats == kDiagRecWords, "warp record size");

// ROWS: whole-tile rows (periodic x, nx a multiple of 32) take the plain kernel's
// warp-uniform tile addressing and its L2 prefetch; every warp is then whole. ESO: the
// esoteric twist on whole-tile rows (the other forms take it from P.eso).
template <int PARITY, typename S, bool HELD, bool SR, bool ROWS, bool ESO = false>
__global__ void __launch_bounds__(128, 3) k_step_diag(const DomainConst P, S* __restrict__ pop,
                                                      const float* __restrict__ ghost,
                                                      unsigned* __restrict__ flag,
                                                      float* __restrict__ ufield,
                                                      float* __restrict__ rec) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  DiagAcc acc;
  diag_zero(acc);
  const int lane = threadIdx.x & (kTile - 1);
  // no early return: every lane takes part in the warp reduction
  if (ROWS ? (x - lane < P.nx) : (x < P.nx)) {
    float d[kF][kQ];
    CellDiag cd;
    if constexpr (ROWS) {
      const WarpTiles T = warp_tiles(P, x - lane, blockIdx.y, blockIdx.z);
      if (P.pf_tiles > 0 && lane == 0) prefetch_future<PARITY, S, ESO>(P, pop, T.t);
      load_cell_rows<PARITY, S, ESO>(P, pop, T, lane, d);
      if (P.collide) {
        const float probe = collide_cell<false, true>(P, d, nullptr, &cd);
        if (!isfinite(probe)) atomicOr(flag, 1u);
      } else {
        SensorOut so;
        collide_cell<true, true>(P, d, &so, &cd);
      }
      store_cell_rows<PARITY, S, SR, ESO>(P, pop, T, lane, d);
    } else {
      const CellIndex c = make_index(P, x, blockIdx.y, blockIdx.z);
      load_cell<PARITY, HELD, S>(P, pop, ghost, c, d);
      if (P.collide) {
        const float probe = collide_cell<false, true>(P, d, nullptr, &cd);
        if (!isfinite(probe)) atomicOr(flag, 1u);
      } else {
        SensorOut so;
        collide_cell<true, true>(P, d, &so, &cd);
      }
      store_cell<PARITY, S, SR>(P, pop, c, d);
    }
    diag_add_cell(P, cd, acc);
    const long long n = P.ncell;
    const long long cell = x + (long long)P.nx * (blockIdx.y + (long long)P.ny * blockIdx.z);
    ufield[cell] = cd.u[0];
    ufield[n + cell] = cd.u[1];
    ufield[2 * n + cell] = cd.u[2];
    ufield[3 * n + cell] = cd.mu_T;
  }
  const long long blk = ((long long)blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
  diag_warp_reduce_store(acc, rec + (blk * (blockDim.x >> 5) + (threadIdx.x >> 5)) * kDiagRecWords);
}

template <typename S, bool SR>
void launch_step_diag_forms(const DomainConst& P, int parity, S* p, const float* ghost,
                            unsigned* flag, float* ufield, float* rec, dim3 grid, dim3 block,
                            cudaStream_t s) {
  if (P.bc_x) {
    if (parity) k_step_diag<1, S, true, SR, false><<<grid, block, 0, s>>>(P, p, ghost, flag, ufield, rec);
    else k_step_diag<0, S, true, SR, false><<<grid, block, 0, s>>>(P, p, ghost, flag, ufield, rec);
  } else if (P.nx % kTile == 0 && P.eso) {
    if (parity) k_step_diag<1, S, false, SR, true, true><<<grid, block, 0, s>>>(P, p, ghost, flag, ufield, rec);
    else k_step_diag<0, S, false, SR, true, true><<<grid, block, 0, s>>>(P, p, ghost, flag, ufield, rec);
  } else if (P.nx % kTile == 0) {
    if (parity) k_step_diag<1, S, false, SR, true><<<grid, block, 0, s>>>(P, p, ghost, flag, ufield, rec);
    else k_step_diag<0, S, false, SR, true><<<grid, block, 0, s>>>(P, p, ghost, flag, ufield, rec);
  } else {
    if (parity) k_step_diag<1, S, false, SR, false><<<grid, block, 0, s>>>(P, p, ghost, flag, ufield, rec);
    else k_step_diag<0, S, false, SR, false><<<grid, block, 0, s>>>(P, p, ghost, flag, ufield, rec);
  }
}

template <typename S>
cudaError_t launch_step_diag_t(const DomainConst& P, int parity, void* pop, const float* ghost,
                               unsigned* flag, float* ufield, float* rec, int block_x,
                               cudaStream_t s) {
  if (block_x < 32 || block_x > 128 || (block_x & 31)) return cudaErrorInvalidConfiguration;
  const dim3 block(block_x);
  const dim3 grid((P.nx + block_x - 1) / block_x, P.ny, P.nz);
  S* p = static_cast<S*>(pop);
  if constexpr (!std::is_same<S, float>::value) {
    if (P.sround) {
      launch_step_diag_forms<S, true>(P, parity, p, ghost, flag, ufield, rec, grid, block, s);
      return cudaGetLastError();
    }
  }
  launch_step_diag_forms<S, false>(P, parity, p, ghost, flag, ufield, rec, grid, block, s);
  return cudaGetLastError();
}

}  // namespace lbm
