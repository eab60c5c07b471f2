// The fused per-time-step kernel: load 98 populations through the AA index map of
// the step's parity, collide in registers, store 98 populations in place.
#pragma once

#include "lbm_internal.h"

namespace lbm {

// Rows of whole tiles (nx a multiple of 32, x periodic): a warp's 32 cells are one
// tile, and the tiles holding its neighbours are the same for all lanes (only the two
// edge lanes of an x neighbour fall into the next tile). Their indices are computed
// once per warp, so every population access is a warp-uniform tile base plus the
// lane's offset.
struct WarpTiles {
  long long t, xm, xp, ym, yp, zm, zp;
};

__device__ __forceinline__ WarpTiles warp_tiles(const DomainConst& P, int x0, int y, int z) {
  const long long tpr = P.nx / kTile, tpp = tpr * P.ny;  // tiles per row, per plane
  WarpTiles T;
  T.t = x0 / kTile + tpr * ((long long)y + (long long)P.ny * z);
  T.xm = x0 > 0 ? T.t - 1 : T.t + tpr - 1;
  T.xp = x0 + kTile < P.nx ? T.t + 1 : T.t - (tpr - 1);
  T.ym = y > 0 ? T.t - tpr : T.t + (tpp - tpr);
  T.yp = y + 1 < P.ny ? T.t + tpr : T.t - (tpp - tpr);
  T.zm = z > 0 ? T.t - tpp : T.t + (P.ntile - tpp);
  T.zp = z + 1 < P.nz ? T.t + tpp : T.t - (P.ntile - tpp);
  return T;
}

// Tile and lane of the cell one lattice link from this lane's cell along direction i
// (i = 1..6: +x, -x, +y, -y, +z, -z), forward (toward = +1) or backward (-1).
__device__ __forceinline__ void link_tile(const WarpTiles& T, int i, int toward, int lane,
                                          long long& tile, int& ln) {
  const int axis = (i - 1) >> 1;
  const int s = ((i & 1) ? 1 : -1) * toward;  // +1: toward +axis
  ln = lane;
  if (axis == 0) {
    if (s > 0) {
      tile = lane < kTile - 1 ? T.t : T.xp;
      ln = lane < kTile - 1 ? lane + 1 : 0;
    } else {
      tile = lane > 0 ? T.t : T.xm;
      ln = lane > 0 ? lane - 1 : kTile - 1;
    }
  } else if (axis == 1) {
    tile = s > 0 ? T.yp : T.ym;
  } else {
    tile = s > 0 ? T.zp : T.zm;
  }
}

// Bulk prefetch of `bytes` (a multiple of 16, 16-byte aligned) into L2.
__device__ __forceinline__ void l2_prefetch(const void* p, unsigned bytes) {
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(bytes) : "memory");
}

// Whole-tile rows: tiles are processed roughly in index order, so the warp on tile t
// asks L2 for the slot blocks that the warp on tile w = t + P.pf_tiles will read, and
// that warp later finds them in L2 instead of waiting on DRAM. Even steps read the 7
// slots of the own tile. Odd steps read slots 0-2 of the own tile, slot 4 of the tile
// a row before, slot 3 of the tile a row after, slot 6 of the tile a plane before and
// slot 5 of the tile a plane after; prefetching slots 0-4 of tile w (its slots 3 and 4
// serve the warps a row before and after w) and the two plane slots covers them.
// Under the esoteric twist every step reads, of tile w, the slots of its own warp and
// those the warps a tile and a row before it take from w, and the z slot (6 even, 5
// odd) of the tile a plane after w; the z slot of w itself was read a plane earlier.
// Only addresses inside the buffer are prefetched (periodic wrap along z); results
// do not depend on the prefetch.
template <int PARITY, typename S, bool ESO = false>
__device__ __forceinline__ void prefetch_future(const DomainConst& P, const S* pop, long long t) {
  const long long w = t + P.pf_tiles;
  if (w >= P.ntile) return;
  constexpr unsigned kSlotBytes = kSlotElems * sizeof(S);
  if constexpr (ESO) {
    const long long tpp = (long long)(P.nx / kTile) * P.ny;
    const long long zp = w + tpp < P.ntile ? w + tpp : w + tpp - P.ntile;
    if (PARITY == 0) {
      l2_prefetch(pop + w * kTileElems, 6 * kSlotBytes);
    } else {
      l2_prefetch(pop + w * kTileElems, 5 * kSlotBytes);
      l2_prefetch(pop + w * kTileElems + 6 * kSlotElems, kSlotBytes);
    }
    l2_prefetch(pop + zp * kTileElems + (PARITY ? 5 : 6) * kSlotElems, kSlotBytes);
  } else if (PARITY == 0) {
    l2_prefetch(pop + w * kTileElems, kQ * kSlotBytes);
  } else {
    const long long tpp = (long long)(P.nx / kTile) * P.ny;
    const long long zm = w >= tpp ? w - tpp : w - tpp + P.ntile;
    const long long zp = w + tpp < P.ntile ? w + tpp : w + tpp - P.ntile;
    l2_prefetch(pop + w * kTileElems, 5 * kSlotBytes);
    l2_prefetch(pop + zm * kTileElems + 6 * kSlotElems, kSlotBytes);
    l2_prefetch(pop + zp * kTileElems + 5 * kSlotElems, kSlotBytes);
  }
}

// load_cell for whole-tile rows: even steps read slot i of the own cell, odd steps
// slot opp(i) of cell x - e_i; ESO: the esoteric twist, directions -x, -y, -z from the
// cell x - e_i (= x + e_x, x + e_y, x + e_z) at both parities, the rest from the own cell.
template <int PARITY, typename S, bool ESO = false>
__device__ __forceinline__ void load_cell_rows(const DomainConst& P, const S* __restrict__ pop,
                                               const WarpTiles& T, int lane, float (&d)[kF][kQ]) {
  using V4 = typename Codec<S>::V4;
  using V2 = typename Codec<S>::V2;
#pragma unroll
  for (int i = 0; i < kQ; ++i) {
    long long tile = T.t;
    int ln = lane;
    if (ESO ? eso_shifted(i) : (PARITY && i > 0)) link_tile(T, i, -1, lane, tile, ln);
    const int slot = PARITY ? opp(i) : i;
    if (!LBM_CHECK(P, tile >= 0 && tile < P.ntile)) {
#pragma unroll
      for (int k = 0; k < kF; ++k) d[k][i] = 0.0f;
      continue;
    }
    const S* base = pop + tile * kTileElems;
    float v[kF];
#pragma unroll
    for (int g = 0; g < 3; ++g) {
      const V4 w = *reinterpret_cast<const V4*>(base + group_offset(slot, g, ln));
      Codec<S>::dec4(w, P.scale + 4 * g, v + 4 * g);
    }
    const V2 w2 = *reinterpret_cast<const V2*>(base + group_offset(slot, 3, ln));
    Codec<S>::dec2(w2, P.scale + 12, v + 12);
#pragma unroll
    for (int k = 0; k < kF; ++k) d[k][i] = v[k];
  }
}

// store_cell for whole-tile rows: even steps write slot opp(i) of the own cell, odd
// steps slot i of cell x + e_i; ESO: directions +x, +y, +z into the cell x + e_i at both
// parities, the rest into the own cell.
template <int PARITY, typename S, bool SR = false, bool ESO = false>
__device__ __forceinline__ void store_cell_rows(const DomainConst& P, S* __restrict__ pop,
                                                const WarpTiles& T, int lane,
                                                const float (&d)[kF][kQ]) {
  [[maybe_unused]] Dither dz(0, 0.0f, 0.0f);
  if constexpr (SR) dz = Dither(T.t * kTile + lane, d[0][0], d[4][0]);  // canonical index
#pragma unroll
  for (int i = 0; i < kQ; ++i) {
    long long tile = T.t;
    int ln = lane;
    if (ESO ? (i == 1 || i == 3 || i == 5) : (PARITY && i > 0)) link_tile(T, i, +1, lane, tile, ln);
    if (!LBM_CHECK(P, tile >= 0 && tile < P.ntile)) continue;
    store_dir<S>(P, pop + tile * kTileElems, PARITY ? i : opp(i), ln, d, i, SR ? &dz : nullptr);
  }
}

// MINB = resident 128-thread blocks per SM the register budget is sized for:
// 3 -> at most 170 registers (no spills), 4 -> at most 128 (a few spilled words).
// ROWS: whole-tile rows (periodic x, nx a multiple of 32), addressed per warp.
// SR: stochastic rounding of 16-bit storage.
// ESO: the esoteric twist on whole-tile rows (the other forms take it from P.eso).
template <int PARITY, typename S, bool HELD, int MINB, bool ROWS, bool SR = false, bool ESO = false>
__global__ void __launch_bounds__(128, MINB) k_step(const DomainConst P, S* __restrict__ pop,
                                                    const float* __restrict__ ghost,
                                                    unsigned* __restrict__ flag) {
  float d[kF][kQ];
  if constexpr (ROWS) {
    const int x0 = blockIdx.x * blockDim.x + (threadIdx.x & ~(kTile - 1));
    if (x0 >= P.nx) return;  // whole warps (nx is a multiple of 32)
    const int lane = threadIdx.x & (kTile - 1);
    const WarpTiles T = warp_tiles(P, x0, blockIdx.y, blockIdx.z);
    if (P.pf_tiles > 0 && lane == 0) prefetch_future<PARITY, S, ESO>(P, pop, T.t);
    load_cell_rows<PARITY, S, ESO>(P, pop, T, lane, d);
    if (P.collide) {
      const float probe = collide_cell<false>(P, d, nullptr);
      if (!isfinite(probe)) atomicOr(flag, 1u);
    }
    store_cell_rows<PARITY, S, SR, ESO>(P, pop, T, lane, d);
  } else {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= P.nx) return;
    const CellIndex c = make_index(P, x, blockIdx.y, blockIdx.z);
    load_cell<PARITY, HELD, S>(P, pop, ghost, c, d);
    if (P.collide) {
      const float probe = collide_cell<false>(P, d, nullptr);
      if (!isfinite(probe)) atomicOr(flag, 1u);
    }
    store_cell<PARITY, S, SR>(P, pop, c, d);
  }
}

template <typename S, int MINB, bool SR>
void launch_forms(const DomainConst& P, int parity, S* p, const float* ghost, unsigned* flag,
                  dim3 grid, dim3 block, cudaStream_t s) {
  if (P.bc_x) {
    if (parity) k_step<1, S, true, MINB, false, SR><<<grid, block, 0, s>>>(P, p, ghost, flag);
    else k_step<0, S, true, MINB, false, SR><<<grid, block, 0, s>>>(P, p, ghost, flag);
  } else if (P.nx % kTile == 0 && P.eso) {
    if (parity) k_step<1, S, false, MINB, true, SR, true><<<grid, block, 0, s>>>(P, p, ghost, flag);
    else k_step<0, S, false, MINB, true, SR, true><<<grid, block, 0, s>>>(P, p, ghost, flag);
  } else if (P.nx % kTile == 0) {
    if (parity) k_step<1, S, false, MINB, true, SR><<<grid, block, 0, s>>>(P, p, ghost, flag);
    else k_step<0, S, false, MINB, true, SR><<<grid, block, 0, s>>>(P, p, ghost, flag);
  } else {
    if (parity) k_step<1, S, false, MINB, false, SR><<<grid, block, 0, s>>>(P, p, ghost, flag);
    else k_step<0, S, false, MINB, false, SR><<<grid, block, 0, s>>>(P, p, ghost, flag);
  }
}

template <typename S, int MINB>
void launch_variant(const DomainConst& P, int parity, S* p, const float* ghost, unsigned* flag,
                    dim3 grid, dim3 block, cudaStream_t s) {
  if constexpr (!std::is_same<S, float>::value) {
    if (P.sround) {
      launch_forms<S, MINB, true>(P, parity, p, ghost, flag, grid, block, s);
      return;
    }
  }
  launch_forms<S, MINB, false>(P, parity, p, ghost, flag, grid, block, s);
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
