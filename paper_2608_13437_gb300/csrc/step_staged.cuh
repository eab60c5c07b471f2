// The fused step with its population reads staged through shared memory by bulk
// asynchronous copies (TMA). Same cell update, same results bit for bit as k_step; only
// the way the 98 populations reach the registers differs. A persistent grid of W-warp
// blocks walks the tiles of 32 cells; every warp owns ST shared-memory stages and keeps
// ST - 1 tiles in flight (one mbarrier per stage) while it updates the current one, so
// the bytes in flight no longer depend on how many warps the registers allow. Writes
// stay plain vector stores (every location is written by the thread that read it).
//
// For periodic domains whose rows are whole tiles (nx a multiple of 32): a tile then
// lies in one row, and its y and z neighbours are whole tiles with the same lanes.
//   even step: the tile's own 98 x 32 populations, one copy;
//   odd step:  own slots 0-2 (one copy: rest, and the x neighbours' slots, shifted by a
//              lane), slot 4 of the tile at y - 1, slot 3 at y + 1, slot 6 at z - 1,
//              slot 5 at z + 1 (shared slots 3..6), and for the two edge lanes slot 2 of
//              the tile left of the row segment and slot 1 of the tile right of it
//              (shared slots 7, 8).
// Each warp takes a contiguous run of tiles and walks it with a cursor.
#pragma once

#include "bulk_copy.cuh"
#include "lbm_internal.h"

namespace lbm {

// Limit of a stage wait: far beyond any copy's latency (copies finish in microseconds),
// short enough that a stuck pipeline ends the kernel within about a second.
constexpr uint64_t kStageWaitNs = 1000000000ull;
// A stage holds 9 slot blocks: the 7 of the tile (even steps), or for odd steps the 7
// blocks the tile reads plus the two x-edge blocks (slot 2 of the tile holding cell
// x0 - 1 and slot 1 of the tile holding cell x0 + 32), so no lane leaves shared memory.
constexpr int kStageElems = 9 * kSlotElems;

// Position of a warp's current tile: first cell and its (x0, y, z), advanced one tile
// at a time along x, then y, then z (no divisions after the start).
struct TileCursor {
  long long t;
  int x0, y, z;
  __device__ void start(const DomainConst& P, long long tile) {
    t = tile;
    cell_xyz(P, tile * kTile, x0, y, z);
  }
  __device__ void next(const DomainConst& P) {
    ++t;
    x0 += kTile;
    if (x0 == P.nx) {
      x0 = 0;
      if (++y == P.ny) {
        y = 0;
        ++z;
      }
    }
  }
};

template <int PARITY, typename S>
__device__ __forceinline__ void issue_tile(const DomainConst& P, const S* pop, const TileCursor& q,
                                           S* sb, uint64_t* bar) {
  constexpr uint32_t es = sizeof(S);
  if (PARITY == 0) {
    constexpr uint32_t bytes = kTileElems * es;
    mbar_arrive_expect_tx(bar, bytes);
    bulk_g2s(sb, pop + q.t * kTileElems, bytes, bar);
  } else {
    const long long cell0 = q.t * kTile;
    const long long row = P.nx, plane = (long long)P.nx * P.ny;
    const long long xm = cell0 + (q.x0 > 0 ? -1 : row - 1);
    const long long xp = cell0 + (q.x0 + kTile < P.nx ? kTile : kTile - row);
    const long long ym = cell0 + (q.y > 0 ? -row : plane - row);
    const long long yp = cell0 + (q.y + 1 < P.ny ? row : row - plane);
    const long long zm = cell0 + (q.z > 0 ? -plane : P.ncell - plane);
    const long long zp = cell0 + (q.z + 1 < P.nz ? plane : plane - P.ncell);
    constexpr uint32_t sbytes = kSlotElems * es;
    mbar_arrive_expect_tx(bar, 9 * sbytes);
    bulk_g2s(sb, pop + q.t * kTileElems, 3 * sbytes, bar);
    bulk_g2s(sb + 3 * kSlotElems, pop + tile_start(ym) + 4 * kSlotElems, sbytes, bar);
    bulk_g2s(sb + 4 * kSlotElems, pop + tile_start(yp) + 3 * kSlotElems, sbytes, bar);
    bulk_g2s(sb + 5 * kSlotElems, pop + tile_start(zm) + 6 * kSlotElems, sbytes, bar);
    bulk_g2s(sb + 6 * kSlotElems, pop + tile_start(zp) + 5 * kSlotElems, sbytes, bar);
    bulk_g2s(sb + 7 * kSlotElems, pop + tile_start(xm) + 2 * kSlotElems, sbytes, bar);
    bulk_g2s(sb + 8 * kSlotElems, pop + tile_start(xp) + 1 * kSlotElems, sbytes, bar);
  }
}

// The 14 fields of one direction from the staged block `slot`, lane `ln`: three 4-wide
// and one 2-wide shared-memory access, decoded as in load_cell.
template <typename S>
__device__ __forceinline__ void load_dir(const DomainConst& P, const S* sb, int slot, int ln,
                                         float (&d)[kF][kQ], int i) {
  using V4 = typename Codec<S>::V4;
  using V2 = typename Codec<S>::V2;
  float v[kF];
#pragma unroll
  for (int g = 0; g < 3; ++g) {
    const V4 w = *reinterpret_cast<const V4*>(sb + group_offset(slot, g, ln));
    Codec<S>::dec4(w, P.scale + 4 * g, v + 4 * g);
  }
  const V2 w2 = *reinterpret_cast<const V2*>(sb + group_offset(slot, 3, ln));
  Codec<S>::dec2(w2, P.scale + 12, v + 12);
#pragma unroll
  for (int k = 0; k < kF; ++k) d[k][i] = v[k];
}

template <int PARITY, typename S>
__device__ __forceinline__ void load_cell_staged(const DomainConst& P, const S* sb, int lane,
                                                 float (&d)[kF][kQ]) {
  if (PARITY == 0) {
#pragma unroll
    for (int i = 0; i < kQ; ++i) load_dir<S>(P, sb, i, lane, d, i);
    return;
  }
  load_dir<S>(P, sb, 0, lane, d, 0);
  // +x: slot 2 of cell x - 1 (the left edge block for lane 0); -x: slot 1 of cell x + 1
  // (the right edge block for lane 31)
  load_dir<S>(P, sb, lane > 0 ? 2 : 7, lane > 0 ? lane - 1 : kTile - 1, d, 1);
  load_dir<S>(P, sb, lane < kTile - 1 ? 1 : 8, lane < kTile - 1 ? lane + 1 : 0, d, 2);
#pragma unroll
  for (int i = 3; i < kQ; ++i) load_dir<S>(P, sb, i, lane, d, i);
}

// skip_first: failure-detection test hook; block 0, warp 0 does not issue the copy of
// its first tile, so its wait for that tile runs out.
template <int PARITY, typename S, int W, int ST, int MINB>
__global__ void __launch_bounds__(W * 32, MINB) k_step_staged(const DomainConst P, S* __restrict__ pop,
                                                              unsigned* __restrict__ flag,
                                                              int skip_first) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  S* stages = reinterpret_cast<S*>(smem_raw) + (size_t)warp * ST * kStageElems;
  uint64_t* bar =
      reinterpret_cast<uint64_t*>(smem_raw + (size_t)W * ST * kStageElems * sizeof(S)) + warp * ST;
  if (lane == 0) {
#pragma unroll
    for (int s = 0; s < ST; ++s) mbar_init(&bar[s], 1);
    mbar_init_fence();
  }
  __syncwarp();
  // this warp's tiles: a contiguous run, as equal as possible across warps
  const long long nwarps = (long long)gridDim.x * W;
  const long long wid = (long long)blockIdx.x * W + warp;
  const long long per = P.ntile / nwarps, extra = P.ntile % nwarps;
  const long long count = per + (wid < extra ? 1 : 0);
  if (count == 0) return;
  TileCursor cur, ahead;
  cur.start(P, wid * per + (wid < extra ? wid : extra));
  ahead = cur;
  const bool skip = skip_first && blockIdx.x == 0 && warp == 0;
  long long issued = 0;
  for (; issued < ST - 1 && issued < count; ++issued) {
    if (lane == 0 && !(skip && issued == 0))
      issue_tile<PARITY, S>(P, pop, ahead, stages + issued * kStageElems, &bar[issued]);
    ahead.next(P);
  }
  long long k = 0;
  bool stuck = false;
  for (; k < count; ++k) {
    const int stage = (int)(k % ST);
    if (issued < count) {  // refill the stage freed by the previous tile
      const int sn = (int)(issued % ST);
      if (lane == 0) {
        fence_proxy_async_smem();
        issue_tile<PARITY, S>(P, pop, ahead, stages + sn * kStageElems, &bar[sn]);
      }
      ahead.next(P);
      ++issued;
    }
    if (!mbar_wait(&bar[stage], (uint32_t)((k / ST) & 1), kStageWaitNs)) {
      stuck = true;
      break;
    }
    const CellIndex c = make_index(P, cur.x0 + lane, cur.y, cur.z);
    float d[kF][kQ];
    load_cell_staged<PARITY, S>(P, stages + stage * kStageElems, lane, d);
    if (P.collide) {
      const float probe = collide_cell<false>(P, d, nullptr);
      if (!isfinite(probe)) atomicOr(flag, 1u);
    }
    store_cell<PARITY, S>(P, pop, c, d);
    cur.next(P);
    __syncwarp();
  }
  if (stuck) {
    // Report, and let the copies still in flight (tiles k .. issued - 1) land before
    // the block's shared memory is released.
    if (lane == 0) atomicOr(flag, 2u);
    for (long long kk = k; kk < issued; ++kk)
      mbar_wait(&bar[kk % ST], (uint32_t)((kk / ST) & 1), kStageWaitNs);
  }
}

// Staged variants: 2 -> 4 warps, 2 stages, 170-register budget; 3 -> 4 warps, 2 stages,
// 128 registers; 4 -> 4 warps, 3 stages, 170 registers.
template <int V>
struct StagedCfg;
template <>
struct StagedCfg<2> {
  static constexpr int W = 4, ST = 2, MINB = 3;
};
template <>
struct StagedCfg<3> {
  static constexpr int W = 4, ST = 2, MINB = 4;
};
template <>
struct StagedCfg<4> {
  static constexpr int W = 4, ST = 3, MINB = 3;
};

template <typename S, int V>
size_t staged_smem() {
  using C = StagedCfg<V>;
  return (size_t)C::W * C::ST * kStageElems * sizeof(S) + (size_t)C::W * C::ST * sizeof(uint64_t);
}

template <typename S, int V>
cudaError_t staged_prepare_v(const DomainConst& P, int* grid) {
  using C = StagedCfg<V>;
  const size_t smem = staged_smem<S, V>();
  cudaError_t e = cudaFuncSetAttribute(k_step_staged<0, S, C::W, C::ST, C::MINB>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_step_staged<1, S, C::W, C::ST, C::MINB>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  int dev = 0, nsm = 0, occ = 0;
  if (e == cudaSuccess) e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_step_staged<1, S, C::W, C::ST, C::MINB>,
                                                      C::W * 32, smem);
  if (e != cudaSuccess) return e;
  if (occ < 1) return cudaErrorInvalidConfiguration;
  long long g = (long long)nsm * occ;
  const long long need = (P.ntile + C::W - 1) / C::W;
  if (g > need) g = need;
  *grid = (int)(g < 1 ? 1 : g);
  return cudaSuccess;
}

template <typename S, int V>
void staged_launch_v(const DomainConst& P, int parity, S* pop, unsigned* flag, int grid,
                     int skip_first, cudaStream_t s) {
  using C = StagedCfg<V>;
  const size_t smem = staged_smem<S, V>();
  if (parity)
    k_step_staged<1, S, C::W, C::ST, C::MINB><<<grid, C::W * 32, smem, s>>>(P, pop, flag, skip_first);
  else
    k_step_staged<0, S, C::W, C::ST, C::MINB><<<grid, C::W * 32, smem, s>>>(P, pop, flag, skip_first);
}

template <typename S>
cudaError_t staged_prepare_t(const DomainConst& P, int variant, int* grid) {
  if (!staged_eligible(P)) return cudaErrorInvalidConfiguration;
  switch (variant) {
    case 2: return staged_prepare_v<S, 2>(P, grid);
    case 3: return staged_prepare_v<S, 3>(P, grid);
    case 4: return staged_prepare_v<S, 4>(P, grid);
    default: return cudaErrorInvalidConfiguration;
  }
}

template <typename S>
cudaError_t staged_launch_t(const DomainConst& P, int parity, void* pop, unsigned* flag, int variant,
                            int grid, int skip_first, cudaStream_t s) {
  if (!staged_eligible(P) || grid < 1) return cudaErrorInvalidConfiguration;
  S* p = static_cast<S*>(pop);
  switch (variant) {
    case 2: staged_launch_v<S, 2>(P, parity, p, flag, grid, skip_first, s); break;
    case 3: staged_launch_v<S, 3>(P, parity, p, flag, grid, skip_first, s); break;
    case 4: staged_launch_v<S, 4>(P, parity, p, flag, grid, skip_first, s); break;
    default: return cudaErrorInvalidConfiguration;
  }
  return cudaGetLastError();
}

}  // namespace lbm
