// Diagnostics of the current state (Sec. 3.2, Eq. 7): conservation sums,
// <rho|u|^2/2>, <mu_local |curl u|^2>, 4/3 <mu_local (div u)^2>, extrema and a
// non-finite count. Per-cell work runs in FP32 exactly as in the step (the moments and
// closure come from collide_cell itself); sums are float-float pairs, widened to FP64
// once per block. Pass A decodes every
// cell and keeps u and mu_local in a scratch field (4 floats per cell); the step
// kernel's diagnostic variant fills the same field and writes one record per warp
// instead (step_diag.cuh), which pass R folds into per-block records. Pass B takes
// central differences of u from the field. Each pass writes one record per block
// (warp shuffles, then shared memory) and a single block reduces the records in a
// fixed order, so results are reproducible run to run.
#include "diag_device.cuh"
#include "lbm_internal.h"

namespace lbm {

namespace {

constexpr int kBlock = 256;

// Reduces one DiagAcc per thread over the block into the FP64 record rec[0..kDiagA).
__device__ void block_reduce_acc(DiagAcc a, double* __restrict__ rec) {
  __shared__ float sh[kBlock / 32][kDiagRecWords];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  diag_warp_reduce(a);
  if (lane == 0) diag_store_words(a, sh[warp]);
  __syncthreads();
  if (threadIdx.x == 0) {
    DiagAcc r;
    diag_load_words(sh[0], r);
    for (int w = 1; w < kBlock / 32; ++w) {
      DiagAcc b;
      diag_load_words(sh[w], b);
      diag_merge(r, b);
    }
    diag_store_partial(r, rec);
  }
}

// Pass A: per cell, the step's own FP32 decode, moments and closure (collide_cell in
// its sensor mode leaves the populations alone). Writes u and mu_local for pass B.
template <typename S, int PARITY, bool HELD>
__global__ void __launch_bounds__(kBlock) k_diag_a(const DomainConst P, const S* __restrict__ pop,
                                                   const float* __restrict__ ghost,
                                                   float* __restrict__ ufield,
                                                   double* __restrict__ partials) {
  DiagAcc acc;
  diag_zero(acc);
  const long long n = P.ncell;
  for (long long cell = blockIdx.x * (long long)blockDim.x + threadIdx.x; cell < n;
       cell += (long long)gridDim.x * blockDim.x) {
    int x, y, z;
    cell_xyz(P, cell, x, y, z);
    const CellIndex c = make_index(P, x, y, z);
    float d[kF][kQ];
    load_cell<PARITY, HELD, S>(P, pop, ghost, c, d);
    SensorOut so;
    CellDiag cd;
    collide_cell<true, true>(P, d, &so, &cd);
    diag_add_cell(P, cd, acc);
    ufield[cell] = cd.u[0];
    ufield[n + cell] = cd.u[1];
    ufield[2 * n + cell] = cd.u[2];
    ufield[3 * n + cell] = cd.mu_T;
  }
  block_reduce_acc(acc, partials + (long long)blockIdx.x * kDiagA);
}

// Pass R: folds nrec warp records of the step's diagnostic variant into one record per
// block (block b takes a contiguous range, in order).
__global__ void __launch_bounds__(kBlock) k_diag_records(const float* __restrict__ rec,
                                                         long long nrec,
                                                         double* __restrict__ partials) {
  const long long per = (nrec + gridDim.x - 1) / gridDim.x;
  const long long lo = blockIdx.x * per;
  const long long hi = lo + per < nrec ? lo + per : nrec;
  DiagAcc acc;
  diag_zero(acc);
  for (long long r = lo + threadIdx.x; r < hi; r += blockDim.x) {
    DiagAcc b;
    diag_load_words(rec + r * kDiagRecWords, b);
    diag_merge(acc, b);
  }
  block_reduce_acc(acc, partials + (long long)blockIdx.x * kDiagA);
}

// Pass B: central differences of u (FP32, from the FP32 field), weighted by mu_local;
// per-cell products in FP32, float-float sums. Work items are columns of 32 x 8 cells
// (x by y) over kZChunk planes; a persistent grid takes them in a fixed order (block b:
// items b, b + grid, ...), so sums are reproducible. A block marches up its column
// through a ring of kRing planes in shared memory: each plane holds u on the column
// with a one-cell halo in x and y (wrapped periodically) and mu_local on the column,
// filled by asynchronous copies (cp.async) two planes ahead of the plane being
// differenced, so DRAM reads of the planes ahead are in flight while the block
// computes. Full rows of 32 cells whose start is 16-byte aligned (nx a multiple of 4)
// move as eight 16-byte copies; other tiles element by element. A thread keeps u of
// its own cell at z - 1 and z in registers. Every value of the field is read from
// DRAM about once (the halo comes from L2: neighbouring columns are processed at
// about the same z).
constexpr int kTileX = 32, kTileY = kBlock / 32, kZChunk = 32, kRing = 5;
// a u row in shared memory: 3 pad, the x - 1 halo, 32 cells (16-byte aligned), the
// x + 32 halo, 3 pad
constexpr int kRowU = kTileX + 8, kRowsU = kTileY + 2, kPlaneU = kRowU * kRowsU;
constexpr int kColX0 = 4;  // column of the first cell of the tile
constexpr int kPlaneMu = kTileX * kTileY;
// copies per plane: element-wise (34 x 10 u values x 3 + 32 x 8 mu values) and
// vectorised (3 x 10 rows x 8 chunks + 3 x 10 x 2 halo values + 8 rows x 8 mu chunks)
constexpr int kScalarCopies = 3 * (kTileX + 2) * kRowsU + kPlaneMu;
constexpr int kVecU = 3 * kRowsU * (kTileX / 4), kVecHalo = 3 * kRowsU * 2,
              kVecMu = kTileY * (kTileX / 4);
constexpr int kVecCopies = kVecU + kVecHalo + kVecMu;
constexpr int kMaxCopiesPerThread = (kScalarCopies + kBlock - 1) / kBlock;

__device__ __forceinline__ void cp_async4(float* dst, const float* src) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async16(float* dst, const float* src) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

__device__ __forceinline__ int wrap_index(int v, int n) {
  v %= n;
  return v < 0 ? v + n : v;
}

struct DiagBPlanes {
  float u[kRing][3][kPlaneU];
  float mu[kRing][kPlaneMu];
};

// One copy of a plane: source offset within a z plane of the field (component
// included), destination in ring slot 0, size (0: none, 4 or 16 bytes) and the ring
// stride of its destination array.
struct PlaneCopy {
  long long off;
  float* dst;
  int bytes, stride;
};

__global__ void __launch_bounds__(kBlock) k_diag_b(const DomainConst P,
                                                   const float* __restrict__ ufield,
                                                   double* __restrict__ partials) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  DiagBPlanes& sm = *reinterpret_cast<DiagBPlanes*>(smem_raw);
  FF acc[2] = {{0.0f, 0.0f}, {0.0f, 0.0f}};
  const long long n = P.ncell;
  const float inv_dx = (float)(1.0 / P.dx64), inv_2dx = (float)(0.5 / P.dx64);
  const int cols_x = (P.nx + kTileX - 1) / kTileX, cols_y = (P.ny + kTileY - 1) / kTileY;
  const int chunks = (P.nz + kZChunk - 1) / kZChunk;
  const long long items = (long long)cols_x * cols_y * chunks;
  const long long nxy = (long long)P.nx * P.ny;
  const int tx = threadIdx.x % kTileX, ty = threadIdx.x / kTileX;
  for (long long it = blockIdx.x; it < items; it += gridDim.x) {
    const int cx = (int)(it % cols_x);
    const long long r = it / cols_x;
    const int cy = (int)(r % cols_y), cz = (int)(r / cols_y);
    const int x0 = cx * kTileX, y0 = cy * kTileY;
    const int z0 = cz * kZChunk, z1 = min(z0 + kZChunk, P.nz);
    const int np = z1 - z0 + 2;  // planes z0 - 1 ... z1 (wrapped)
    const bool vec = (P.nx % 4 == 0) && (x0 + kTileX <= P.nx);
    // this thread's copies of every plane (the same offsets for each plane)
    PlaneCopy cp[kMaxCopiesPerThread];
#pragma unroll
    for (int k = 0; k < kMaxCopiesPerThread; ++k) {
      const int q = threadIdx.x + k * kBlock;
      cp[k].bytes = 0;
      cp[k].off = 0;
      cp[k].dst = sm.mu[0];
      cp[k].stride = 0;
      if (vec) {
        if (q < kVecU) {  // 16-byte chunk of a full u row
          const int c = q / (kRowsU * 8), rem = q - c * (kRowsU * 8);
          const int row = rem / 8, ch = rem - row * 8;
          const int gy = wrap_index(y0 - 1 + row, P.ny);
          cp[k] = {(long long)c * n + (long long)gy * P.nx + x0 + 4 * ch,
                   &sm.u[0][c][row * kRowU + kColX0 + 4 * ch], 16, 3 * kPlaneU};
        } else if (q < kVecU + kVecHalo) {  // the x halo of a u row
          const int h = q - kVecU;
          const int c = h / (kRowsU * 2), rem = h - c * (kRowsU * 2);
          const int row = rem / 2, side = rem - row * 2;
          const int gy = wrap_index(y0 - 1 + row, P.ny);
          const int gx = side ? wrap_index(x0 + kTileX, P.nx) : wrap_index(x0 - 1, P.nx);
          cp[k] = {(long long)c * n + (long long)gy * P.nx + gx,
                   &sm.u[0][c][row * kRowU + (side ? kColX0 + kTileX : kColX0 - 1)], 4,
                   3 * kPlaneU};
        } else if (q < kVecCopies) {  // 16-byte chunk of a mu row
          const int m = q - kVecU - kVecHalo;
          const int row = m / 8, ch = m - row * 8;
          const int gy = min(y0 + row, P.ny - 1);
          cp[k] = {3 * n + (long long)gy * P.nx + x0 + 4 * ch, &sm.mu[0][row * kTileX + 4 * ch], 16,
                   kPlaneMu};
        }
      } else if (q < 3 * (kTileX + 2) * kRowsU) {  // one u value of the halo tile
        const int c = q / ((kTileX + 2) * kRowsU), j = q - c * ((kTileX + 2) * kRowsU);
        const int row = j / (kTileX + 2), lx = j - row * (kTileX + 2);
        const int gx = wrap_index(x0 - 1 + lx, P.nx), gy = wrap_index(y0 - 1 + row, P.ny);
        cp[k] = {(long long)c * n + (long long)gy * P.nx + gx,
                 &sm.u[0][c][row * kRowU + kColX0 - 1 + lx], 4, 3 * kPlaneU};
      } else if (q < kScalarCopies) {  // one mu value of the tile
        const int j = q - 3 * (kTileX + 2) * kRowsU;
        const int row = j / kTileX, lx = j - row * kTileX;
        const int gx = min(x0 + lx, P.nx - 1), gy = min(y0 + row, P.ny - 1);
        cp[k] = {3 * n + (long long)gy * P.nx + gx, &sm.mu[0][j], 4, kPlaneMu};
      }
    }
    // plane p of the column is z = z0 - 1 + p (wrapped), held in ring slot p % kRing
    auto issue = [&](int p) {
      if (p < np) {
        const long long zoff = (long long)wrap_index(z0 - 1 + p, P.nz) * nxy;
        const int slot = p % kRing;
#pragma unroll
        for (int k = 0; k < kMaxCopiesPerThread; ++k) {
          if (cp[k].bytes == 16) cp_async16(cp[k].dst + slot * cp[k].stride, ufield + cp[k].off + zoff);
          else if (cp[k].bytes == 4) cp_async4(cp[k].dst + slot * cp[k].stride, ufield + cp[k].off + zoff);
        }
      }
      cp_async_commit();  // an empty group past the last plane keeps the count uniform
    };
#pragma unroll
    for (int p = 0; p < kRing - 1; ++p) issue(p);
    const int x = x0 + tx, y = y0 + ty;
    const bool valid = x < P.nx && y < P.ny;
    // x neighbours in the halo tile: one-sided at held ends (the own value)
    const int hc = (ty + 1) * kRowU + kColX0 + tx;
    int hxh = hc + 1, hxl = hc - 1;
    float wxd = inv_2dx;
    if (P.bc_x) {
      if (x == P.nx - 1) hxh = hc;
      if (x == 0) hxl = hc;
      const int span = (x < P.nx - 1) + (x > 0);
      wxd = span == 2 ? inv_2dx : (span == 1 ? inv_dx : 0.0f);
    }
    float pu[3], cu[3];  // u of the own cell at z - 1 and z
    for (int i = 0; i < z1 - z0; ++i) {
      cp_async_wait<kRing - 4>();  // planes up to i + 2 have landed (this thread's copies)
      __syncthreads();             // ... everyone's; and everyone is done with plane i - 1
      issue(i + kRing - 1);        // into the slot of plane i - 1
      const int s0 = (i + 1) % kRing, sp = (i + 2) % kRing;
      if (i == 0) {
#pragma unroll
        for (int b = 0; b < 3; ++b) {
          pu[b] = sm.u[0][b][hc];
          cu[b] = sm.u[1 % kRing][b][hc];
        }
      }
      if (valid) {
        const float(*U)[kPlaneU] = sm.u[s0];
        float g[3][3];  // g[a][b] = d_a u_b
#pragma unroll
        for (int b = 0; b < 3; ++b) {
          const float nu = sm.u[sp][b][hc];
          g[0][b] = mul(sub(U[b][hxh], U[b][hxl]), wxd);
          g[1][b] = mul(sub(U[b][hc + kRowU], U[b][hc - kRowU]), inv_2dx);
          g[2][b] = mul(sub(nu, pu[b]), inv_2dx);
          pu[b] = cu[b];
          cu[b] = nu;
        }
        const float wx = sub(g[1][2], g[2][1]), wy = sub(g[2][0], g[0][2]), wz = sub(g[0][1], g[1][0]);
        const float div = add(add(g[0][0], g[1][1]), g[2][2]);
        const float mu_loc = sm.mu[s0][ty * kTileX + tx];
        ff_add(acc[0], mul(mu_loc, fma_(wz, wz, fma_(wy, wy, mul(wx, wx)))));
        ff_add(acc[1], mul(mu_loc, mul(div, div)));
      }
    }
    cp_async_wait<0>();
    __syncthreads();  // the next item refills every slot
  }
  __shared__ FF sh[kBlock / 32][2];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int j = 0; j < 2; ++j) {
    for (int o = 16; o > 0; o >>= 1) {
      FF b;
      b.hi = __shfl_down_sync(0xffffffffu, acc[j].hi, o);
      b.lo = __shfl_down_sync(0xffffffffu, acc[j].lo, o);
      ff_merge(acc[j], b);
    }
    if (lane == 0) sh[warp][j] = acc[j];
  }
  __syncthreads();
  if (threadIdx.x < 2) {
    FF r = sh[0][threadIdx.x];
    for (int w = 1; w < kBlock / 32; ++w) ff_merge(r, sh[w][threadIdx.x]);
    partials[(long long)blockIdx.x * 2 + threadIdx.x] = ff_value(r);
  }
}

constexpr size_t kDiagBSmem = sizeof(DiagBPlanes);

// Fixed-order FP64 reduction of the block records of both passes (one block of
// kBlock threads): thread t folds blocks t, t + kBlock, ... of every quantity, then a
// shared-memory tree combines the threads in a fixed pattern. The reference density
// and energy are added back once per cell at the end.
__global__ void __launch_bounds__(kBlock) k_diag_final(const DomainConst P,
                                                       const double* __restrict__ pa,
                                                       const double* __restrict__ pb, int nblocks,
                                                       double* __restrict__ out) {
  constexpr int kN = kDiagA + 2;
  __shared__ double sh[kN][kBlock];
  const int t = threadIdx.x;
  double r[kN];
#pragma unroll
  for (int j = 0; j < kN; ++j) r[j] = (j >= 9 && j < 11) ? -INFINITY : ((j == 11 || j == 12) ? INFINITY : 0.0);
  for (int b = t; b < nblocks; b += kBlock) {
#pragma unroll
    for (int j = 0; j < kDiagA; ++j) {
      const double v = pa[(long long)b * kDiagA + j];
      r[j] = j < 9 ? r[j] + v : (j < 11 ? fmax(r[j], v) : fmin(r[j], v));
    }
    r[kDiagA] += pb[(long long)b * 2];
    r[kDiagA + 1] += pb[(long long)b * 2 + 1];
  }
#pragma unroll
  for (int j = 0; j < kN; ++j) sh[j][t] = r[j];
  __syncthreads();
  for (int half = kBlock / 2; half > 0; half >>= 1) {
    if (t < half) {
#pragma unroll
      for (int j = 0; j < kN; ++j) {
        const double v = sh[j][t + half];
        sh[j][t] = (j < 9 || j >= kDiagA) ? sh[j][t] + v
                                          : (j < 11 ? fmax(sh[j][t], v) : fmin(sh[j][t], v));
      }
    }
    __syncthreads();
  }
  if (t < kN) {
    double v = sh[t][0];
    if (t == 0) v += (double)P.rho_ref * (double)P.ncell;
    if (t == 4) v += (double)P.E_ref * (double)P.ncell;
    out[t] = v;
  }
}

template <typename S, int PARITY, bool HELD>
void launch_a(const DomainConst& P, const void* pop, const float* ghost, float* ufield, double* pa,
              cudaStream_t s) {
  k_diag_a<S, PARITY, HELD><<<kDiagBlocks, kBlock, 0, s>>>(P, static_cast<const S*>(pop), ghost,
                                                           ufield, pa);
}

template <typename S>
void launch_a_store(const DomainConst& P, int parity, const void* pop, const float* ghost,
                    float* ufield, double* pa, cudaStream_t s) {
  if (P.bc_x) {
    if (parity) launch_a<S, 1, true>(P, pop, ghost, ufield, pa, s);
    else launch_a<S, 0, true>(P, pop, ghost, ufield, pa, s);
  } else {
    if (parity) launch_a<S, 1, false>(P, pop, ghost, ufield, pa, s);
    else launch_a<S, 0, false>(P, pop, ghost, ufield, pa, s);
  }
}

}  // namespace

cudaError_t launch_diag(const DomainConst& P, int store, int parity, const void* pop,
                        const float* ghost, float* ufield, double* partials, double* out16,
                        cudaStream_t s) {
  double* pa = partials;
  double* pb = partials + (long long)kDiagBlocks * kDiagA;
  switch (store) {
    case 0: launch_a_store<float>(P, parity, pop, ghost, ufield, pa, s); break;
    case 1: launch_a_store<__half>(P, parity, pop, ghost, ufield, pa, s); break;
    default: launch_a_store<__nv_bfloat16>(P, parity, pop, ghost, ufield, pa, s); break;
  }
  k_diag_b<<<kDiagBlocks, kBlock, kDiagBSmem, s>>>(P, ufield, pb);
  k_diag_final<<<1, kBlock, 0, s>>>(P, pa, pb, kDiagBlocks, out16);
  return cudaGetLastError();
}

cudaError_t launch_diag_records(const DomainConst& P, const float* rec, long long nrec,
                                const float* ufield, double* partials, double* out16,
                                cudaStream_t s) {
  double* pa = partials;
  double* pb = partials + (long long)kDiagBlocks * kDiagA;
  k_diag_records<<<kDiagBlocks, kBlock, 0, s>>>(rec, nrec, pa);
  k_diag_b<<<kDiagBlocks, kBlock, kDiagBSmem, s>>>(P, ufield, pb);
  k_diag_final<<<1, kBlock, 0, s>>>(P, pa, pb, kDiagBlocks, out16);
  return cudaGetLastError();
}

}  // namespace lbm
