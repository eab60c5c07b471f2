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
// per-cell products in FP32, float-float sums. Work items are columns of 32 x 16 cells
// (x by y) over kZChunk planes; a grid of resident blocks takes them in a fixed order
// (block b: items b, b + grid, ...), so sums are reproducible. A block of 128 threads
// marches up its column; a thread owns 4 consecutive cells of one row. u of the
// column with a one-cell halo in x and y (wrapped periodically) passes through a ring
// of kRingB planes in shared memory, filled by asynchronous copies (cp.async) two
// planes ahead of the plane being differenced (16-byte copies for full tile rows that
// start 16-byte aligned, element copies otherwise), so the DRAM reads of the planes
// ahead are in flight while the block computes. A thread keeps u of its own cells at
// z - 1, z and z + 1 in registers and reads mu_local of its cells straight from the
// field one plane ahead. The differences are taken unscaled and the products scaled
// once by (1 / 2 dx)^2 (one-sided x differences at held ends carry a factor 2).
// Every value of the field is read from DRAM about once (the halo comes from L2:
// neighbouring columns are processed at about the same z).
constexpr int kBlockB = 128, kTileX = 32, kTileY = 16, kCells = 4, kZChunk = 32, kRingB = 4;
constexpr int kRowF = kTileX + 8;           // 3 pad, x - 1 halo, 32 cells, x + 32 halo, 3 pad
constexpr int kRowsB = kTileY + 2;          // y - 1 halo, 16 rows, y + 16 halo
constexpr int kColX0 = 4;                   // column of the tile's first cell (16-byte aligned)
constexpr int kPlaneB = 3 * kRowsB * kRowF; // floats of one plane (three components)
constexpr int kVecRows = 3 * kRowsB * (kTileX / 4), kVecHalo = 3 * kRowsB * 2;
constexpr int kScalarCopies = 3 * kRowsB * (kTileX + 2);

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

__device__ __forceinline__ float4 lds4(const float* p) { return *reinterpret_cast<const float4*>(p); }

__global__ void __launch_bounds__(kBlockB) k_diag_b(const DomainConst P,
                                                    const float* __restrict__ ufield,
                                                    double* __restrict__ partials) {
  extern __shared__ __align__(16) float ring[];  // [kRingB][3][kRowsB][kRowF]
  __shared__ long long rowoff[kRowsB];           // (wrapped y) * nx of each tile row
  __shared__ int halo_x[2];                      // wrapped x0 - 1 and x0 + 32
  FF acc[2] = {{0.0f, 0.0f}, {0.0f, 0.0f}};
  const long long n = P.ncell;
  const float inv_2dx = (float)(0.5 / P.dx64);
  const float s2 = mul(inv_2dx, inv_2dx);
  const int cols_x = (P.nx + kTileX - 1) / kTileX, cols_y = (P.ny + kTileY - 1) / kTileY;
  const int chunks = (P.nz + kZChunk - 1) / kZChunk;
  const long long items = (long long)cols_x * cols_y * chunks;
  const long long nxy = (long long)P.nx * P.ny;
  const int tx = threadIdx.x & 7, ty = threadIdx.x >> 3;  // cells 4 tx .. 4 tx + 3 of row ty
  const float* MU = ufield + 3 * n;
  for (long long it = blockIdx.x; it < items; it += gridDim.x) {
    const int cx = (int)(it % cols_x);
    const long long r = it / cols_x;
    const int cy = (int)(r % cols_y), cz = (int)(r / cols_y);
    const int x0 = cx * kTileX, y0 = cy * kTileY;
    const int z0 = cz * kZChunk, z1 = min(z0 + kZChunk, P.nz);
    const int np = z1 - z0 + 2;  // planes z0 - 1 ... z1 (wrapped)
    const bool vec = (P.nx % 4 == 0) && (x0 + kTileX <= P.nx);
    if (threadIdx.x < kRowsB) rowoff[threadIdx.x] = (long long)wrap_index(y0 - 1 + threadIdx.x, P.ny) * P.nx;
    if (threadIdx.x == kRowsB) halo_x[0] = wrap_index(x0 - 1, P.nx);
    if (threadIdx.x == kRowsB + 1) halo_x[1] = wrap_index(x0 + kTileX, P.nx);
    __syncthreads();
    // plane p of the column is z = z0 - 1 + p (wrapped), held in ring slot p % kRingB
    auto issue = [&](int p) {
      if (p < np) {
        const long long zoff = (long long)wrap_index(z0 - 1 + p, P.nz) * nxy;
        float* slot = ring + (p % kRingB) * kPlaneB;
        if (vec) {
          for (int q = threadIdx.x; q < kVecRows + kVecHalo; q += kBlockB) {
            if (q < kVecRows) {  // 16-byte chunk of a full row
              const int c = q / (kRowsB * 8), rem = q - c * (kRowsB * 8);
              const int row = rem >> 3, ch = rem & 7;
              cp_async16(slot + (c * kRowsB + row) * kRowF + kColX0 + 4 * ch,
                         ufield + c * n + zoff + rowoff[row] + x0 + 4 * ch);
            } else {  // the x halo of a row
              const int h = q - kVecRows;
              const int c = h / (kRowsB * 2), rem = h - c * (kRowsB * 2);
              const int row = rem >> 1, side = rem & 1;
              cp_async4(slot + (c * kRowsB + row) * kRowF + (side ? kColX0 + kTileX : kColX0 - 1),
                        ufield + c * n + zoff + rowoff[row] + halo_x[side]);
            }
          }
        } else {
          for (int q = threadIdx.x; q < kScalarCopies; q += kBlockB) {
            const int c = q / (kRowsB * (kTileX + 2)), rem = q - c * (kRowsB * (kTileX + 2));
            const int row = rem / (kTileX + 2), lx = rem - row * (kTileX + 2);
            cp_async4(slot + (c * kRowsB + row) * kRowF + kColX0 - 1 + lx,
                      ufield + c * n + zoff + rowoff[row] + wrap_index(x0 - 1 + lx, P.nx));
          }
        }
      }
      cp_async_commit();  // an empty group past the last plane keeps the count uniform
    };
#pragma unroll
    for (int p = 0; p < kRingB; ++p) issue(p);
    const int xa = x0 + kCells * tx, y = y0 + ty;
    const bool row_ok = y < P.ny;
    int nvalid = row_ok ? min(kCells, P.nx - xa) : 0;
    if (nvalid < 0) nvalid = 0;
    // mu_local of the own cells at plane z (direct loads, one plane ahead)
    const long long own = (long long)y * P.nx + xa;
    auto load_mu = [&](int z, float (&m)[kCells]) {
      const long long o = (long long)z * nxy + own;
      if (vec && row_ok) {
        const float4 v = *reinterpret_cast<const float4*>(MU + o);
        m[0] = v.x; m[1] = v.y; m[2] = v.z; m[3] = v.w;
      } else {
#pragma unroll
        for (int j = 0; j < kCells; ++j) m[j] = j < nvalid ? MU[o + j] : 0.0f;
      }
    };
    // one-sided x differences at held ends: factor 2 on the one available difference
    float fx[kCells];
    bool own_l[kCells], own_r[kCells];
#pragma unroll
    for (int j = 0; j < kCells; ++j) {
      const int x = xa + j;
      own_l[j] = P.bc_x && x == 0;
      own_r[j] = P.bc_x && x == P.nx - 1;
      const int span = (x < P.nx - 1) + (x > 0);
      fx[j] = !P.bc_x ? 1.0f : (span == 2 ? 1.0f : (span == 1 ? 2.0f : 0.0f));
    }
    const int hc = (ty + 1) * kRowF + kColX0 + kCells * tx;  // own first cell in a plane
    float pu[3][kCells], cu[3][kCells], mu[kCells], mu_n[kCells];
    cp_async_wait<kRingB - 2>();  // planes 0 and 1
    __syncthreads();
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const float4 a = lds4(ring + 0 * kPlaneB + c * kRowsB * kRowF + hc);
      const float4 b = lds4(ring + 1 * kPlaneB + c * kRowsB * kRowF + hc);
      pu[c][0] = a.x; pu[c][1] = a.y; pu[c][2] = a.z; pu[c][3] = a.w;
      cu[c][0] = b.x; cu[c][1] = b.y; cu[c][2] = b.z; cu[c][3] = b.w;
    }
    load_mu(z0, mu);
    for (int i = 0; i < z1 - z0; ++i) {
      cp_async_wait<kRingB - 3>();  // planes up to i + 2 have landed (this thread's copies)
      __syncthreads();              // ... everyone's; and everyone is done with plane i
      issue(i + kRingB);            // into the slot of plane i
      if (i + 1 < z1 - z0) load_mu(z0 + i + 1, mu_n);
      const float* S0 = ring + ((i + 1) % kRingB) * kPlaneB;  // plane z
      const float* SP = ring + ((i + 2) % kRingB) * kPlaneB;  // plane z + 1
      float d[3][3][kCells];  // d[a][b][j]: unscaled central difference of u_b along a
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        const float* C0 = S0 + c * kRowsB * kRowF + hc;
        const float4 nu = lds4(SP + c * kRowsB * kRowF + hc);
        const float4 ym = lds4(C0 - kRowF), yp = lds4(C0 + kRowF);
        const float xl = C0[-1], xr = C0[kCells];
        const float nv[kCells] = {nu.x, nu.y, nu.z, nu.w};
        const float ymv[kCells] = {ym.x, ym.y, ym.z, ym.w}, ypv[kCells] = {yp.x, yp.y, yp.z, yp.w};
#pragma unroll
        for (int j = 0; j < kCells; ++j) {
          float right = j + 1 < kCells ? cu[c][j + 1] : xr;
          float left = j > 0 ? cu[c][j - 1] : xl;
          if (own_r[j]) right = cu[c][j];
          if (own_l[j]) left = cu[c][j];
          d[0][c][j] = mul(sub(right, left), fx[j]);
          d[1][c][j] = sub(ypv[j], ymv[j]);
          d[2][c][j] = sub(nv[j], pu[c][j]);
        }
#pragma unroll
        for (int j = 0; j < kCells; ++j) {  // march: z becomes z - 1, z + 1 becomes z
          pu[c][j] = cu[c][j];
          cu[c][j] = nv[j];
        }
      }
      float ss = 0.0f, sd = 0.0f;
#pragma unroll
      for (int j = 0; j < kCells; ++j) {
        if (j < nvalid) {
          const float wx = sub(d[1][2][j], d[2][1][j]), wy = sub(d[2][0][j], d[0][2][j]),
                      wz = sub(d[0][1][j], d[1][0][j]);
          const float div = add(add(d[0][0][j], d[1][1][j]), d[2][2][j]);
          ss = fma_(mu[j], fma_(wz, wz, fma_(wy, wy, mul(wx, wx))), ss);
          sd = fma_(mu[j], mul(div, div), sd);
        }
      }
      ff_add(acc[0], mul(ss, s2));
      ff_add(acc[1], mul(sd, s2));
#pragma unroll
      for (int j = 0; j < kCells; ++j) mu[j] = mu_n[j];
    }
    cp_async_wait<0>();
    __syncthreads();  // the next item refills every slot and the row table
  }
  __shared__ FF sh[kBlockB / 32][2];
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
    for (int w = 1; w < kBlockB / 32; ++w) ff_merge(r, sh[w][threadIdx.x]);
    partials[(long long)blockIdx.x * 2 + threadIdx.x] = ff_value(r);
  }
}

constexpr size_t kDiagBSmem = sizeof(float) * kRingB * kPlaneB;

// Grid of pass B: the blocks resident on the device at once (one wave), at most
// kDiagBlocks (the partials buffer holds that many).
int diag_b_grid() {
  int dev = 0, sms = 0, per_sm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_diag_b, kBlockB, kDiagBSmem) !=
          cudaSuccess) {
    cudaGetLastError();
    return kDiagBlocks;
  }
  const int g = sms * per_sm;
  return g < 1 ? 1 : (g > kDiagBlocks ? kDiagBlocks : g);
}

// Fixed-order FP64 reduction of the block records of both passes (nblocks records of
// pass A or R, nblocks_b <= nblocks of pass B; one block of kBlock threads): thread t
// folds blocks t, t + kBlock, ... of every quantity, then a
// shared-memory tree combines the threads in a fixed pattern. The reference density
// and energy are added back once per cell at the end.
__global__ void __launch_bounds__(kBlock) k_diag_final(const DomainConst P,
                                                       const double* __restrict__ pa,
                                                       const double* __restrict__ pb, int nblocks,
                                                       int nblocks_b, double* __restrict__ out) {
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
    if (b < nblocks_b) {
      r[kDiagA] += pb[(long long)b * 2];
      r[kDiagA + 1] += pb[(long long)b * 2 + 1];
    }
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
  const int gb = diag_b_grid();
  k_diag_b<<<gb, kBlockB, kDiagBSmem, s>>>(P, ufield, pb);
  k_diag_final<<<1, kBlock, 0, s>>>(P, pa, pb, kDiagBlocks, gb, out16);
  return cudaGetLastError();
}

cudaError_t launch_diag_records(const DomainConst& P, const float* rec, long long nrec,
                                const float* ufield, double* partials, double* out16,
                                cudaStream_t s) {
  double* pa = partials;
  double* pb = partials + (long long)kDiagBlocks * kDiagA;
  k_diag_records<<<kDiagBlocks, kBlock, 0, s>>>(rec, nrec, pa);
  const int gb = diag_b_grid();
  k_diag_b<<<gb, kBlockB, kDiagBSmem, s>>>(P, ufield, pb);
  k_diag_final<<<1, kBlock, 0, s>>>(P, pa, pb, kDiagBlocks, gb, out16);
  return cudaGetLastError();
}

}  // namespace lbm
