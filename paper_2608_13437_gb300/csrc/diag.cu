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
  diag_warp_reduce_store(a, sh[threadIdx.x >> 5]);
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
// marches up its column; a thread owns 4 consecutive cells of one row (128-bit shared
// loads). u of the column
// with a one-cell halo in x and y (wrapped periodically), and mu_local of the column,
// pass through a ring of kRingB planes in shared memory, filled by asynchronous copies
// (cp.async) two planes ahead of the plane being differenced, so the DRAM reads of the
// planes ahead are in flight while the block computes. When nx is a multiple of 32
// every tile row is a full, 16-byte aligned row and moves as 16-byte copies whose
// addresses a thread fixes once per item; otherwise element copies (a separate
// instantiation). A thread keeps u of its own cells at z - 1, z and z + 1 in three
// register sets whose roles rotate. The differences are taken unscaled and the
// products scaled once by (1 / 2 dx)^2 (one-sided x differences at held ends carry a
// factor 2); the products of two planes are summed in FP32 before each float-float
// addition. Every value of the field is read from DRAM about once (the halo comes
// from L2: neighbouring columns are processed at about the same z).
constexpr int kCells = 4;  // consecutive cells of a row per thread
constexpr int kTileX = 32, kTileY = 16, kZChunk = 32, kRingB = 4;
constexpr int kThreadsX = kTileX / kCells, kBlockB = kThreadsX * kTileY;
constexpr int kRowF = kTileX + 8;           // 3 pad, x - 1 halo, 32 cells, x + 32 halo, 3 pad
constexpr int kRowsB = kTileY + 2;          // y - 1 halo, 16 rows, y + 16 halo
constexpr int kColX0 = 4;                   // column of the tile's first cell (16-byte aligned)
constexpr int kPlaneU = 3 * kRowsB * kRowF; // floats of u on one plane (three components)
constexpr int kPlaneB = kPlaneU + kTileX * kTileY;  // ... followed by mu_local of the tile
constexpr int kVecRows = 3 * kRowsB * (kTileX / 4), kVecHalo = 3 * kRowsB * 2;
constexpr int kVecMu = kTileY * (kTileX / 4);
constexpr int kVecCopies = kVecRows + kVecHalo + kVecMu;
constexpr int kMaxCopies = (kVecCopies + kBlockB - 1) / kBlockB;  // per thread and plane
constexpr int kScalarCopies = 3 * kRowsB * (kTileX + 2) + kTileX * kTileY;

__device__ __forceinline__ void cp_async4(float* dst, const float* src) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(d), "l"(src) : "memory");
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

// kCells consecutive floats from a kCells * 4-byte aligned address
__device__ __forceinline__ void ldv(const float* p, float (&o)[kCells]) {
  if constexpr (kCells == 4) {
    const float4 v = *reinterpret_cast<const float4*>(p);
    o[0] = v.x; o[1] = v.y; o[2] = v.z; o[3] = v.w;
  } else {
    const float2 v = *reinterpret_cast<const float2*>(p);
    o[0] = v.x; o[1] = v.y;
  }
}

// kVec: nx is a multiple of 32, so every tile row is a full, 16-byte aligned row of 32
// cells (vector copies and loads); otherwise element copies with wrapped x.
template <bool kVec>
__global__ void __launch_bounds__(kBlockB, 4) k_diag_b(const DomainConst P,
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
  const int tx = threadIdx.x % kThreadsX, ty = threadIdx.x / kThreadsX;  // cells kCells tx... of row ty
  for (long long it = blockIdx.x; it < items; it += gridDim.x) {
    const int cx = (int)(it % cols_x);
    const long long r = it / cols_x;
    const int cy = (int)(r % cols_y), cz = (int)(r / cols_y);
    const int x0 = cx * kTileX, y0 = cy * kTileY;
    const int z0 = cz * kZChunk, z1 = min(z0 + kZChunk, P.nz);
    const int np = z1 - z0 + 2;  // planes z0 - 1 ... z1 (wrapped)
    constexpr bool vec = kVec;
    if (threadIdx.x < kRowsB) rowoff[threadIdx.x] = (long long)wrap_index(y0 - 1 + threadIdx.x, P.ny) * P.nx;
    if (threadIdx.x == kRowsB) halo_x[0] = wrap_index(x0 - 1, P.nx);
    if (threadIdx.x == kRowsB + 1) halo_x[1] = wrap_index(x0 + kTileX, P.nx);
    __syncthreads();
    // plane p of the column is z = z0 - 1 + p (wrapped), held in ring slot p % kRingB.
    // Full rows: this thread's copies of every plane (16-byte u row chunks, 4-byte
    // x-halo values, 16-byte mu_local row chunks, kVecCopies in all over the block),
    // fixed per item: source without the plane offset, shared-memory destination in
    // slot 0, size in bytes (0: none).
    const float* csrc[kMaxCopies];
    unsigned cdst[kMaxCopies];
    int cbytes[kMaxCopies];
#pragma unroll
    for (int k = 0; k < kMaxCopies; ++k) {
      csrc[k] = ufield;
      cdst[k] = 0u;
      cbytes[k] = 0;
    }
    if constexpr (vec) {
#pragma unroll
      for (int k = 0; k < kMaxCopies; ++k) {
        const int q = threadIdx.x + k * kBlockB;
        if (q < kVecRows) {
          const int c = q / (kRowsB * 8), rem = q - c * (kRowsB * 8);
          const int row = rem >> 3, ch = rem & 7;
          csrc[k] = ufield + c * n + rowoff[row] + x0 + 4 * ch;
          cdst[k] = (unsigned)__cvta_generic_to_shared(ring + (c * kRowsB + row) * kRowF + kColX0 + 4 * ch);
          cbytes[k] = 16;
        } else if (q < kVecRows + kVecHalo) {
          const int h = q - kVecRows;
          const int c = h / (kRowsB * 2), rem = h - c * (kRowsB * 2);
          const int row = rem >> 1, side = rem & 1;
          csrc[k] = ufield + c * n + rowoff[row] + halo_x[side];
          cdst[k] = (unsigned)__cvta_generic_to_shared(
              ring + (c * kRowsB + row) * kRowF + (side ? kColX0 + kTileX : kColX0 - 1));
          cbytes[k] = 4;
        } else if (q < kVecCopies) {  // mu_local rows (no halo)
          const int m = q - kVecRows - kVecHalo;
          const int row = m >> 3, ch = m & 7;
          const int gy = min(y0 + row, P.ny - 1);
          csrc[k] = ufield + 3 * n + (long long)gy * P.nx + x0 + 4 * ch;
          cdst[k] = (unsigned)__cvta_generic_to_shared(ring + kPlaneU + row * kTileX + 4 * ch);
          cbytes[k] = 16;
        }
      }
    }
    long long zoff = (long long)wrap_index(z0 - 1, P.nz) * nxy;  // of the next plane to issue
    auto issue = [&](int p) {
      if (p < np) {
        const unsigned so = (unsigned)((p % kRingB) * kPlaneB * sizeof(float));
        if constexpr (vec) {
#pragma unroll
          for (int k = 0; k < kMaxCopies; ++k) {
            if (cbytes[k] == 16)
              asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(cdst[k] + so),
                           "l"(csrc[k] + zoff) : "memory");
            else if (cbytes[k] == 4)
              asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(cdst[k] + so),
                           "l"(csrc[k] + zoff) : "memory");
          }
        } else {
          float* slot = ring + (p % kRingB) * kPlaneB;
          for (int q = threadIdx.x; q < kScalarCopies; q += kBlockB) {
            if (q < 3 * kRowsB * (kTileX + 2)) {
              const int c = q / (kRowsB * (kTileX + 2)), rem = q - c * (kRowsB * (kTileX + 2));
              const int row = rem / (kTileX + 2), lx = rem - row * (kTileX + 2);
              cp_async4(slot + (c * kRowsB + row) * kRowF + kColX0 - 1 + lx,
                        ufield + c * n + zoff + rowoff[row] + wrap_index(x0 - 1 + lx, P.nx));
            } else {  // mu_local of the tile (clamped to the domain; unused outside)
              const int j = q - 3 * kRowsB * (kTileX + 2);
              const int row = j / kTileX, lx = j - row * kTileX;
              const int gx = min(x0 + lx, P.nx - 1), gy = min(y0 + row, P.ny - 1);
              cp_async4(slot + kPlaneU + j, ufield + 3 * n + zoff + (long long)gy * P.nx + gx);
            }
          }
        }
        zoff += nxy;
        if (zoff >= n) zoff -= n;
      }
      cp_async_commit();  // an empty group past the last plane keeps the count uniform
    };
#pragma unroll
    for (int p = 0; p < kRingB; ++p) issue(p);
    const int xa = x0 + kCells * tx, y = y0 + ty;
    const bool row_ok = y < P.ny;
    int nvalid = row_ok ? min(kCells, P.nx - xa) : 0;
    if (nvalid < 0) nvalid = 0;
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
    // u of the own cells on three planes, in three register sets whose roles (z - 1, z,
    // z + 1) rotate from plane to plane, so the march moves no registers
    float ua[3][kCells], ub[3][kCells], uc[3][kCells];
    cp_async_wait<kRingB - 2>();  // planes 0 and 1
    __syncthreads();
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      ldv(ring + 0 * kPlaneB + c * kRowsB * kRowF + hc, ua[c]);
      ldv(ring + 1 * kPlaneB + c * kRowsB * kRowF + hc, ub[c]);
    }
    // FP32 sums of the products over two planes, added to the float-float totals
    float ss = 0.0f, sd = 0.0f;
    // one plane of the march: pu, cu hold u at z - 1 and z, nu receives z + 1
    auto plane = [&](int i, const float (&pu)[3][kCells], const float (&cu)[3][kCells],
                     float (&nu)[3][kCells]) {
      cp_async_wait<kRingB - 3>();  // planes up to i + 2 have landed (this thread's copies)
      __syncthreads();              // ... everyone's; and everyone is done with plane i
      issue(i + kRingB);            // into the slot of plane i
      const float* S0 = ring + ((i + 1) % kRingB) * kPlaneB;  // plane z
      const float* SP = ring + ((i + 2) % kRingB) * kPlaneB;  // plane z + 1
      float mu[kCells];
      ldv(S0 + kPlaneU + ty * kTileX + kCells * tx, mu);
      // curl and divergence of the unscaled central differences, built component by
      // component: w = (d_y u_z - d_z u_y, d_z u_x - d_x u_z, d_x u_y - d_y u_x)
      float wx[kCells], wy[kCells], wz[kCells], dv[kCells];
#pragma unroll
      for (int j = 0; j < kCells; ++j) wx[j] = wy[j] = wz[j] = dv[j] = 0.0f;
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        const float* C0 = S0 + c * kRowsB * kRowF + hc;
        float ymv[kCells], ypv[kCells];
        ldv(SP + c * kRowsB * kRowF + hc, nu[c]);
        ldv(C0 - kRowF, ymv);
        ldv(C0 + kRowF, ypv);
        const float xl = C0[-1], xr = C0[kCells];
#pragma unroll
        for (int j = 0; j < kCells; ++j) {
          float right = j + 1 < kCells ? cu[c][j + 1] : xr;
          float left = j > 0 ? cu[c][j - 1] : xl;
          float dx_;
          if (P.bc_x) {
            if (own_r[j]) right = cu[c][j];
            if (own_l[j]) left = cu[c][j];
            dx_ = mul(sub(right, left), fx[j]);
          } else {
            dx_ = sub(right, left);
          }
          const float dy_ = sub(ypv[j], ymv[j]);
          const float dz_ = sub(nu[c][j], pu[c][j]);
          if (c == 0) {
            dv[j] = add(dv[j], dx_);
            wz[j] = sub(wz[j], dy_);
            wy[j] = add(wy[j], dz_);
          } else if (c == 1) {
            wz[j] = add(wz[j], dx_);
            dv[j] = add(dv[j], dy_);
            wx[j] = sub(wx[j], dz_);
          } else {
            wy[j] = sub(wy[j], dx_);
            wx[j] = add(wx[j], dy_);
            dv[j] = add(dv[j], dz_);
          }
        }
      }
#pragma unroll
      for (int j = 0; j < kCells; ++j) {
        if (j < nvalid) {
          ss = fma_(mu[j], fma_(wz[j], wz[j], fma_(wy[j], wy[j], mul(wx[j], wx[j]))), ss);
          sd = fma_(mu[j], mul(dv[j], dv[j]), sd);
        }
      }
      if (i & 1) {
        ff_add(acc[0], mul(ss, s2));
        ff_add(acc[1], mul(sd, s2));
        ss = sd = 0.0f;
      }
    };
    const int nzc = z1 - z0;
    for (int i = 0; i < nzc; i += 6) {  // period of the register roles (3) and of the sums (2)
      plane(i, ua, ub, uc);
      if (i + 1 < nzc) plane(i + 1, ub, uc, ua);
      if (i + 2 < nzc) plane(i + 2, uc, ua, ub);
      if (i + 3 < nzc) plane(i + 3, ua, ub, uc);
      if (i + 4 < nzc) plane(i + 4, ub, uc, ua);
      if (i + 5 < nzc) plane(i + 5, uc, ua, ub);
    }
    ff_add(acc[0], mul(ss, s2));  // an odd plane count leaves one plane's sums
    ff_add(acc[1], mul(sd, s2));
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
template <bool kVec>
int diag_b_grid() {
  int dev = 0, sms = 0, per_sm = 0;
  if (cudaFuncSetAttribute(k_diag_b<kVec>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)kDiagBSmem) != cudaSuccess ||
      cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_diag_b<kVec>, kBlockB, kDiagBSmem) !=
          cudaSuccess) {
    cudaGetLastError();
    return kDiagBlocks;
  }
  const int g = sms * per_sm;
  return g < 1 ? 1 : (g > kDiagBlocks ? kDiagBlocks : g);
}

// Pass B into pb; returns its grid (the number of records written).
int launch_b(const DomainConst& P, const float* ufield, double* pb, cudaStream_t s) {
  if (P.nx % kTileX == 0) {
    const int g = diag_b_grid<true>();
    k_diag_b<true><<<g, kBlockB, kDiagBSmem, s>>>(P, ufield, pb);
    return g;
  }
  const int g = diag_b_grid<false>();
  k_diag_b<false><<<g, kBlockB, kDiagBSmem, s>>>(P, ufield, pb);
  return g;
}

// Fixed-order FP64 reduction of the block records of both passes (nblocks records of
// pass A or R, nblocks_b <= nblocks of pass B; one block of kBlock threads): thread t
// folds blocks t, t + kBlock, ... of every quantity, then a
// shared-memory tree combines the threads in a fixed pattern. The reference density
// and energy are added back once per cell at the end, the maximum Mach number is the
// root of the maximum of Mach^2 and the maximum CFL number the maximum speed / c.
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
    if (t == 9) v = sqrt(v);
    if (t == 10) v = v / (double)P.c;
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
  const int gb = launch_b(P, ufield, pb, s);
  k_diag_final<<<1, kBlock, 0, s>>>(P, pa, pb, kDiagBlocks, gb, out16);
  return cudaGetLastError();
}

cudaError_t launch_diag_records(const DomainConst& P, const float* rec, long long nrec,
                                const float* ufield, double* partials, double* out16,
                                cudaStream_t s) {
  double* pa = partials;
  double* pb = partials + (long long)kDiagBlocks * kDiagA;
  k_diag_records<<<kDiagBlocks, kBlock, 0, s>>>(rec, nrec, pa);
  const int gb = launch_b(P, ufield, pb, s);
  k_diag_final<<<1, kBlock, 0, s>>>(P, pa, pb, kDiagBlocks, gb, out16);
  return cudaGetLastError();
}

}  // namespace lbm
