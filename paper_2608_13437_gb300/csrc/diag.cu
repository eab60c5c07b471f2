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
// (x by y) over kZChunk planes; a persistent grid of kDiagBlocks blocks takes them
// in a fixed order (block b: items b, b + grid, ...), so sums are reproducible. Each
// thread marches up its (x, y) column: u at z - 1, z and z + 1 stays in registers, so
// every value of the field is read from DRAM about once (plus one halo plane per
// chunk); the x and y neighbours are loads of lines the block (or its neighbour
// column, at about the same z) has just brought into L1 / L2.
constexpr int kTileX = 32, kTileY = kBlock / 32, kZChunk = 32;

__global__ void __launch_bounds__(kBlock, 4) k_diag_b(const DomainConst P,
                                                   const float* __restrict__ ufield,
                                                   double* __restrict__ partials) {
  FF acc[2] = {{0.0f, 0.0f}, {0.0f, 0.0f}};
  const long long n = P.ncell;
  const float inv_dx = (float)(1.0 / P.dx64), inv_2dx = (float)(0.5 / P.dx64);
  const float* __restrict__ U0 = ufield;
  const float* __restrict__ U1 = ufield + n;
  const float* __restrict__ U2 = ufield + 2 * n;
  const float* __restrict__ MU = ufield + 3 * n;
  const int cols_x = (P.nx + kTileX - 1) / kTileX, cols_y = (P.ny + kTileY - 1) / kTileY;
  const int chunks = (P.nz + kZChunk - 1) / kZChunk;
  const long long items = (long long)cols_x * cols_y * chunks;
  const long long nxy = (long long)P.nx * P.ny;
  const int tx = threadIdx.x % kTileX, ty = threadIdx.x / kTileX;
  for (long long it = blockIdx.x; it < items; it += gridDim.x) {
    const int cx = (int)(it % cols_x);
    const long long r = it / cols_x;
    const int cy = (int)(r % cols_y), cz = (int)(r / cols_y);
    const int x = cx * kTileX + tx, y = cy * kTileY + ty;
    if (x >= P.nx || y >= P.ny) continue;
    // x neighbours (one-sided at held ends) and y neighbours (periodic)
    int xh, xl;
    float wxd = inv_2dx;
    if (P.bc_x) {
      xh = x < P.nx - 1 ? x + 1 : x;
      xl = x > 0 ? x - 1 : x;
      const int span = (x < P.nx - 1) + (x > 0);
      wxd = span == 2 ? inv_2dx : (span == 1 ? inv_dx : 0.0f);
    } else {
      xh = x + 1 < P.nx ? x + 1 : 0;
      xl = x > 0 ? x - 1 : P.nx - 1;
    }
    const long long yh = (y + 1 < P.ny ? y + 1 : 0) * (long long)P.nx;
    const long long yl = (y > 0 ? y - 1 : P.ny - 1) * (long long)P.nx;
    const long long col = x + (long long)y * P.nx;  // cell of the column at z = 0
    const int z0 = cz * kZChunk, z1 = min(z0 + kZChunk, P.nz);
    // u at z - 1, z, z + 1 and mu_local at z in registers; the loads of u at z + 2 and
    // of mu_local at z + 1 are issued one plane ahead, so two planes' DRAM reads are in
    // flight per thread
    const long long zlo = (z0 > 0 ? z0 - 1 : P.nz - 1) * nxy;
    long long c = z0 * nxy + col;
    const long long c1 = (z0 + 1 < P.nz ? c + nxy : col);
    float pu0 = U0[zlo + col], pu1 = U1[zlo + col], pu2 = U2[zlo + col];
    float cu0 = U0[c], cu1 = U1[c], cu2 = U2[c];
    float nu0 = U0[c1], nu1 = U1[c1], nu2 = U2[c1];
    float mu_loc = MU[c];
    for (int z = z0; z < z1; ++z, c += nxy) {
      const bool more = z + 1 < z1;
      float qu0 = 0.0f, qu1 = 0.0f, qu2 = 0.0f, mu_n = 0.0f;
      if (more) {
        const long long c2 = (z + 2 < P.nz ? c + 2 * nxy : (z + 2 - P.nz) * nxy + col);
        qu0 = U0[c2];
        qu1 = U1[c2];
        qu2 = U2[c2];
        mu_n = MU[c + nxy];
      }
      const long long plane = c - col;  // z * nx * ny
      const long long ch = plane + y * (long long)P.nx + xh, cl = plane + y * (long long)P.nx + xl;
      const long long cyh = plane + yh + x, cyl = plane + yl + x;
      float g[3][3];  // g[a][b] = d_a u_b
      g[0][0] = mul(sub(U0[ch], U0[cl]), wxd);
      g[0][1] = mul(sub(U1[ch], U1[cl]), wxd);
      g[0][2] = mul(sub(U2[ch], U2[cl]), wxd);
      g[1][0] = mul(sub(U0[cyh], U0[cyl]), inv_2dx);
      g[1][1] = mul(sub(U1[cyh], U1[cyl]), inv_2dx);
      g[1][2] = mul(sub(U2[cyh], U2[cyl]), inv_2dx);
      g[2][0] = mul(sub(nu0, pu0), inv_2dx);
      g[2][1] = mul(sub(nu1, pu1), inv_2dx);
      g[2][2] = mul(sub(nu2, pu2), inv_2dx);
      const float wx = sub(g[1][2], g[2][1]), wy = sub(g[2][0], g[0][2]), wz = sub(g[0][1], g[1][0]);
      const float div = add(add(g[0][0], g[1][1]), g[2][2]);
      ff_add(acc[0], mul(mu_loc, fma_(wz, wz, fma_(wy, wy, mul(wx, wx)))));
      ff_add(acc[1], mul(mu_loc, mul(div, div)));
      pu0 = cu0; pu1 = cu1; pu2 = cu2;
      cu0 = nu0; cu1 = nu1; cu2 = nu2;
      nu0 = qu0; nu1 = qu1; nu2 = qu2;
      mu_loc = mu_n;
    }
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
  k_diag_b<<<kDiagBlocks, kBlock, 0, s>>>(P, ufield, pb);
  k_diag_final<<<1, kBlock, 0, s>>>(P, pa, pb, kDiagBlocks, out16);
  return cudaGetLastError();
}

cudaError_t launch_diag_records(const DomainConst& P, const float* rec, long long nrec,
                                const float* ufield, double* partials, double* out16,
                                cudaStream_t s) {
  double* pa = partials;
  double* pb = partials + (long long)kDiagBlocks * kDiagA;
  k_diag_records<<<kDiagBlocks, kBlock, 0, s>>>(rec, nrec, pa);
  k_diag_b<<<kDiagBlocks, kBlock, 0, s>>>(P, ufield, pb);
  k_diag_final<<<1, kBlock, 0, s>>>(P, pa, pb, kDiagBlocks, out16);
  return cudaGetLastError();
}

}  // namespace lbm
