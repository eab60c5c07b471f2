// Diagnostics of the current state (Sec. 3.2, Eq. 7): conservation sums,
// <rho|u|^2/2>, <mu_local |curl u|^2>, 4/3 <mu_local (div u)^2>, extrema and a
// non-finite count. Per-cell work runs in FP32 exactly as in the step; FP64 is used
// for the sums, extrema and differences. Pass A decodes every cell and keeps u and
// mu_local in a scratch field (4 floats per cell); pass B takes central differences of
// u from that field; each
// pass writes one partial per block (warp shuffles, then shared memory), and a
// single block reduces the partials in a fixed order, so results are
// reproducible run to run.
#include "lbm_internal.h"

namespace lbm {

namespace {

constexpr int kBlock = 256;

__device__ __forceinline__ double warp_sum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ double warp_max(double v) {
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_down_sync(0xffffffffu, v, o));
  return v;
}
__device__ __forceinline__ double warp_min(double v) {
  for (int o = 16; o > 0; o >>= 1) v = fmin(v, __shfl_down_sync(0xffffffffu, v, o));
  return v;
}

// Reduces n values per thread (sums for j < nsum, maxima for nsum <= j < nsum+nmax,
// minima after) over the block into out[0..n).
template <int N>
__device__ void block_reduce(double (&v)[N], int nsum, int nmax, double* out) {
  __shared__ double sh[kBlock / 32][N];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int j = 0; j < N; ++j) {
    const double r = j < nsum ? warp_sum(v[j]) : (j < nsum + nmax ? warp_max(v[j]) : warp_min(v[j]));
    if (lane == 0) sh[warp][j] = r;
  }
  __syncthreads();
  if (threadIdx.x < N) {
    const int j = threadIdx.x;
    double r = sh[0][j];
    for (int w = 1; w < kBlock / 32; ++w)
      r = j < nsum ? r + sh[w][j] : (j < nsum + nmax ? fmax(r, sh[w][j]) : fmin(r, sh[w][j]));
    out[j] = r;
  }
}

// Pass A: per cell, the step's own FP32 decode, moments and closure; FP64 only for the
// running sums, extrema and counts. Writes u and mu_local (FP32) for pass B.
template <typename S, int PARITY, bool HELD>
__global__ void __launch_bounds__(kBlock) k_diag_a(const DomainConst P, const S* __restrict__ pop,
                                                   const float* __restrict__ ghost,
                                                   float* __restrict__ ufield,
                                                   double* __restrict__ partials) {
  double acc[kDiagA];
  for (int j = 0; j < 9; ++j) acc[j] = 0.0;  // rho mx my mz E ke nonfinite, 2 spare
  acc[9] = acc[10] = 0.0;                    // max mach, max cfl
  acc[11] = acc[12] = INFINITY;              // min rho, min T
  const double c64 = P.dx64 / P.dt64;
  for (long long cell = blockIdx.x * (long long)blockDim.x + threadIdx.x; cell < P.ncell;
       cell += (long long)gridDim.x * blockDim.x) {
    int x, y, z;
    cell_xyz(P, cell, x, y, z);
    const CellIndex c = make_index(P, x, y, z);
    float d[kF][kQ];
    load_cell<PARITY, HELD, S>(P, pop, ghost, c, d);
    float D[kF];
    bool finite = true;
#pragma unroll
    for (int k = 0; k < kF; ++k) {
      float t = d[k][0];
#pragma unroll
      for (int i = 1; i < kQ; ++i) t = add(t, d[k][i]);
      D[k] = t;
      finite = finite && isfinite(t);
    }
    float Q[kF];
#pragma unroll
    for (int k = 0; k < kF; ++k) Q[k] = D[k];
    Q[0] = add(Q[0], P.rho_ref);
    Q[4] = add(Q[4], P.E_ref);
    Prim<float> s;
    closure<float>(Q, P.gm1, P.mu, P.visc0, P.heat0, P.inv_T_ref, P.sutherland, s);
    // reference + deviation in FP64, so the totals keep the deviations' precision
    acc[0] += (double)P.rho_ref + (double)D[0];
    acc[1] += (double)D[1];
    acc[2] += (double)D[2];
    acc[3] += (double)D[3];
    acc[4] += (double)P.E_ref + (double)D[4];
    acc[5] += 0.5 * ((double)s.m[0] * s.u[0] + (double)s.m[1] * s.u[1] + (double)s.m[2] * s.u[2]);
    acc[6] += finite ? 0.0 : 1.0;
    if (finite) {
      const double a = sqrt((P.gm1_64 + 1.0) * (double)s.T);
      const double ux = s.u[0], uy = s.u[1], uz = s.u[2];
      acc[9] = fmax(acc[9], sqrt(ux * ux + uy * uy + uz * uz) / a);
      acc[10] = fmax(acc[10], (fmax(fabs(ux), fmax(fabs(uy), fabs(uz))) + a) / c64);  // (|u_a|+a) dt/dx
      acc[11] = fmin(acc[11], (double)s.rho);
      acc[12] = fmin(acc[12], (double)s.T);
    }
    ufield[cell] = s.u[0];
    ufield[P.ncell + cell] = s.u[1];
    ufield[2 * P.ncell + cell] = s.u[2];
    ufield[3 * P.ncell + cell] = s.mu_T;
  }
  block_reduce<kDiagA>(acc, 9, 2, partials + (long long)blockIdx.x * kDiagA);
}

// Pass B: central differences of u (FP64 differences of the FP32 field), weighted by
// mu_local, summed in FP64.
__global__ void __launch_bounds__(kBlock) k_diag_b(const DomainConst P,
                                                   const float* __restrict__ ufield,
                                                   double* __restrict__ partials) {
  double acc[2] = {0.0, 0.0};
  const long long n = P.ncell;
  for (long long cell = blockIdx.x * (long long)blockDim.x + threadIdx.x; cell < n;
       cell += (long long)gridDim.x * blockDim.x) {
    int x, y, z;
    cell_xyz(P, cell, x, y, z);
    const CellIndex c = make_index(P, x, y, z);
    double g[3][3];  // g[a][b] = d_a u_b
    for (int a = 0; a < 3; ++a) {
      long long hi = c.nb[2 * a + 1], lo = c.nb[2 * a + 2];
      double span = 2.0;
      if (a == 0 && P.bc_x) {
        hi = (x < P.nx - 1) ? c.nb[1] : c.own;
        lo = (x > 0) ? c.nb[2] : c.own;
        span = (double)((x < P.nx - 1) + (x > 0));
      }
      for (int b = 0; b < 3; ++b)
        g[a][b] = span > 0.0 ? ((double)ufield[b * n + hi] - (double)ufield[b * n + lo]) / (span * P.dx64)
                             : 0.0;
    }
    const double wx = g[1][2] - g[2][1], wy = g[2][0] - g[0][2], wz = g[0][1] - g[1][0];
    const double div = g[0][0] + g[1][1] + g[2][2];
    const double mu_loc = ufield[3 * n + cell];
    acc[0] += mu_loc * (wx * wx + wy * wy + wz * wz);
    acc[1] += mu_loc * div * div;
  }
  block_reduce<2>(acc, 2, 0, partials + (long long)blockIdx.x * 2);
}

// Fixed-order reduction of the partials of both passes (one block).
__global__ void k_diag_final(const double* __restrict__ pa, const double* __restrict__ pb,
                             int nblocks, double* __restrict__ out) {
  if (threadIdx.x >= kDiagA + 2) return;
  const int j = threadIdx.x;
  if (j < kDiagA) {
    double r = pa[j];
    for (int b = 1; b < nblocks; ++b) {
      const double v = pa[(long long)b * kDiagA + j];
      r = j < 9 ? r + v : (j < 11 ? fmax(r, v) : fmin(r, v));
    }
    out[j] = r;
  } else {
    double r = 0.0;
    for (int b = 0; b < nblocks; ++b) r += pb[(long long)b * 2 + (j - kDiagA)];
    out[j] = r;
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
  k_diag_final<<<1, 32, 0, s>>>(pa, pb, kDiagBlocks, out16);
  return cudaGetLastError();
}

}  // namespace lbm
