// FP64 diagnostics of the current state (Sec. 3.2, Eq. 7): conservation sums,
// <rho|u|^2/2>, <mu_local |curl u|^2>, 4/3 <mu_local (div u)^2>, extrema and a
// non-finite count. Pass A decodes every cell (FP64) and keeps u and mu_local in
// a scratch field; pass B takes central differences of u from that field; each
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

template <typename S>
__global__ void __launch_bounds__(kBlock) k_diag_a(const DomainConst P, int parity,
                                                   const S* __restrict__ pop,
                                                   const float* __restrict__ ghost,
                                                   double* __restrict__ ufield,
                                                   double* __restrict__ partials) {
  double acc[kDiagA];
  for (int j = 0; j < 7; ++j) acc[j] = 0.0;
  acc[7] = acc[8] = 0.0;            // max mach, max cfl
  acc[9] = acc[10] = INFINITY;      // min rho, min T
  acc[11] = acc[12] = 0.0;          // spare sums (zero)
  for (long long cell = blockIdx.x * (long long)blockDim.x + threadIdx.x; cell < P.ncell;
       cell += (long long)gridDim.x * blockDim.x) {
    const int x = (int)(cell % P.nx);
    const long long yz = cell / P.nx;
    const CellIndex c = make_index(P, x, (int)(yz % P.ny), (int)(yz / P.ny));
    double Q[kF];
    bool finite = true;
    for (int k = 0; k < kF; ++k) {
      double s = 0.0;
      for (int i = 0; i < kQ; ++i) {
        const double v = from_ghost(P, c, i)
                             ? (double)ghost_value(P, ghost, c, k, i)
                             : Codec<S>::dec64(pop[read_pos(P, c, parity, k, i)], (double)P.scale[k]);
        s += v;
      }
      Q[k] = s;
    }
    Q[0] += (double)P.rho_ref;
    Q[4] += (double)P.E_ref;
    for (int k = 0; k < kF; ++k) finite = finite && isfinite(Q[k]);
    Prim<double> s;
    closure<double>(Q, P.gm1_64, P.mu64, 0.0, 0.0, P.inv_T_ref64, P.sutherland, s);
    acc[0] += Q[0];
    acc[1] += Q[1];
    acc[2] += Q[2];
    acc[3] += Q[3];
    acc[4] += Q[4];
    acc[5] += 0.5 * (s.m[0] * s.u[0] + s.m[1] * s.u[1] + s.m[2] * s.u[2]);
    acc[6] += finite ? 0.0 : 1.0;
    const double a = sqrt((P.gm1_64 + 1.0) * s.T);
    const double umag = sqrt(s.u[0] * s.u[0] + s.u[1] * s.u[1] + s.u[2] * s.u[2]);
    const double umax = fmax(fabs(s.u[0]), fmax(fabs(s.u[1]), fabs(s.u[2])));
    if (finite) {
      acc[7] = fmax(acc[7], umag / a);
      acc[8] = fmax(acc[8], (umax + a) * P.dt64 / P.dx64);  // (|u_a| + a) dt / dx
      acc[9] = fmin(acc[9], s.rho);
      acc[10] = fmin(acc[10], s.T);
    }
    ufield[cell] = s.u[0];
    ufield[P.ncell + cell] = s.u[1];
    ufield[2 * P.ncell + cell] = s.u[2];
    ufield[3 * P.ncell + cell] = s.mu_T;
  }
  // partial layout: 9 sums (rho, mx, my, mz, E, ke, nonfinite, 0, 0), 2 maxima, 2 minima
  double v[kDiagA] = {acc[0], acc[1], acc[2], acc[3], acc[4], acc[5], acc[6], acc[11], acc[12],
                      acc[7], acc[8], acc[9], acc[10]};
  block_reduce<kDiagA>(v, 9, 2, partials + (long long)blockIdx.x * kDiagA);
}

__global__ void __launch_bounds__(kBlock) k_diag_b(const DomainConst P,
                                                   const double* __restrict__ ufield,
                                                   double* __restrict__ partials) {
  double acc[2] = {0.0, 0.0};
  const long long n = P.ncell;
  for (long long cell = blockIdx.x * (long long)blockDim.x + threadIdx.x; cell < n;
       cell += (long long)gridDim.x * blockDim.x) {
    const int x = (int)(cell % P.nx);
    const long long yz = cell / P.nx;
    const int y = (int)(yz % P.ny), z = (int)(yz / P.ny);
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
        g[a][b] = span > 0.0 ? (ufield[b * n + hi] - ufield[b * n + lo]) / (span * P.dx64)
                             : 0.0;
    }
    const double wx = g[1][2] - g[2][1], wy = g[2][0] - g[0][2], wz = g[0][1] - g[1][0];
    const double div = g[0][0] + g[1][1] + g[2][2];
    const double mu_loc = ufield[3 * n + cell];
    acc[0] += mu_loc * (wx * wx + wy * wy + wz * wz);
    acc[1] += mu_loc * div * div;
  }
  double v[2] = {acc[0], acc[1]};
  block_reduce<2>(v, 2, 0, partials + (long long)blockIdx.x * 2);
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

}  // namespace

cudaError_t launch_diag(const DomainConst& P, int store, int parity, const void* pop,
                        const float* ghost, double* ufield, double* partials, double* out16,
                        cudaStream_t s) {
  const int nb = kDiagBlocks;
  double* pa = partials;
  double* pb = partials + (long long)nb * kDiagA;
  switch (store) {
    case 0: k_diag_a<float><<<nb, kBlock, 0, s>>>(P, parity, (const float*)pop, ghost, ufield, pa); break;
    case 1: k_diag_a<__half><<<nb, kBlock, 0, s>>>(P, parity, (const __half*)pop, ghost, ufield, pa); break;
    default: k_diag_a<__nv_bfloat16><<<nb, kBlock, 0, s>>>(P, parity, (const __nv_bfloat16*)pop, ghost, ufield, pa); break;
  }
  k_diag_b<<<nb, kBlock, 0, s>>>(P, ufield, pb);
  k_diag_final<<<1, 32, 0, s>>>(pa, pb, nb, out16);
  return cudaGetLastError();
}

}  // namespace lbm
