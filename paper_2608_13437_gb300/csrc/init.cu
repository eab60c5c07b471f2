// Initial states (Sec. 3): TGV, Riemann problem, caller fields (rho, u, p) or caller
// zeroth moments (all 14 fields). Each cell gets the linear equilibrium of its state
// (tau = q = 0 unless given), computed in FP64 and stored as the deviation from
// w_i Q_ref in the storage type.
#include "lbm_internal.h"

namespace lbm {

namespace {

// Zeroth moments Q of the initial state of the cell: (rho, rho u, E) with tau = q = 0
// for the TGV, Riemann and (rho, u, p)-field initial states, or all 14 fields given.
__device__ void initial_Q(const DomainConst& P, const InitSpec& sp, int x, int y, int z,
                          long long cell, double Q[kF]) {
  for (int k = 0; k < kF; ++k) Q[k] = 0.0;
  if (sp.kind == 3) {
    const long long n = P.ncell;
    for (int k = 0; k < kF; ++k)
      Q[k] = sp.fields_f64 ? static_cast<const double*>(sp.fields)[k * n + cell]
                           : (double)static_cast<const float*>(sp.fields)[k * n + cell];
    return;
  }
  double rho, u[3], p;
  if (sp.kind == 0) {
    // Supersonic TGV (Sec. 3.2), nodes at (x, y, z) dx.
    const double X = x * sp.dx, Y = y * sp.dx, Z = z * sp.dx;
    const double p0 = sp.rho0 * sp.U0 * sp.U0 / (sp.gamma * sp.M0 * sp.M0);
    const double T0 = p0 / sp.rho0;
    u[0] = sp.U0 * sin(X) * cos(Y) * cos(Z);
    u[1] = -sp.U0 * cos(X) * sin(Y) * cos(Z);
    u[2] = 0.0;
    p = p0 + sp.rho0 * sp.U0 * sp.U0 / 16.0 * (cos(2.0 * X) + cos(2.0 * Y)) * (cos(2.0 * Z) + 2.0);
    rho = p / T0;
  } else if (sp.kind == 1) {
    const int idx = sp.axis == 0 ? x : (sp.axis == 1 ? y : z);
    const double* s = idx < sp.split ? sp.left : sp.right;
    rho = s[0];
    u[0] = u[1] = u[2] = 0.0;
    u[sp.axis] = s[1];
    p = s[2];
  } else {
    const long long n = P.ncell;
    if (sp.fields_f64) {
      const double* f = static_cast<const double*>(sp.fields);
      rho = f[cell]; u[0] = f[n + cell]; u[1] = f[2 * n + cell]; u[2] = f[3 * n + cell]; p = f[4 * n + cell];
    } else {
      const float* f = static_cast<const float*>(sp.fields);
      rho = f[cell]; u[0] = f[n + cell]; u[1] = f[2 * n + cell]; u[2] = f[3 * n + cell]; p = f[4 * n + cell];
    }
  }
  Q[0] = rho;
  for (int a = 0; a < 3; ++a) Q[1 + a] = rho * u[a];
  Q[4] = p / (sp.gamma - 1.0) + 0.5 * rho * (u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
}

// Deviations d_{k,i} = feq_{k,i}(Q) - w_i Q_ref,k of the linear equilibrium of Q.
__device__ void equilibrium_dev(const DomainConst& P, const InitSpec& sp, const double Q[kF],
                                double dev[kF][kQ]) {
  Prim<double> s;
  closure<double>(Q, sp.gamma - 1.0, sp.mu, sp.mu / sp.tau_R, sp.kappa / sp.tau_q, sp.inv_T_ref,
                  sp.sutherland, s);
  const double hic = 0.5 / sp.c;
  for (int k = 0; k < kF; ++k) {
    double fx, fy, fz;
    field_flux<double>(k, s, fx, fy, fz);
    const double qr = (k == 0) ? (double)P.rho_ref : (k == 4 ? (double)P.E_ref : 0.0);
    const double D = Q[k] - qr;
    dev[k][0] = 0.25 * D;
    dev[k][1] = 0.125 * D + hic * fx;
    dev[k][2] = 0.125 * D - hic * fx;
    dev[k][3] = 0.125 * D + hic * fy;
    dev[k][4] = 0.125 * D - hic * fy;
    dev[k][5] = 0.125 * D + hic * fz;
    dev[k][6] = 0.125 * D - hic * fz;
  }
}

template <typename S>
__global__ void k_init(const DomainConst P, const InitSpec sp, int mode, S* __restrict__ pop,
                       float* __restrict__ ghost, unsigned* __restrict__ maxbits) {
  const long long n = P.ncell;
  const long long planes = (long long)P.ny * P.nz;
  for (long long cell = blockIdx.x * (long long)blockDim.x + threadIdx.x; cell < n;
       cell += (long long)gridDim.x * blockDim.x) {
    int x, y, z;
    cell_xyz(P, cell, x, y, z);
    const long long yz = (long long)y + (long long)P.ny * z;  // ghost-plane index
    double Q[kF];
    initial_Q(P, sp, x, y, z, cell, Q);
    double dev[kF][kQ];
    equilibrium_dev(P, sp, Q, dev);
    if (mode == 0) {
      for (int k = 0; k < kF; ++k) {
        float m = 0.0f;
        for (int i = 0; i < kQ; ++i) m = fmaxf(m, (float)fabs(dev[k][i]));
        atomicMax(&maxbits[k], __float_as_uint(m));  // order of non-negative floats = order of bits
      }
      continue;
    }
    for (int k = 0; k < kF; ++k)
      for (int i = 0; i < kQ; ++i)
        pop[pop_index(cell, k, i)] = Codec<S>::enc((float)dev[k][i], P.inv_scale[k]);
    if (P.bc_x && ghost) {
      const long long plane = yz;
      if (x == 0)
        for (int k = 0; k < kF; ++k) ghost[(0 * kF + k) * planes + plane] = (float)dev[k][1];
      if (x == P.nx - 1)
        for (int k = 0; k < kF; ++k) ghost[(1LL * kF + k) * planes + plane] = (float)dev[k][2];
    }
  }
}

constexpr int kMeanBlocks = (kFieldSumDoubles - 2) / 2, kMeanThreads = 256;

// Sums of rho and E of the caller's fields, in a fixed order (per thread, then a
// shared-memory tree per block, then the blocks in order), so Q_ref is reproducible.
__global__ void __launch_bounds__(kMeanThreads) k_field_sums(const DomainConst P, const InitSpec sp,
                                                             double* __restrict__ partials) {
  __shared__ double sh[2][kMeanThreads];
  double s_rho = 0.0, s_E = 0.0;
  for (long long cell = blockIdx.x * (long long)blockDim.x + threadIdx.x; cell < P.ncell;
       cell += (long long)gridDim.x * blockDim.x) {
    double Q[kF];
    initial_Q(P, sp, 0, 0, 0, cell, Q);
    s_rho += Q[0];
    s_E += Q[4];
  }
  sh[0][threadIdx.x] = s_rho;
  sh[1][threadIdx.x] = s_E;
  __syncthreads();
  for (int half = kMeanThreads / 2; half > 0; half >>= 1) {
    if (threadIdx.x < half) {
      sh[0][threadIdx.x] += sh[0][threadIdx.x + half];
      sh[1][threadIdx.x] += sh[1][threadIdx.x + half];
    }
    __syncthreads();
  }
  if (threadIdx.x < 2) partials[2 * blockIdx.x + threadIdx.x] = sh[threadIdx.x][0];
}

__global__ void k_field_sums_final(const double* __restrict__ partials, int nblocks,
                                   double* __restrict__ sums) {
  if (threadIdx.x >= 2) return;
  double r = 0.0;
  for (int b = 0; b < nblocks; ++b) r += partials[2 * b + threadIdx.x];
  sums[threadIdx.x] = r;
}

int grid_for(long long n, int block) {
  long long g = (n + block - 1) / block;
  if (g > 152LL * 32) g = 152LL * 32;
  return (int)(g < 1 ? 1 : g);
}

}  // namespace

cudaError_t launch_init(const DomainConst& P, int store, const InitSpec& spec, int mode, void* pop,
                        float* ghost, unsigned* maxbits, cudaStream_t s) {
  const int block = 128;
  const int grid = grid_for(P.ncell, block);
  switch (store) {
    case 0: k_init<float><<<grid, block, 0, s>>>(P, spec, mode, static_cast<float*>(pop), ghost, maxbits); break;
    case 1: k_init<__half><<<grid, block, 0, s>>>(P, spec, mode, static_cast<__half*>(pop), ghost, maxbits); break;
    default: k_init<__nv_bfloat16><<<grid, block, 0, s>>>(P, spec, mode, static_cast<__nv_bfloat16*>(pop), ghost, maxbits); break;
  }
  return cudaGetLastError();
}

cudaError_t launch_field_means(const DomainConst& P, const InitSpec& spec, double* sums,
                               cudaStream_t s) {
  // sums holds 2 results followed by 2 * kMeanBlocks partials
  double* partials = sums + 2;
  k_field_sums<<<kMeanBlocks, kMeanThreads, 0, s>>>(P, spec, partials);
  k_field_sums_final<<<1, 32, 0, s>>>(partials, kMeanBlocks, sums);
  return cudaGetLastError();
}

}  // namespace lbm
