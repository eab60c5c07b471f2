// Outputs of the current state through the AA read map of its parity: per-cell
// moments (float-float sums) and primitives as the step computes them, the sensor
// exactly as the next step computes it, canonical population arrays in and out, and
// raw slot planes.
#include "diag_device.cuh"
#include "lbm_internal.h"

namespace lbm {

namespace {

__device__ __forceinline__ void decompose(const DomainConst& P, long long cell, int& x, int& y,
                                          int& z) {
  cell_xyz(P, cell, x, y, z);
}

template <typename S>
__device__ __forceinline__ double read_dev64(const DomainConst& P, const S* pop, const float* ghost,
                                             const CellIndex& c, int parity, int k, int i) {
  if (from_ghost(P, c, i)) return (double)ghost_value(P, ghost, c, k, i);
  return Codec<S>::dec64(pop[read_pos(P, c, parity, k, i)], (double)P.scale[k]);
}

// Moments of cells [c0, c0 + cnt) through the AA read map of the step's parity, from
// the step's own loads and FP32 decode. LBM_MOM_Q: per field a float-float sum of the
// seven populations and the reference (two-sum, about 48 significant bits), widened to
// the output type. LBM_MOM_PRIM: the primitives exactly as the step computes them (its
// FP32 sums and closure). No FP64 arithmetic: FP64 here is only an output format.
template <typename S, int PARITY, bool HELD>
__global__ void k_moments(const DomainConst P, const S* __restrict__ pop,
                          const float* __restrict__ ghost, int which, void* out, int out_f64,
                          long long c0, long long cnt) {
  for (long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x; r < cnt;
       r += (long long)gridDim.x * blockDim.x) {
    const long long cell = c0 + r;
    int x, y, z;
    decompose(P, cell, x, y, z);
    const CellIndex c = make_index(P, x, y, z);
    float d[kF][kQ];
    load_cell<PARITY, HELD, S>(P, pop, ghost, c, d);
    if (which == 1) {
      float Q[kF];
#pragma unroll
      for (int k = 0; k < kF; ++k) {
        float t = d[k][0];
#pragma unroll
        for (int i = 1; i < kQ; ++i) t = add(t, d[k][i]);
        Q[k] = t;
      }
      Q[0] = add(Q[0], P.rho_ref);
      Q[4] = add(Q[4], P.E_ref);
      Prim<float> s;
      closure<float>(Q, P.gm1, P.mu, P.visc0, P.heat0, P.inv_T_ref, P.sutherland, s);
      const float v[6] = {s.rho, s.u[0], s.u[1], s.u[2], s.T, s.p};
#pragma unroll
      for (int j = 0; j < 6; ++j) {
        if (out_f64) static_cast<double*>(out)[(long long)j * cnt + r] = (double)v[j];
        else static_cast<float*>(out)[(long long)j * cnt + r] = v[j];
      }
    } else {
#pragma unroll
      for (int k = 0; k < kF; ++k) {
        FF a = {d[k][0], 0.0f};
#pragma unroll
        for (int i = 1; i < kQ; ++i) ff_add(a, d[k][i]);
        if (k == 0) ff_add(a, P.rho_ref);
        if (k == 4) ff_add(a, P.E_ref);
        if (out_f64) static_cast<double*>(out)[(long long)k * cnt + r] = ff_value(a);
        else static_cast<float*>(out)[(long long)k * cnt + r] = add(a.hi, a.lo);
      }
    }
  }
}

template <typename S>
void launch_moments_t(const DomainConst& P, int parity, const S* pop, const float* ghost, int which,
                      void* out, int out_f64, long long c0, long long cnt, int grid, int block,
                      cudaStream_t s) {
  if (P.bc_x) {
    if (parity) k_moments<S, 1, true><<<grid, block, 0, s>>>(P, pop, ghost, which, out, out_f64, c0, cnt);
    else k_moments<S, 0, true><<<grid, block, 0, s>>>(P, pop, ghost, which, out, out_f64, c0, cnt);
  } else {
    if (parity) k_moments<S, 1, false><<<grid, block, 0, s>>>(P, pop, ghost, which, out, out_f64, c0, cnt);
    else k_moments<S, 0, false><<<grid, block, 0, s>>>(P, pop, ghost, which, out, out_f64, c0, cnt);
  }
}

template <typename S>
__global__ void k_sensor(const DomainConst P, int parity, const S* __restrict__ pop,
                         const float* __restrict__ ghost, void* out, int out_f64, long long c0,
                         long long cnt) {
  for (long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x; r < cnt;
       r += (long long)gridDim.x * blockDim.x) {
    const long long cell = c0 + r;
    int x, y, z;
    decompose(P, cell, x, y, z);
    const CellIndex c = make_index(P, x, y, z);
    float d[kF][kQ];
    if (parity) {
      if (P.bc_x) load_cell<1, true, S>(P, pop, ghost, c, d);
      else load_cell<1, false, S>(P, pop, ghost, c, d);
    } else {
      if (P.bc_x) load_cell<0, true, S>(P, pop, ghost, c, d);
      else load_cell<0, false, S>(P, pop, ghost, c, d);
    }
    SensorOut so;
    collide_cell<true>(P, d, &so);
    const double v[3] = {(double)so.theta_dt / (double)P.dt, (double)so.chi, (double)so.omega_h};
    for (int j = 0; j < 3; ++j) {
      if (out_f64) static_cast<double*>(out)[(long long)j * cnt + r] = v[j];
      else static_cast<float*>(out)[(long long)j * cnt + r] = (float)v[j];
    }
  }
}

__device__ __forceinline__ double weight(int i) { return i == 0 ? 0.25 : 0.125; }

__device__ __forceinline__ double ref_of(const DomainConst& P, int k) {
  return k == 0 ? (double)P.rho_ref : (k == 4 ? (double)P.E_ref : 0.0);
}

template <typename S>
__global__ void k_pop_get(const DomainConst P, int parity, const S* __restrict__ pop,
                          const float* __restrict__ ghost, int k, int i, void* out, int dtype) {
  for (long long cell = blockIdx.x * (long long)blockDim.x + threadIdx.x; cell < P.ncell;
       cell += (long long)gridDim.x * blockDim.x) {
    int x, y, z;
    decompose(P, cell, x, y, z);
    const CellIndex c = make_index(P, x, y, z);
    if (dtype == 2) {  // native bits; the ghost value is encoded like a stored one
      S g = from_ghost(P, c, i) ? Codec<S>::enc(ghost_value(P, ghost, c, k, i), P.inv_scale[k])
                                : pop[read_pos(P, c, parity, k, i)];
      static_cast<S*>(out)[cell] = g;
      continue;
    }
    const double f = weight(i) * ref_of(P, k) + read_dev64(P, pop, ghost, c, parity, k, i);
    if (dtype == 1) static_cast<double*>(out)[cell] = f;
    else static_cast<float*>(out)[cell] = (float)f;
  }
}

template <typename S>
__global__ void k_pop_set(const DomainConst P, int parity, S* __restrict__ pop, int k, int i,
                          const void* in, int dtype) {
  for (long long cell = blockIdx.x * (long long)blockDim.x + threadIdx.x; cell < P.ncell;
       cell += (long long)gridDim.x * blockDim.x) {
    int x, y, z;
    decompose(P, cell, x, y, z);
    const CellIndex c = make_index(P, x, y, z);
    if (from_ghost(P, c, i)) continue;  // held ends keep the ghost inflow
    S g;
    if (dtype == 2) {
      g = static_cast<const S*>(in)[cell];
    } else {
      const double f = dtype == 1 ? static_cast<const double*>(in)[cell]
                                  : (double)static_cast<const float*>(in)[cell];
      g = Codec<S>::enc((float)(f - weight(i) * ref_of(P, k)), P.inv_scale[k]);
    }
    pop[read_pos(P, c, parity, k, i)] = g;
  }
}

// Raw stored values of storage slot `slot` of all fields on plane z, [k][y][x]; T is an
// unsigned integer of the element's size, so the bits move unchanged.
template <typename T>
__global__ void k_plane(const DomainConst P, T* __restrict__ pop, int z, int slot,
                        T* __restrict__ buf, int set) {
  const long long plane = (long long)P.nx * P.ny;
  for (long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x; r < plane * kF;
       r += (long long)gridDim.x * blockDim.x) {
    const int k = (int)(r / plane);
    const long long cell = r - k * plane + plane * z;
    if (!LBM_CHECK(P, cell >= 0 && cell < P.ncell)) continue;
    const long long at = pop_index(cell, k, slot);
    if (set) pop[at] = buf[r];
    else buf[r] = pop[at];
  }
}

int grid_for(long long n, int block) {
  long long g = (n + block - 1) / block;
  if (g > 152LL * 32) g = 152LL * 32;
  return (int)(g < 1 ? 1 : g);
}

}  // namespace


cudaError_t launch_moments(const DomainConst& P, int store, int parity, const void* pop,
                           const float* ghost, int which, void* out, int out_f64, long long c0,
                           long long cnt, cudaStream_t s) {
  const int block = 128, grid = grid_for(cnt, block);
  switch (store) {
    case 0: launch_moments_t(P, parity, (const float*)pop, ghost, which, out, out_f64, c0, cnt, grid, block, s); break;
    case 1: launch_moments_t(P, parity, (const __half*)pop, ghost, which, out, out_f64, c0, cnt, grid, block, s); break;
    default: launch_moments_t(P, parity, (const __nv_bfloat16*)pop, ghost, which, out, out_f64, c0, cnt, grid, block, s); break;
  }
  return cudaGetLastError();
}

cudaError_t launch_sensor(const DomainConst& P, int store, int parity, const void* pop,
                          const float* ghost, void* out, int out_f64, long long c0, long long cnt,
                          cudaStream_t s) {
  const int block = 128, grid = grid_for(cnt, block);
  switch (store) {
    case 0: k_sensor<float><<<grid, block, 0, s>>>(P, parity, (const float*)pop, ghost, out, out_f64, c0, cnt); break;
    case 1: k_sensor<__half><<<grid, block, 0, s>>>(P, parity, (const __half*)pop, ghost, out, out_f64, c0, cnt); break;
    default: k_sensor<__nv_bfloat16><<<grid, block, 0, s>>>(P, parity, (const __nv_bfloat16*)pop, ghost, out, out_f64, c0, cnt); break;
  }
  return cudaGetLastError();
}

cudaError_t launch_pop_get(const DomainConst& P, int store, int parity, const void* pop,
                           const float* ghost, int k, int i, void* out, int dtype, cudaStream_t s) {
  const int block = 256, grid = grid_for(P.ncell, block);
  switch (store) {
    case 0: k_pop_get<float><<<grid, block, 0, s>>>(P, parity, (const float*)pop, ghost, k, i, out, dtype); break;
    case 1: k_pop_get<__half><<<grid, block, 0, s>>>(P, parity, (const __half*)pop, ghost, k, i, out, dtype); break;
    default: k_pop_get<__nv_bfloat16><<<grid, block, 0, s>>>(P, parity, (const __nv_bfloat16*)pop, ghost, k, i, out, dtype); break;
  }
  return cudaGetLastError();
}

cudaError_t launch_pop_set(const DomainConst& P, int store, int parity, void* pop, int k, int i,
                           const void* in, int dtype, cudaStream_t s) {
  const int block = 256, grid = grid_for(P.ncell, block);
  switch (store) {
    case 0: k_pop_set<float><<<grid, block, 0, s>>>(P, parity, (float*)pop, k, i, in, dtype); break;
    case 1: k_pop_set<__half><<<grid, block, 0, s>>>(P, parity, (__half*)pop, k, i, in, dtype); break;
    default: k_pop_set<__nv_bfloat16><<<grid, block, 0, s>>>(P, parity, (__nv_bfloat16*)pop, k, i, in, dtype); break;
  }
  return cudaGetLastError();
}

cudaError_t launch_plane(const DomainConst& P, int store, void* pop, int z, int slot, void* buf,
                         int set, cudaStream_t s) {
  const int block = 256, grid = grid_for((long long)P.nx * P.ny * kF, block);
  if (store == 0)
    k_plane<unsigned><<<grid, block, 0, s>>>(P, (unsigned*)pop, z, slot, (unsigned*)buf, set);
  else
    k_plane<unsigned short><<<grid, block, 0, s>>>(P, (unsigned short*)pop, z, slot,
                                                   (unsigned short*)buf, set);
  return cudaGetLastError();
}

}  // namespace lbm
