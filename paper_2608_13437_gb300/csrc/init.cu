// Initial states (Sec. 3): TGV, Riemann problem, caller fields (rho, u, p) or caller
// zeroth moments (all 14 fields). Each cell gets the linear equilibrium of its state
// (tau = q = 0 unless given), stored as the deviation d_{k,i} = feq_{k,i} - w_i Q_ref,k
// in the storage type.
//
// All device arithmetic is FP32. The shifted storage only keeps its precision if the
// zeroth-moment deviations D_k = Q_k - Q_ref,k are formed without cancellation, so they
// are never taken as the difference of two rounded FP32 totals:
//   * TGV: D_rho = (p - p0)/T0 and D_E = (p - p0)/(gamma - 1) + rho|u|^2/2 straight from
//     the analytic pressure deviation rho0 U0^2/16 (cos 2x + cos 2y)(cos 2z + 2); the
//     trigonometric values of the node coordinates come from a per-axis table computed
//     on the host in FP64 and rounded once; the difference between the FP64 reference
//     (rho0, p0/(gamma-1)) and its FP32 copy enters as a host-computed constant.
//   * Riemann: two constant states, their deviations computed on the host in FP64.
//   * Caller fields: FP64 inputs are split into float-float pairs with integer
//     operations (no FP64 arithmetic), and rho - rho_ref and E - E_ref are float-float
//     differences rounded once.
// The fluxes of the equilibrium are not deviations; they are evaluated in FP32 from the
// cell's primitives. Populations are written with the step kernels' vector stores (one
// warp fills one 32-cell tile).
#include <cmath>
#include <cstring>

#include "diag_device.cuh"
#include "lbm_internal.h"

namespace lbm {

namespace {

// x = hi + lo with hi = x truncated to 24 significant bits and lo the remainder rounded
// to 24 bits, by integer and FP32 operations only (no FP64 arithmetic or conversion).
// Magnitudes outside the normal FP32 range become 0 or infinity; NaN stays NaN.
__device__ __forceinline__ FF split_f64(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const unsigned sign = (unsigned)(b >> 63) << 31;
  const int e = (int)((b >> 52) & 0x7FFu);
  const unsigned long long m = b & ((1ull << 52) - 1ull);
  FF r{0.0f, 0.0f};
  if (e == 0x7FF) {  // infinity or NaN
    r.hi = __int_as_float((int)(sign | 0x7F800000u | (m ? 0x400000u : 0u)));
    return r;
  }
  const int ef = e - 1023 + 127;  // biased FP32 exponent
  if (e == 0 || ef <= 0) {        // zero, or below the normal FP32 range
    r.hi = __int_as_float((int)sign);
    return r;
  }
  if (ef >= 255) {
    r.hi = __int_as_float((int)(sign | 0x7F800000u));
    return r;
  }
  r.hi = __int_as_float((int)(sign | ((unsigned)ef << 23) | (unsigned)(m >> 29)));
  // lo = (low 29 mantissa bits) * 2^(e - 1023 - 52)
  const unsigned low = (unsigned)(m & ((1ull << 29) - 1ull));
  const int s = e - 1075 + 127;  // biased FP32 exponent of 2^(e - 1075)
  if (low != 0 && s > 0) {
    const float mag = __fmul_rn(__uint2float_rn(low), __int_as_float(s << 23));
    r.lo = sign ? -mag : mag;
  }
  return r;
}

// Element idx of a caller array of FP32 or FP64 values as a float-float pair.
__device__ __forceinline__ FF load_ff(const InitSpec& sp, long long idx) {
  if (sp.fields_f64) return split_f64(static_cast<const double*>(sp.fields)[idx]);
  return FF{static_cast<const float*>(sp.fields)[idx], 0.0f};
}

__device__ __forceinline__ float ff_round(const FF& a) { return __fadd_rn(a.hi, a.lo); }

// (a.hi + a.lo) - r rounded once (a float-float difference).
__device__ __forceinline__ float ff_minus(FF a, float r) {
  ff_add(a, -r);
  return ff_round(a);
}

// (a.hi + a.lo) (g.hi + g.lo) as a float-float pair (about 44 significant bits).
__device__ __forceinline__ FF ff_mul(const FF& a, const FF& g) {
  const float p = __fmul_rn(a.hi, g.hi);
  const float e = __fmaf_rn(a.hi, g.hi, -p);  // exact error of the leading product
  const float t = __fmaf_rn(a.hi, g.lo, __fmaf_rn(a.lo, g.hi, e));
  FF r;
  r.hi = __fadd_rn(p, t);
  r.lo = __fsub_rn(t, __fsub_rn(r.hi, p));
  return r;
}

// E = p/(gamma - 1) + rho|u|^2/2 of caller fields as a float-float pair.
__device__ __forceinline__ FF total_energy(const InitSpec& sp, const FF& p, float ke) {
  FF E = ff_mul(p, FF{sp.inv_gm1_hi, sp.inv_gm1_lo});
  ff_add(E, ke);
  return E;
}

// Zeroth-moment deviations and primitives of the initial state of the cell.
struct InitCell {
  float D[kF];
  Prim<float> s;
};

__device__ void initial_cell(const DomainConst& P, const InitSpec& sp, int x, int y, int z,
                             long long cell, InitCell& c) {
  Prim<float>& s = c.s;
#pragma unroll
  for (int k = 0; k < kF; ++k) c.D[k] = 0.0f;
  if (sp.kind == 3) {  // all 14 zeroth moments given: the step's own FP32 closure
    const long long n = P.ncell;
    float Q[kF];
#pragma unroll
    for (int k = 0; k < kF; ++k) {
      const FF q = load_ff(sp, k * n + cell);
      Q[k] = ff_round(q);
      c.D[k] = k == 0 ? ff_minus(q, P.rho_ref) : (k == 4 ? ff_minus(q, P.E_ref) : Q[k]);
    }
    closure<float>(Q, P.gm1, P.mu, P.visc0, P.heat0, P.inv_T_ref, P.sutherland, s);
    return;
  }
#pragma unroll
  for (int j = 0; j < 6; ++j) s.tau[j] = 0.0f;
#pragma unroll
  for (int j = 0; j < 3; ++j) s.q[j] = 0.0f;
  float dp = 0.0f;
  FF p_ff{0.0f, 0.0f};
  if (sp.kind == 0) {  // supersonic TGV (Sec. 3.2), nodes at (x, y, z) dx
    const float* t = sp.trig;
    const float* ty = t + 3 * P.nx;
    const float* tz = ty + 3 * P.ny;
    const float sx = t[x], cx = t[P.nx + x], c2x = t[2 * P.nx + x];
    const float sy = ty[y], cy = ty[P.ny + y], c2y = ty[2 * P.ny + y];
    const float cz = tz[P.nz + z], c2z = tz[2 * P.nz + z];
    s.u[0] = mul(mul(mul(sp.U0, sx), cy), cz);
    s.u[1] = -mul(mul(mul(sp.U0, cx), sy), cz);
    s.u[2] = 0.0f;
    dp = mul(mul(sp.c_dp, add(c2x, c2y)), add(c2z, 2.0f));  // p - p0
    c.D[0] = fma_(dp, sp.inv_T0, sp.drho_ref);
    s.rho = add(P.rho_ref, c.D[0]);
    s.p = add(sp.p0, dp);
    s.T = sp.T0;  // uniform T0
  } else if (sp.kind == 1) {  // Riemann problem: one of two constant states
    const int idx = sp.axis == 0 ? x : (sp.axis == 1 ? y : z);
    const int side = idx < sp.split ? 0 : 1;
#pragma unroll
    for (int j = 0; j < 5; ++j) c.D[j] = sp.sD[side][j];
    s.rho = sp.sprim[side][0];
#pragma unroll
    for (int a = 0; a < 3; ++a) s.u[a] = sp.sprim[side][1 + a];
    s.p = sp.sprim[side][4];
    s.T = sp.sT[side];
  } else {  // caller fields rho, u_x, u_y, u_z, p
    const long long n = P.ncell;
    const FF rho = load_ff(sp, cell);
    c.D[0] = ff_minus(rho, P.rho_ref);
    s.rho = ff_round(rho);
#pragma unroll
    for (int a = 0; a < 3; ++a) s.u[a] = ff_round(load_ff(sp, (1 + a) * n + cell));
    p_ff = load_ff(sp, 4 * n + cell);
    s.p = ff_round(p_ff);
    s.T = __fdiv_rn(s.p, s.rho);
  }
  s.inv_rho = __frcp_rn(s.rho);
  if (sp.kind == 1) {
#pragma unroll
    for (int a = 0; a < 3; ++a) s.m[a] = c.D[1 + a];
  } else {
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      s.m[a] = mul(s.rho, s.u[a]);
      c.D[1 + a] = s.m[a];
    }
  }
  const float ke = mul(0.5f, fma_(s.m[2], s.u[2], fma_(s.m[1], s.u[1], mul(s.m[0], s.u[0]))));
  if (sp.kind == 0) c.D[4] = fma_(dp, sp.inv_gm1_hi, add(ke, sp.dE_ref));
  if (sp.kind == 2) c.D[4] = ff_minus(total_energy(sp, p_ff, ke), P.E_ref);
  s.E = add(P.E_ref, c.D[4]);
  const float r = P.sutherland ? sutherland_ratio<float>(s.T, P.inv_T_ref) : 1.0f;
  s.mu_T = mul(P.mu, r);
  s.visc = mul(P.visc0, r);
  s.heat = mul(P.heat0, r);
}

// Deviations of the linear equilibrium: d_0 = D/4, d_{+-a} = D/8 +- Phi_a / (2c).
__device__ __forceinline__ void equilibrium_dev(const DomainConst& P, const InitCell& c,
                                                float (&dev)[kF][kQ]) {
#pragma unroll
  for (int k = 0; k < kF; ++k) {
    float fx, fy, fz;
    field_flux<float>(k, c.s, fx, fy, fz);
    const float e0 = mul(0.25f, c.D[k]), e1 = mul(0.125f, c.D[k]);
    const float ax = mul(P.half_inv_c, fx), ay = mul(P.half_inv_c, fy), az = mul(P.half_inv_c, fz);
    dev[k][0] = e0;
    dev[k][1] = add(e1, ax);
    dev[k][2] = sub(e1, ax);
    dev[k][3] = add(e1, ay);
    dev[k][4] = sub(e1, ay);
    dev[k][5] = add(e1, az);
    dev[k][6] = sub(e1, az);
  }
}

// mode 0: per-field max |d| into maxbits (for the FP16 scales); mode 1: write the
// populations (canonical slots: slot i of a cell holds f_i, under the esoteric twist
// with slots 2, 4, 6 one cell further along +x, +y, +z) and the held-x ghosts, and
// set *bad (if given) when a cell's state is not finite. Blocks of whole warps, so a
// warp covers one 32-cell tile.
template <typename S>
__global__ void __launch_bounds__(128) k_init(const DomainConst P, const InitSpec sp, int mode,
                                              S* __restrict__ pop, float* __restrict__ ghost,
                                              unsigned* __restrict__ maxbits,
                                              unsigned* __restrict__ bad) {
  const long long n = P.ncell;
  const long long planes = (long long)P.ny * P.nz;
  const long long stride = (long long)gridDim.x * blockDim.x;
  // uniform trip count per warp, so the warp reduction of mode 0 sees full warps
  const long long n_pad = (n + 31) / 32 * 32;
  float mx[kF];
#pragma unroll
  for (int k = 0; k < kF; ++k) mx[k] = 0.0f;
  for (long long cell = blockIdx.x * (long long)blockDim.x + threadIdx.x; cell < n_pad;
       cell += stride) {
    if (cell >= n) continue;
    int x, y, z;
    cell_xyz(P, cell, x, y, z);
    InitCell c;
    initial_cell(P, sp, x, y, z, cell, c);
    float dev[kF][kQ];
    equilibrium_dev(P, c, dev);
    if (mode == 0) {
#pragma unroll
      for (int k = 0; k < kF; ++k)
#pragma unroll
        for (int i = 0; i < kQ; ++i) mx[k] = fmaxf(mx[k], fabsf(dev[k][i]));
      continue;
    }
    if (bad) {  // a non-finite input or state ends up in the moments or the fluxes
      float probe = 0.0f;
#pragma unroll
      for (int k = 0; k < kF; ++k) probe += dev[k][1] + dev[k][2];
      if (!isfinite(probe)) atomicOr(bad, 1u);
    }
    if (!LBM_CHECK(P, cell < P.ntile * kTile)) continue;
    if (P.eso) {  // esoteric twist: slots 2, 4, 6 live with the cell one step along +x, +y, +z
      const CellIndex ci = make_index(P, x, y, z);
#pragma unroll
      for (int i = 0; i < kQ; ++i) {
        const long long tc = eso_shifted(i) ? ci.nb[i - 1] : cell;
        if (!LBM_CHECK(P, tc >= 0 && tc < P.ntile * kTile)) continue;
        store_dir<S>(P, pop + tile_start(tc), i, (int)(tc & (kTile - 1)), dev, i, nullptr);
      }
    } else {
      S* base = pop + tile_start(cell);
      const int lane = (int)(cell & (kTile - 1));
#pragma unroll
      for (int i = 0; i < kQ; ++i) store_dir<S>(P, base, i, lane, dev, i, nullptr);
    }
    if (P.bc_x && ghost) {
      const long long plane = (long long)y + (long long)P.ny * z;
      if (x == 0)
        for (int k = 0; k < kF; ++k) ghost[(0 * kF + k) * planes + plane] = dev[k][1];
      if (x == P.nx - 1)
        for (int k = 0; k < kF; ++k) ghost[(1LL * kF + k) * planes + plane] = dev[k][2];
    }
  }
  if (mode == 0) {
#pragma unroll
    for (int k = 0; k < kF; ++k) {
      float m = mx[k];
      for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
      // order of non-negative floats = order of their bits
      if ((threadIdx.x & 31) == 0 && m > 0.0f) atomicMax(&maxbits[k], __float_as_uint(m));
    }
  }
}

constexpr int kMeanBlocks = (kFieldSumDoubles - 2) / 2, kMeanThreads = 256;

// Sums of rho and E of the caller's fields over the sample of field_sample(), in a
// fixed order: per thread as float-float pairs (E = p/(gamma - 1) + rho|u|^2/2 per cell
// in float-float), widened to FP64 once per thread, then a shared-memory tree per block
// and the blocks in order, so Q_ref is reproducible. Sampled runs are 32 consecutive
// cells (128-byte reads of each field).
__global__ void __launch_bounds__(kMeanThreads) k_field_sums(const DomainConst P, const InitSpec sp,
                                                             long long run_stride,
                                                             double* __restrict__ partials) {
  __shared__ double sh[2][kMeanThreads];
  FF s_rho{0.0f, 0.0f}, s_E{0.0f, 0.0f};
  const long long n = P.ncell;
  const long long runs = (n + kTile - 1) / kTile;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;; t += (long long)gridDim.x * blockDim.x) {
    const long long run = (t / kTile) * run_stride;
    if (run >= runs) break;
    const long long cell = run * kTile + (t % kTile);
    if (cell >= n) continue;
    const FF rho = load_ff(sp, cell);
    ff_merge(s_rho, rho);
    if (sp.kind == 3) {
      ff_merge(s_E, load_ff(sp, 4 * n + cell));
    } else {
      const float r = ff_round(rho);
      float u[3], m[3];
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        u[a] = ff_round(load_ff(sp, (1 + a) * n + cell));
        m[a] = mul(r, u[a]);
      }
      const float ke = mul(0.5f, fma_(m[2], u[2], fma_(m[1], u[1], mul(m[0], u[0]))));
      ff_merge(s_E, total_energy(sp, load_ff(sp, 4 * n + cell), ke));
    }
  }
  sh[0][threadIdx.x] = ff_value(s_rho);
  sh[1][threadIdx.x] = ff_value(s_E);
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

// 1/(gamma - 1) as a float-float pair.
void inv_gm1_pair(double gamma, InitSpec* sp) {
  const double g = 1.0 / (gamma - 1.0);
  sp->inv_gm1_hi = (float)g;
  sp->inv_gm1_lo = (float)(g - (double)sp->inv_gm1_hi);
}

}  // namespace

size_t tgv_table_floats(int nx, int ny, int nz) { return 3 * ((size_t)nx + ny + nz); }

void tgv_spec(const DomainConst& P, double gamma, double U0, double M0, double rho0, double dx,
              InitSpec* sp, std::vector<float>* table) {
  std::memset(sp, 0, sizeof(*sp));
  sp->kind = 0;
  const double p0 = rho0 * U0 * U0 / (gamma * M0 * M0);
  const double T0 = p0 / rho0;
  sp->U0 = (float)U0;
  sp->c_dp = (float)(rho0 * U0 * U0 / 16.0);
  sp->inv_T0 = (float)(1.0 / T0);
  sp->p0 = (float)p0;
  sp->T0 = (float)T0;
  inv_gm1_pair(gamma, sp);
  // the FP32 reference differs from (rho0, p0/(gamma-1)) by these amounts
  sp->drho_ref = (float)(rho0 - (double)P.rho_ref);
  sp->dE_ref = (float)(p0 / (gamma - 1.0) - (double)P.E_ref);
  const int n[3] = {P.nx, P.ny, P.nz};
  table->assign(tgv_table_floats(P.nx, P.ny, P.nz), 0.0f);
  size_t o = 0;
  for (int a = 0; a < 3; ++a) {
    for (int i = 0; i < n[a]; ++i) {
      const double X = i * dx;
      (*table)[o + i] = (float)std::sin(X);
      (*table)[o + n[a] + i] = (float)std::cos(X);
      (*table)[o + 2 * n[a] + i] = (float)std::cos(2.0 * X);
    }
    o += 3 * (size_t)n[a];
  }
}

void riemann_spec(const DomainConst& P, double gamma, int axis, int split, const double left[3],
                  const double right[3], InitSpec* sp) {
  std::memset(sp, 0, sizeof(*sp));
  sp->kind = 1;
  sp->axis = axis;
  sp->split = split;
  inv_gm1_pair(gamma, sp);
  const double* st[2] = {left, right};
  for (int s = 0; s < 2; ++s) {
    const double rho = st[s][0], u = st[s][1], p = st[s][2];
    const double E = p / (gamma - 1.0) + 0.5 * rho * u * u;
    sp->sD[s][0] = (float)(rho - (double)P.rho_ref);
    sp->sD[s][1 + axis] = (float)(rho * u);
    sp->sD[s][4] = (float)(E - (double)P.E_ref);
    sp->sprim[s][0] = (float)rho;
    sp->sprim[s][1 + axis] = (float)u;
    sp->sprim[s][4] = (float)p;
    sp->sT[s] = (float)(p / rho);
  }
}

void fields_spec(double gamma, int kind, const void* fields, int f64, InitSpec* sp) {
  std::memset(sp, 0, sizeof(*sp));
  sp->kind = kind;
  sp->fields = fields;
  sp->fields_f64 = f64;
  inv_gm1_pair(gamma, sp);
}

cudaError_t launch_init(const DomainConst& P, int store, const InitSpec& spec, int mode, void* pop,
                        float* ghost, unsigned* maxbits, unsigned* bad, cudaStream_t s) {
  const int block = 128;
  const int grid = grid_for(P.ncell, block);
  switch (store) {
    case 0: k_init<float><<<grid, block, 0, s>>>(P, spec, mode, static_cast<float*>(pop), ghost, maxbits, bad); break;
    case 1: k_init<__half><<<grid, block, 0, s>>>(P, spec, mode, static_cast<__half*>(pop), ghost, maxbits, bad); break;
    default: k_init<__nv_bfloat16><<<grid, block, 0, s>>>(P, spec, mode, static_cast<__nv_bfloat16*>(pop), ghost, maxbits, bad); break;
  }
  return cudaGetLastError();
}

FieldSample field_sample(long long ncell) {
  const long long runs = (ncell + kTile - 1) / kTile;
  FieldSample f;
  f.run_stride = runs > kSampleRuns ? runs / kSampleRuns : 1;
  f.cells = 0;
  for (long long r = 0; r < runs; r += f.run_stride)
    f.cells += (r + 1) * kTile <= ncell ? kTile : ncell - r * kTile;
  return f;
}

cudaError_t launch_field_means(const DomainConst& P, const InitSpec& spec, double* sums,
                               cudaStream_t s) {
  // sums holds 2 results followed by 2 * kMeanBlocks partials
  double* partials = sums + 2;
  k_field_sums<<<kMeanBlocks, kMeanThreads, 0, s>>>(P, spec, field_sample(P.ncell).run_stride,
                                                     partials);
  k_field_sums_final<<<1, 32, 0, s>>>(partials, kMeanBlocks, sums);
  return cudaGetLastError();
}

}  // namespace lbm
