// Device-side building blocks of the fused compressible-NSF D3Q7 step:
// domain constants, storage codecs, the AA-pattern index maps and the per-cell
// moments -> closure -> sensor -> collision arithmetic.
//
// Scheme (Bukreev, Kummerlaender, Krause): 14 fields Q = (rho, rho u, E, tau, q),
// one D3Q7 population set each (Eq. 2, Sec. 2.2); linear equilibrium
// feq_{k,i} = w_i (Q_k + c_i . Phi_k / c_s^2) with w_0 = 1/4, w_{+-a} = 1/8,
// c_s^2 = c^2/4; BGK collision with the source on the weights (Sec. 2.2); the
// cell-local sensor and blended rate of Sec. 2.3 (Eqs. 3-6).
//
// Populations are held as deviations d = f - w_i Q_ref,k from a reference state
// Q_ref = (rho_ref, 0, 0, 0, E_ref, 0...) (the reference-shifted form the paper
// runs in single precision), so every sum below works on small numbers.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace lbm {

constexpr int kF = 14;   // fields
constexpr int kQ = 7;    // D3Q7 directions: 0 rest, 1 +x, 2 -x, 3 +y, 4 -y, 5 +z, 6 -z
constexpr int kP = kF * kQ;
constexpr float kSutherlandT = 0.4042f;

__host__ __device__ constexpr int opp(int i) { return i == 0 ? 0 : ((i & 1) ? i + 1 : i - 1); }

// Constants of one domain, passed by value to every kernel.
struct DomainConst {
  int nx, ny, nz, bc_x;
  long long ncell;
  long long stride;   // elements between consecutive population arrays (>= ncell)
  float c, inv_c, half_inv_c, dt;
  float gm1;          // gamma - 1
  float gamma;
  float mu;           // reference viscosity
  float visc0;        // mu / tau_R
  float heat0;        // kappa / tau_q
  float inv_T_ref;
  float fmu_coef;     // 4 f_mu dt / dx^2 (Eq. 6)
  float C_sigma, J_min, omega_min;
  float src_R, src_q; // dS_k = src * Q_k for tau and q fields
  float rho_ref, E_ref;
  float scale[kF], inv_scale[kF];
  int sutherland, sensor_mode, collide, pad_;
  double dx64, dt64, mu64, inv_T_ref64, gm1_64;  // FP64 copies for the diagnostics
};

// ---------------------------------------------------------------- storage codecs
template <typename S>
struct Codec;

template <>
struct Codec<float> {
  static __device__ __forceinline__ float dec(float g, float) { return g; }
  static __device__ __forceinline__ float enc(float d, float) { return d; }
  static __device__ __forceinline__ double dec64(float g, double) { return (double)g; }
};

template <>
struct Codec<__half> {
  static __device__ __forceinline__ float dec(__half g, float s) { return __half2float(g) * s; }
  static __device__ __forceinline__ __half enc(float d, float inv_s) {
    return __float2half_rn(d * inv_s);
  }
  static __device__ __forceinline__ double dec64(__half g, double s) {
    return (double)__half2float(g) * s;
  }
};

template <>
struct Codec<__nv_bfloat16> {
  static __device__ __forceinline__ float dec(__nv_bfloat16 g, float s) {
    return __bfloat162float(g) * s;
  }
  static __device__ __forceinline__ __nv_bfloat16 enc(float d, float inv_s) {
    return __float2bfloat16_rn(d * inv_s);
  }
  static __device__ __forceinline__ double dec64(__nv_bfloat16 g, double s) {
    return (double)__bfloat162float(g) * s;
  }
};

// ---------------------------------------------------------------- AA index maps
// The state is one buffer pop[k][slot][cell]. After an even number of steps slot
// i of cell x holds f_i(x) (canonical). An even step reads its own slots and
// writes f*_i into slot opp(i) of the same cell; an odd step reads f_i(x) from
// slot opp(i) of cell x - e_i and writes f*_i into slot i of cell x + e_i. Every
// location is read and then written by the same thread, so the update is in place.
struct CellIndex {
  long long own;
  long long nb[kQ];  // nb[i] = cell x + e_i (periodic), nb[0] = own
  int x, plane;
};

__device__ __forceinline__ CellIndex make_index(const DomainConst& P, int x, int y, int z) {
  CellIndex c;
  const long long nx = P.nx, nxy = (long long)P.nx * P.ny;
  c.own = x + nx * ((long long)y + (long long)P.ny * z);
  c.x = x;
  c.plane = y + P.ny * z;
  c.nb[0] = c.own;
  c.nb[1] = c.own + (x + 1 < P.nx ? 1 : 1 - nx);
  c.nb[2] = c.own + (x > 0 ? -1 : nx - 1);
  c.nb[3] = c.own + (y + 1 < P.ny ? nx : nx - nxy);
  c.nb[4] = c.own + (y > 0 ? -nx : nxy - nx);
  c.nb[5] = c.own + (z + 1 < P.nz ? nxy : nxy - P.ncell);
  c.nb[6] = c.own + (z > 0 ? -nxy : P.ncell - nxy);
  return c;
}

// Cell and slot from which direction i of this cell is read at `parity`.
__device__ __forceinline__ long long read_pos(const DomainConst& P, const CellIndex& c, int parity,
                                              int k, int i) {
  const long long cell = parity ? c.nb[opp(i)] : c.own;
  const int slot = parity ? opp(i) : i;
  return (long long)(k * kQ + slot) * P.stride + cell;
}

// Cell and slot into which post-collision direction i of this cell is written.
__device__ __forceinline__ long long write_pos(const DomainConst& P, const CellIndex& c,
                                               int parity, int k, int i) {
  const long long cell = parity ? c.nb[i] : c.own;
  const int slot = parity ? i : opp(i);
  return (long long)(k * kQ + slot) * P.stride + cell;
}

// Held x ends: the inward population of a boundary cell comes from the ghost
// layer, ghost[side][k][plane] (deviation, unscaled).
__device__ __forceinline__ bool from_ghost(const DomainConst& P, const CellIndex& c, int i) {
  return P.bc_x && ((i == 1 && c.x == 0) || (i == 2 && c.x == P.nx - 1));
}

__device__ __forceinline__ float ghost_value(const DomainConst& P, const float* ghost,
                                             const CellIndex& c, int k, int i) {
  const long long planes = (long long)P.ny * P.nz;
  const int side = (i == 1) ? 0 : 1;
  return ghost[((long long)side * kF + k) * planes + c.plane];
}

template <int PARITY, bool HELD, typename S>
__device__ __forceinline__ void load_cell(const DomainConst& P, const S* __restrict__ pop,
                                          const float* __restrict__ ghost, const CellIndex& c,
                                          float (&d)[kF][kQ]) {
#pragma unroll
  for (int k = 0; k < kF; ++k) {
#pragma unroll
    for (int i = 0; i < kQ; ++i) {
      const S g = pop[read_pos(P, c, PARITY, k, i)];
      d[k][i] = Codec<S>::dec(g, P.scale[k]);
      if (HELD && (i == 1 || i == 2) && from_ghost(P, c, i)) d[k][i] = ghost_value(P, ghost, c, k, i);
    }
  }
}

template <int PARITY, typename S>
__device__ __forceinline__ void store_field(const DomainConst& P, S* __restrict__ pop,
                                            const CellIndex& c, int k, const float (&dk)[kQ]) {
#pragma unroll
  for (int i = 0; i < kQ; ++i) pop[write_pos(P, c, PARITY, k, i)] = Codec<S>::enc(dk[i], P.inv_scale[k]);
}

// ---------------------------------------------------------------- closure and flux
// Primitive state of one cell in precision R (float in the step, double in the
// initialisation and the moment outputs).
template <typename R>
struct Prim {
  R rho, inv_rho, m[3], u[3], E, p, T;
  R visc;     // mu_T / tau_R  (stress flux coefficient, Listing 1)
  R heat;     // kappa_T / tau_q (heat-flux flux coefficient, Listing 1)
  R mu_T;
  R tau[6];   // xx yy zz xy xz yz
  R q[3];
};

template <typename R>
__device__ __forceinline__ R sutherland_ratio(R T, R inv_T_ref) {
  const R t = T * inv_T_ref;
  return (R)(1.0 + 0.4042) * t * sqrt(t) / (t + (R)0.4042);
}

// Sec. 2.1: u = (rho u)/rho, p = (gamma-1)(E - rho|u|^2/2), T = p/rho; Sutherland.
template <typename R>
__device__ __forceinline__ void closure(const R Q[kF], R gm1, R mu, R visc0, R heat0,
                                        R inv_T_ref, int sutherland, Prim<R>& s) {
  s.rho = Q[0];
  s.inv_rho = (R)1 / s.rho;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    s.m[a] = Q[1 + a];
    s.u[a] = s.m[a] * s.inv_rho;
  }
  s.E = Q[4];
  const R ke = (R)0.5 * (s.m[0] * s.u[0] + s.m[1] * s.u[1] + s.m[2] * s.u[2]);
  s.p = gm1 * (s.E - ke);
  s.T = s.p * s.inv_rho;
  const R r = sutherland ? sutherland_ratio<R>(s.T, inv_T_ref) : (R)1;
  s.mu_T = mu * r;
  s.visc = visc0 * r;
  s.heat = heat0 * r;
#pragma unroll
  for (int j = 0; j < 6; ++j) s.tau[j] = Q[5 + j];
#pragma unroll
  for (int j = 0; j < 3; ++j) s.q[j] = Q[11 + j];
}

// Flux Phi_k (Eq. 2, Newtonian sign convention of tau) of field k, written out per
// component; Lambda_{bc,a} = delta_ab u_c + delta_ac u_b - 2/3 delta_bc u_a.
template <typename R>
__device__ __forceinline__ void field_flux(int k, const Prim<R>& s, R& fx, R& fy, R& fz) {
  const R ux = s.u[0], uy = s.u[1], uz = s.u[2];
  const R txx = s.tau[0], tyy = s.tau[1], tzz = s.tau[2];
  const R txy = s.tau[3], txz = s.tau[4], tyz = s.tau[5];
  const R v = s.visc, two3 = (R)(2.0 / 3.0), four3 = (R)(4.0 / 3.0);
  switch (k) {
    case 0: fx = s.m[0]; fy = s.m[1]; fz = s.m[2]; break;
    case 1: fx = s.m[0] * ux + s.p - txx; fy = s.m[0] * uy - txy; fz = s.m[0] * uz - txz; break;
    case 2: fx = s.m[1] * ux - txy; fy = s.m[1] * uy + s.p - tyy; fz = s.m[1] * uz - tyz; break;
    case 3: fx = s.m[2] * ux - txz; fy = s.m[2] * uy - tyz; fz = s.m[2] * uz + s.p - tzz; break;
    case 4: {
      const R h = s.E + s.p;
      fx = h * ux - (txx * ux + txy * uy + txz * uz) + s.q[0];
      fy = h * uy - (txy * ux + tyy * uy + tyz * uz) + s.q[1];
      fz = h * uz - (txz * ux + tyz * uy + tzz * uz) + s.q[2];
      break;
    }
    case 5: fx = txx * ux - v * four3 * ux; fy = txx * uy + v * two3 * uy; fz = txx * uz + v * two3 * uz; break;
    case 6: fx = tyy * ux + v * two3 * ux; fy = tyy * uy - v * four3 * uy; fz = tyy * uz + v * two3 * uz; break;
    case 7: fx = tzz * ux + v * two3 * ux; fy = tzz * uy + v * two3 * uy; fz = tzz * uz - v * four3 * uz; break;
    case 8: fx = txy * ux - v * uy; fy = txy * uy - v * ux; fz = txy * uz; break;
    case 9: fx = txz * ux - v * uz; fy = txz * uy; fz = txz * uz - v * ux; break;
    case 10: fx = tyz * ux; fy = tyz * uy - v * uz; fz = tyz * uz - v * uy; break;
    case 11: fx = s.q[0] * ux + s.heat * s.T; fy = s.q[0] * uy; fz = s.q[0] * uz; break;
    case 12: fx = s.q[1] * ux; fy = s.q[1] * uy + s.heat * s.T; fz = s.q[1] * uz; break;
    default: fx = s.q[2] * ux; fy = s.q[2] * uy; fz = s.q[2] * uz + s.heat * s.T; break;
  }
}

// ---------------------------------------------------------------- the cell update
struct SensorOut {
  float theta_dt;  // div u * dt (lattice units)
  float chi;
  float omega_h;
};

// Collides one cell in place on its decoded deviations d[k][i]. Returns the sum of
// the zeroth-moment deviations (a finiteness probe). With kSensor the sensor
// values are reported and the populations are left unchanged.
template <bool kSensor>
__device__ __forceinline__ float collide_cell(const DomainConst& P, float (&d)[kF][kQ],
                                              SensorOut* so) {
  // Zeroth moments (Sec. 2.2: Q from the zeroth moment alone), i ascending.
  float D[kF];
#pragma unroll
  for (int k = 0; k < kF; ++k) {
    float s = d[k][0];
#pragma unroll
    for (int i = 1; i < kQ; ++i) s += d[k][i];
    D[k] = s;
  }
  float Q[kF];
#pragma unroll
  for (int k = 0; k < kF; ++k) Q[k] = D[k];
  Q[0] += P.rho_ref;
  Q[4] += P.E_ref;
  Prim<float> s;
  closure<float>(Q, P.gm1, P.mu, P.visc0, P.heat0, P.inv_T_ref, P.sutherland, s);

  // Eq. 6: tau_base = 1/2 + 4 f_mu (mu_T/rho) dt/dx^2, omega = 1/tau_base.
  const float tau_b = 0.5f + P.fmu_coef * s.mu_T * s.inv_rho;
  const float omega = 1.0f / tau_b;

  // Local dilatation from the cell's own non-equilibrium moments (pre-collision):
  //   fneq_{k,0} = d_{k,0} - D_k/4 = tau dt div(Phi_k)/4,
  //   m1_{rho,a} = c (d_{rho,+a} - d_{rho,-a}) - (rho u)_a
  //             = -tau dt (d_t (rho u)_a + (c^2/4) d_a rho),
  // so, in lattice units (theta dt) with tau = tau_base:
  //   theta dt = 4 omega / rho [fneq_{rho,0} - sum_a (u_a/c)(4 fneq_{rho u_a,0}/c
  //                                                   - (d_{rho,+a} - d_{rho,-a}) + m_a/c)].
  float acc = d[0][0] - 0.25f * D[0];
  if (P.sensor_mode == 0) {
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const float fneq_m0 = d[1 + a][0] - 0.25f * D[1 + a];
      const float g = 4.0f * fneq_m0 * P.inv_c - (d[0][2 * a + 1] - d[0][2 * a + 2]) + s.m[a] * P.inv_c;
      acc -= s.u[a] * P.inv_c * g;
    }
  }
  const float theta_dt = 4.0f * omega * s.inv_rho * acc;
  // Eq. 3: s = max(0, -div u)/c_s with c_s = 1/2 in lattice units.
  const float smach = 2.0f * fmaxf(0.0f, -theta_dt);
  // Eq. 4 and Eq. 5.
  const float chi = (smach > P.J_min) ? fminf(P.C_sigma * smach, 1.0f) : 0.0f;
  const float om = omega - chi * (omega - P.omega_min);
  if constexpr (kSensor) {
    so->theta_dt = theta_dt;
    so->chi = chi;
    so->omega_h = om;
    return D[0];
  } else {

  // Collision, field by field: d* = d + omega_h (deq - d) + w_i dS_k with
  // deq_0 = D/4, deq_{+-a} = D/8 +- Phi_a / (2c).
#pragma unroll
  for (int k = 0; k < kF; ++k) {
    float fx, fy, fz;
    field_flux<float>(k, s, fx, fy, fz);
    const float e0 = 0.25f * D[k], e1 = 0.125f * D[k];
    const float ax = P.half_inv_c * fx, ay = P.half_inv_c * fy, az = P.half_inv_c * fz;
    float dS = 0.0f;
    if (k >= 5) dS = (k < 11 ? P.src_R : P.src_q) * D[k];
    const float s0 = 0.25f * dS, s1 = 0.125f * dS;
    d[k][0] = fmaf(om, e0 - d[k][0], d[k][0]) + s0;
    d[k][1] = fmaf(om, (e1 + ax) - d[k][1], d[k][1]) + s1;
    d[k][2] = fmaf(om, (e1 - ax) - d[k][2], d[k][2]) + s1;
    d[k][3] = fmaf(om, (e1 + ay) - d[k][3], d[k][3]) + s1;
    d[k][4] = fmaf(om, (e1 - ay) - d[k][4], d[k][4]) + s1;
    d[k][5] = fmaf(om, (e1 + az) - d[k][5], d[k][5]) + s1;
    d[k][6] = fmaf(om, (e1 - az) - d[k][6], d[k][6]) + s1;
  }
  float probe = 0.0f;
#pragma unroll
  for (int k = 0; k < kF; ++k) probe += D[k];
  return probe;
  }
}

}  // namespace lbm
