// FP64 CPU oracle of the compressible Navier-Stokes-Fourier lattice Boltzmann
// scheme of Bukreev, Kummerlaender and Krause, "Lattice Boltzmann Method for
// Compressible Navier-Stokes-Fourier Equations".
//
// TEST INFRASTRUCTURE. Only the test suite, the smoke check and the benchmark's
// CPU-baseline leg load this library. It shares no code, header or constant with
// the CUDA library; the two agree only because both follow the paper.
//
// The scheme, step by step, for every cell of a periodic 3-D grid:
//   1. zeroth moments       Q_k = sum_i f_{k,i}                          (Sec. 2.2)
//   2. closure              u, p, T, Sutherland mu_T, kappa_T            (Sec. 2.1, Listing 1)
//   3. flux                 Phi_k(Q), 14 x 3                             (Eq. 2)
//   4. sensor               theta = div u from the cell's own moments,
//                           s, chi, omega_h                              (Sec. 2.3, Eqs. 3-6)
//   5. collision            f* = f - omega_h (f - feq) + w_i dS_k        (Sec. 2.2)
//   6. streaming            f_{k,i}(x) <- f*_{k,i}(x - e_i)              (Sec. 1, Sec. 2.2)
// The state kept between steps is the pre-collision (post-streaming) population
// set, in the layout f[k][i][z][y][x]. Two buffers are used: collide every cell
// into `post`, then pull-stream `post` into `f`. Nothing is fused or reordered.
//
// Points the paper leaves open are marked READING; each names the choice made.
//
// Fields k (Eq. 2): 0 rho, 1-3 rho u, 4 E, 5-10 tau (xx yy zz xy xz yz), 11-13 q.
// Directions i (D3Q7): 0 rest, 1 +x, 2 -x, 3 +y, 4 -y, 5 +z, 6 -z.

#include <cmath>
#include <cstdint>
#include <cstdlib>
#include <cstring>
#include <new>
#include <vector>
#ifdef _OPENMP
#include <omp.h>
#endif

namespace {

constexpr int NF = 14;
constexpr int NQ = 7;
constexpr int NP = NF * NQ;

enum { RHO = 0, MX = 1, EN = 4, TAU0 = 5, QX = 11 };

// Unit lattice vectors e_i; the lattice velocity is c_i = c e_i with c = dx/dt.
const int E[NQ][3] = {{0, 0, 0}, {1, 0, 0}, {-1, 0, 0}, {0, 1, 0},
                      {0, -1, 0}, {0, 0, 1}, {0, 0, -1}};

// READING (weights). Sec. 2.2 states only c_s^2 = 1/4 (lattice units) for D3Q7.
// sum_i w_i = 1, sum_i w_i e_ia e_ib = c_s^2 delta_ab and six equivalent moving
// directions give w_moving = c_s^2 / 2 = 1/8 and w_rest = 1 - 6/8 = 1/4.
const double W[NQ] = {0.25, 0.125, 0.125, 0.125, 0.125, 0.125, 0.125};
const double CS2_LATTICE = 0.25;

// Symmetric stress components carried as fields 5..10: (b, c) pairs.
const int TAU_BC[6][2] = {{0, 0}, {1, 1}, {2, 2}, {0, 1}, {0, 2}, {1, 2}};

// Sutherland temperature in units of T_ref (Listing 1; Sec. 3.2 prints the same
// law as 1.4042 (T/T0)^{3/2} / (T/T0 + 0.4042) mu).
const double T_SUTHERLAND = 0.4042;

}  // namespace

extern "C" {

// Parameters; the ctypes structure in oracle.py mirrors this layout.
struct orc_params {
  int nx, ny, nz;
  int bc_x;          // 0: periodic in x; 1: x ends held at the initial state
  double dx;         // lattice spacing
  double dt;         // > 0: time step as given; <= 0: cfl * dx / (2 lambda_ref)
  double cfl;        // acoustic Courant number (Table 1)
  double lambda_ref; // largest signal speed |u| + a of the problem
  double gamma, mu, kappa, tau_R, tau_q, T_ref;
  int relax_in_dt;   // 1: tau_R and tau_q are given in units of dt (Sec. 3.1)
  int sutherland;    // 1: mu, kappa follow Sutherland's law; 0: constant
  int source_mode;   // 0: explicit w_i dt S_k; 1: exact integration of the relaxation
  double f_mu, C_sigma, J_min, omega_min;  // Table 1, Sec. 2.3
  int sensor_mode;   // 0: full dilatation; 1: div(rho u) / rho only
  int collide;       // 1: collide and stream; 0: stream only
};

// Diagnostics of one state; the ctypes structure in oracle.py mirrors this.
struct orc_diag {
  double step, time;
  double sum_rho, sum_mx, sum_my, sum_mz, sum_E;
  double ek_mean;        // <1/2 rho |u|^2>
  double eps_s_raw;      // <mu_local |curl u|^2>           (Eq. 7 without 1/rho_ref)
  double eps_d_raw;      // 4/3 <mu_local (div u)^2>        (Eq. 7 without 1/rho_ref)
  double max_mach, max_cfl, min_rho, min_T;
  double nonfinite;      // cells with a non-finite zeroth moment
};

}  // extern "C"

namespace {

struct Domain {
  orc_params p;
  double dt = 0, c = 0;  // time step and lattice speed dx/dt
  int64_t ncell = 0;
  int64_t step = 0;
  std::vector<double> f;     // pre-collision state [k][i][cell]
  std::vector<double> post;  // post-collision populations [k][i][cell]
  // Held x ends: populations of the ghost layers at x = -1 and x = nx, kept at the
  // initial populations of the adjacent boundary cells, [k][i][y][z-plane].
  std::vector<double> ghost_lo, ghost_hi;

  int64_t cell(int x, int y, int z) const {
    return (int64_t)x + (int64_t)p.nx * ((int64_t)y + (int64_t)p.ny * z);
  }
  double& at(std::vector<double>& a, int k, int i, int64_t c) {
    return a[((int64_t)k * NQ + i) * ncell + c];
  }
  double at(const std::vector<double>& a, int k, int i, int64_t c) const {
    return a[((int64_t)k * NQ + i) * ncell + c];
  }
};

// ---------------------------------------------------------------------------
// Closure: Sec. 2.1 (ideal gas, T = p / rho) and Listing 1 (Sutherland law).
// ---------------------------------------------------------------------------
struct Closure {
  double rho, u[3], E, p, T, mu_T, kappa_T;
};

double sutherland_ratio(const orc_params& p, double T) {
  if (!p.sutherland) return 1.0;
  const double t = T / p.T_ref;
  return (1.0 + T_SUTHERLAND) * std::pow(t, 1.5) / (t + T_SUTHERLAND);
}

Closure closure(const orc_params& p, const double Q[NF]) {
  Closure c;
  c.rho = Q[RHO];
  for (int a = 0; a < 3; ++a) c.u[a] = Q[MX + a] / c.rho;
  c.E = Q[EN];
  double u2 = 0;
  for (int a = 0; a < 3; ++a) u2 += c.u[a] * c.u[a];
  c.p = (p.gamma - 1.0) * (c.E - 0.5 * c.rho * u2);
  c.T = c.p / c.rho;
  const double r = sutherland_ratio(p, c.T);
  c.mu_T = p.mu * r;
  c.kappa_T = p.kappa * r;  // Listing 1: heat = kappa (mu_T / mu) / tau_q
  return c;
}

// Stress tensor entry tau_ab read from the state.
double tau_of(const double Q[NF], int a, int b) {
  for (int s = 0; s < 6; ++s)
    if ((TAU_BC[s][0] == a && TAU_BC[s][1] == b) || (TAU_BC[s][0] == b && TAU_BC[s][1] == a))
      return Q[TAU0 + s];
  return 0.0;
}

inline double delta(int a, int b) { return a == b ? 1.0 : 0.0; }

// READING (Lambda, Sec. 2.1): the rank-3 velocity flux whose divergence is the
// deviatoric strain rate, d_a Lambda_{bc,a} = d_b u_c + d_c u_b - 2/3 delta_bc div u.
// Taken linear in u: Lambda_{bc,a} = delta_ab u_c + delta_ac u_b - 2/3 delta_bc u_a.
double lambda_dev(int b, int c, int a, const double u[3]) {
  return delta(a, b) * u[c] + delta(a, c) * u[b] - (2.0 / 3.0) * delta(b, c) * u[a];
}

// Physical flux Phi_{k,a}, Eq. 2.
// READING (sign of the stress): Eq. 2 carries the Newtonian stress tau (momentum
// flux -tau, stress flux -(mu/tau_R) Lambda). Listing 1 declares the opposite sign
// of tau; the two systems map onto each other by tau -> -tau. Eq. 2 is used.
void flux(const orc_params& p, const double Q[NF], const Closure& c, double Phi[NF][3]) {
  const double visc = c.mu_T / p.tau_R;     // Listing 1: visc = mu_T / tau_R
  const double heat = c.kappa_T / p.tau_q;  // Listing 1: heat = kappa mu_T / mu / tau_q
  for (int a = 0; a < 3; ++a) {
    Phi[RHO][a] = Q[MX + a];
    for (int b = 0; b < 3; ++b)
      Phi[MX + b][a] = Q[MX + b] * c.u[a] + c.p * delta(a, b) - tau_of(Q, b, a);
    double tau_u = 0;
    for (int b = 0; b < 3; ++b) tau_u += tau_of(Q, a, b) * c.u[b];
    Phi[EN][a] = (c.E + c.p) * c.u[a] - tau_u + Q[QX + a];
    for (int s = 0; s < 6; ++s) {
      const int b = TAU_BC[s][0], cc = TAU_BC[s][1];
      Phi[TAU0 + s][a] = Q[TAU0 + s] * c.u[a] - visc * lambda_dev(b, cc, a, c.u);
    }
    for (int b = 0; b < 3; ++b)
      Phi[QX + b][a] = Q[QX + b] * c.u[a] + heat * c.T * delta(a, b);
  }
}

// Source S_k of Eq. 2: zero for the conserved fields, -tau/tau_R, -q/tau_q.
// READING (time integration of the source, Sec. 2.2 "projected onto the lattice
// weights"): mode 0 (default) adds w_i dt S_k, the literal explicit form, stable
// for dt/tau < 2; mode 1 adds w_i dS_k with dS_k = (exp(-dt/tau) - 1) Q_k, the
// exact solution of the linear relaxation over one step, stable for any dt/tau.
double source_increment(const orc_params& p, double dt, int k, double Qk) {
  if (k < TAU0) return 0.0;
  const double trelax = (k < QX) ? p.tau_R : p.tau_q;
  if (p.source_mode == 1) return std::expm1(-dt / trelax) * Qk;
  return -dt * Qk / trelax;
}

// Linear equilibrium with the flux exactly in the first moment (Sec. 2.2):
// feq_{k,i} = w_i (Q_k + c_i . Phi_k / c_s^2), c_i = c e_i, c_s^2 = c^2 / 4.
void equilibrium(double c, const double Q[NF], const double Phi[NF][3], double feq[NF][NQ]) {
  const double cs2 = CS2_LATTICE * c * c;
  for (int k = 0; k < NF; ++k)
    for (int i = 0; i < NQ; ++i) {
      double cphi = 0;
      for (int a = 0; a < 3; ++a) cphi += c * E[i][a] * Phi[k][a];
      feq[k][i] = W[i] * (Q[k] + cphi / cs2);
    }
}

// Baseline relaxation time, Eq. 6: tau_base = 1/2 + 4 f_mu (mu/rho) dt/dx^2.
// READING: mu is the local molecular viscosity mu_T of the cell.
double tau_base(const Domain& d, const Closure& c) {
  return 0.5 + 4.0 * d.p.f_mu * (c.mu_T / c.rho) * d.dt / (d.p.dx * d.p.dx);
}

// READING (local dilatation, Sec. 2.3 gives no formula). First-order
// Chapman-Enskog of this scheme gives, for the pre-collision non-equilibrium
// fneq = f - feq(Q) of a field with zero source:
//   rest population:  fneq_0 = w_0 tau dt div Phi
//   first moment:     sum_i c_i fneq_i = -tau dt (d_t Phi + c_s^2 grad Q)
// So div(rho u) = fneq_{rho,0} / (w_0 tau dt); d_t(rho u_a) = -div Phi_{rho u_a}
// = -fneq_{rho u_a,0} / (w_0 tau dt); and
//   grad_a rho = (fneq_{rho u_a,0} / w_0 - m1_{rho,a}) / (tau dt c_s^2),
// with m1_{rho,a} = sum_i c_ia f_{rho,i} - rho u_a. Then
//   theta = div u = (div(rho u) - u . grad rho) / rho.
// tau is the cell's baseline tau_base (the blended rate depends on theta).
double dilatation(const Domain& d, const double f[NF][NQ], const double Q[NF],
                  const Closure& c, double tau) {
  const double tdt = tau * d.dt;
  const double cs2 = CS2_LATTICE * d.c * d.c;
  const double fneq_rho0 = f[RHO][0] - W[0] * Q[RHO];
  const double div_m = fneq_rho0 / (W[0] * tdt);
  if (d.p.sensor_mode == 1) return div_m / c.rho;
  double u_grad_rho = 0;
  for (int a = 0; a < 3; ++a) {
    double first = 0;
    for (int i = 0; i < NQ; ++i) first += d.c * E[i][a] * f[RHO][i];
    const double m1 = first - Q[MX + a];
    const double fneq_m0 = f[MX + a][0] - W[0] * Q[MX + a];
    const double grad_rho = (fneq_m0 / W[0] - m1) / (tdt * cs2);
    u_grad_rho += c.u[a] * grad_rho;
  }
  return (div_m - u_grad_rho) / c.rho;
}

// Eq. 3 (compression Mach number, lattice units) and Eq. 4 (sensor).
// theta in lattice units is theta * dt; the lattice sound speed is sqrt(1/4).
double compression_mach(const Domain& d, double theta) {
  const double theta_lat = theta * d.dt;
  return std::fmax(0.0, -theta_lat) / std::sqrt(CS2_LATTICE);
}

double sensor_chi(const orc_params& p, double s) {
  if (!(s > p.J_min)) return 0.0;
  return std::fmin(std::fmax(p.C_sigma * s, 0.0), 1.0);
}

struct CellOut {
  double theta, chi, omega_h;
};

// One cell: moments, closure, flux, sensor, collision (steps 1-5 above).
CellOut collide_cell(const Domain& d, const double f[NF][NQ], double fout[NF][NQ]) {
  double Q[NF];
  for (int k = 0; k < NF; ++k) {
    double s = 0;
    for (int i = 0; i < NQ; ++i) s += f[k][i];
    Q[k] = s;  // Sec. 2.2: Q_k from the zeroth moment alone
  }
  const Closure c = closure(d.p, Q);
  double Phi[NF][3];
  flux(d.p, Q, c, Phi);
  double feq[NF][NQ];
  equilibrium(d.c, Q, Phi, feq);

  const double tb = tau_base(d, c);
  const double omega = 1.0 / tb;
  CellOut out;
  out.theta = dilatation(d, f, Q, c, tb);
  out.chi = sensor_chi(d.p, compression_mach(d, out.theta));
  out.omega_h = omega - out.chi * (omega - d.p.omega_min);  // Eq. 5

  for (int k = 0; k < NF; ++k) {
    const double dS = source_increment(d.p, d.dt, k, Q[k]);
    for (int i = 0; i < NQ; ++i) {
      if (d.p.collide)
        fout[k][i] = f[k][i] - out.omega_h * (f[k][i] - feq[k][i]) + W[i] * dS;
      else
        fout[k][i] = f[k][i];
    }
  }
  return out;
}

void gather(const Domain& d, const std::vector<double>& a, int64_t cell, double f[NF][NQ]) {
  for (int k = 0; k < NF; ++k)
    for (int i = 0; i < NQ; ++i) f[k][i] = d.at(a, k, i, cell);
}

// Held x ends: the inward-moving population of a boundary cell always comes from
// the ghost layer (whose populations stay at the initial ones of that cell).
void apply_held_inflow(Domain& d) {
  if (d.p.bc_x != 1) return;
  const int nx = d.p.nx;
  for (int z = 0; z < d.p.nz; ++z)
    for (int y = 0; y < d.p.ny; ++y) {
      const int64_t plane = (int64_t)y + (int64_t)d.p.ny * z;
      const int64_t nplane = (int64_t)d.p.ny * d.p.nz;
      for (int k = 0; k < NF; ++k) {
        d.at(d.f, k, 1, d.cell(0, y, z)) = d.ghost_lo[((int64_t)k * NQ + 1) * nplane + plane];
        d.at(d.f, k, 2, d.cell(nx - 1, y, z)) =
            d.ghost_hi[((int64_t)k * NQ + 2) * nplane + plane];
      }
    }
}

void record_ghosts(Domain& d) {
  if (d.p.bc_x != 1) return;
  const int64_t nplane = (int64_t)d.p.ny * d.p.nz;
  d.ghost_lo.assign((size_t)NP * nplane, 0.0);
  d.ghost_hi.assign((size_t)NP * nplane, 0.0);
  for (int z = 0; z < d.p.nz; ++z)
    for (int y = 0; y < d.p.ny; ++y) {
      const int64_t plane = (int64_t)y + (int64_t)d.p.ny * z;
      for (int k = 0; k < NF; ++k)
        for (int i = 0; i < NQ; ++i) {
          d.ghost_lo[((int64_t)k * NQ + i) * nplane + plane] = d.at(d.f, k, i, d.cell(0, y, z));
          d.ghost_hi[((int64_t)k * NQ + i) * nplane + plane] =
              d.at(d.f, k, i, d.cell(d.p.nx - 1, y, z));
        }
    }
}

void step_once(Domain& d) {
  const int nx = d.p.nx, ny = d.p.ny, nz = d.p.nz;
  // Collide every cell.
#pragma omp parallel for schedule(static)
  for (int z = 0; z < nz; ++z)
    for (int y = 0; y < ny; ++y)
      for (int x = 0; x < nx; ++x) {
        const int64_t cl = d.cell(x, y, z);
        double f[NF][NQ], fo[NF][NQ];
        gather(d, d.f, cl, f);
        collide_cell(d, f, fo);
        for (int k = 0; k < NF; ++k)
          for (int i = 0; i < NQ; ++i) d.at(d.post, k, i, cl) = fo[k][i];
      }
  // Stream: f_{k,i}(x) = post_{k,i}(x - e_i), periodic wrap.
#pragma omp parallel for schedule(static)
  for (int z = 0; z < nz; ++z)
    for (int y = 0; y < ny; ++y)
      for (int x = 0; x < nx; ++x) {
        const int64_t cl = d.cell(x, y, z);
        for (int i = 0; i < NQ; ++i) {
          const int xs = ((x - E[i][0]) % nx + nx) % nx;
          const int ys = ((y - E[i][1]) % ny + ny) % ny;
          const int zs = ((z - E[i][2]) % nz + nz) % nz;
          const int64_t src = d.cell(xs, ys, zs);
          for (int k = 0; k < NF; ++k) d.at(d.f, k, i, cl) = d.at(d.post, k, i, src);
        }
      }
  apply_held_inflow(d);  // replaces the wrapped x inflow at held ends
  d.step += 1;
}

// Equilibrium populations of a macroscopic state with tau = q = 0 (READING:
// "all state fields' populations at equilibrium" with zero stress and heat flux).
void set_equilibrium_cell(Domain& d, int64_t cl, double rho, const double u[3], double p) {
  double Q[NF] = {0};
  Q[RHO] = rho;
  double u2 = 0;
  for (int a = 0; a < 3; ++a) {
    Q[MX + a] = rho * u[a];
    u2 += u[a] * u[a];
  }
  Q[EN] = p / (d.p.gamma - 1.0) + 0.5 * rho * u2;
  const Closure c = closure(d.p, Q);
  double Phi[NF][3], feq[NF][NQ];
  flux(d.p, Q, c, Phi);
  equilibrium(d.c, Q, Phi, feq);
  for (int k = 0; k < NF; ++k)
    for (int i = 0; i < NQ; ++i) d.at(d.f, k, i, cl) = feq[k][i];
}

void finish_init(Domain& d) {
  d.step = 0;
  record_ghosts(d);
}

void macroscopic(const Domain& d, int64_t cl, double Q[NF]) {
  for (int k = 0; k < NF; ++k) {
    double s = 0;
    for (int i = 0; i < NQ; ++i) s += d.at(d.f, k, i, cl);
    Q[k] = s;
  }
}

}  // namespace

extern "C" {

void* orc_create(const orc_params* prm) {
  if (!prm || prm->nx < 1 || prm->ny < 1 || prm->nz < 1 || !(prm->dx > 0)) return nullptr;
  Domain* d = new (std::nothrow) Domain();
  if (!d) return nullptr;
  d->p = *prm;
  // READING (Table 1: the acoustic Courant number fixes dt at a given dx). The
  // Courant number is taken against the lattice sound speed c_s = c/2:
  // CFL = lambda_ref / c_s, so dt = CFL (1/2) dx / lambda_ref, with lambda_ref the
  // largest |u| + a of the problem. A given dt > 0 overrides.
  d->dt = prm->dt > 0 ? prm->dt : prm->cfl * std::sqrt(CS2_LATTICE) * prm->dx / prm->lambda_ref;
  if (!(d->dt > 0) || !std::isfinite(d->dt)) {
    delete d;
    return nullptr;
  }
  if (prm->relax_in_dt) {  // Sec. 3.1: tau_R = tau_q = (given multiple) * dt
    d->p.tau_R = prm->tau_R * d->dt;
    d->p.tau_q = prm->tau_q * d->dt;
  }
  d->c = prm->dx / d->dt;
  d->ncell = (int64_t)prm->nx * prm->ny * prm->nz;
  try {
    d->f.assign((size_t)NP * d->ncell, 0.0);
    d->post.assign((size_t)NP * d->ncell, 0.0);
  } catch (...) {
    delete d;
    return nullptr;
  }
  return d;
}

void orc_destroy(void* h) { delete static_cast<Domain*>(h); }

double orc_dt(void* h) { return static_cast<Domain*>(h)->dt; }
long long orc_step_count(void* h) { return static_cast<Domain*>(h)->step; }

void orc_set_threads(int n) {
#ifdef _OPENMP
  if (n > 0) omp_set_num_threads(n);
#else
  (void)n;
#endif
}

int orc_get_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

// Supersonic Taylor-Green vortex (Sec. 3.2): u = U0 sin x cos y cos z,
// v = -U0 cos x sin y cos z, w = 0, p = p0 + rho0 U0^2/16 (cos 2x + cos 2y)(cos 2z + 2),
// uniform T0 = p0 / rho0 with p0 = rho0 U0^2 / (gamma M0^2), rho = p / T0.
// Cell (i, j, l) sits at the global node ((gx0+i) mod gn, ...) * dx, so a window of
// a larger periodic box can be initialised.
int orc_init_tgv(void* h, double U0, double M0, double rho0, int gn, int gx0, int gy0, int gz0) {
  Domain& d = *static_cast<Domain*>(h);
  if (gn <= 0) gn = d.p.nx;
  const double p0 = rho0 * U0 * U0 / (d.p.gamma * M0 * M0);
  const double T0 = p0 / rho0;
#pragma omp parallel for schedule(static)
  for (int z = 0; z < d.p.nz; ++z)
    for (int y = 0; y < d.p.ny; ++y)
      for (int x = 0; x < d.p.nx; ++x) {
        const double X = (double)(((gx0 + x) % gn + gn) % gn) * d.p.dx;
        const double Y = (double)(((gy0 + y) % gn + gn) % gn) * d.p.dx;
        const double Z = (double)(((gz0 + z) % gn + gn) % gn) * d.p.dx;
        const double u[3] = {U0 * std::sin(X) * std::cos(Y) * std::cos(Z),
                             -U0 * std::cos(X) * std::sin(Y) * std::cos(Z), 0.0};
        const double p = p0 + rho0 * U0 * U0 / 16.0 * (std::cos(2 * X) + std::cos(2 * Y)) *
                                  (std::cos(2 * Z) + 2.0);
        set_equilibrium_cell(d, d.cell(x, y, z), p / T0, u, p);
      }
  finish_init(d);
  return 0;
}

// Riemann problem along `axis`: cells with index < i_split take the left state
// (rho, u_axis, p), the others the right state.
int orc_init_riemann(void* h, int axis, int i_split, const double* L, const double* R) {
  Domain& d = *static_cast<Domain*>(h);
  if (axis < 0 || axis > 2) return 1;
#pragma omp parallel for schedule(static)
  for (int z = 0; z < d.p.nz; ++z)
    for (int y = 0; y < d.p.ny; ++y)
      for (int x = 0; x < d.p.nx; ++x) {
        const int idx = axis == 0 ? x : (axis == 1 ? y : z);
        const double* s = idx < i_split ? L : R;
        double u[3] = {0, 0, 0};
        u[axis] = s[1];
        set_equilibrium_cell(d, d.cell(x, y, z), s[0], u, s[2]);
      }
  finish_init(d);
  return 0;
}

// Equilibrium initialisation from given fields rho, u_x, u_y, u_z, p (each [cell]).
int orc_init_fields(void* h, const double* rho, const double* ux, const double* uy,
                    const double* uz, const double* p) {
  Domain& d = *static_cast<Domain*>(h);
#pragma omp parallel for schedule(static)
  for (int64_t cl = 0; cl < d.ncell; ++cl) {
    const double u[3] = {ux[cl], uy[cl], uz[cl]};
    set_equilibrium_cell(d, cl, rho[cl], u, p[cl]);
  }
  finish_init(d);
  return 0;
}

// Equilibrium initialisation from given zeroth moments Q[k][cell] (all 14 fields).
int orc_init_state(void* h, const double* Qin) {
  Domain& d = *static_cast<Domain*>(h);
#pragma omp parallel for schedule(static)
  for (int64_t cl = 0; cl < d.ncell; ++cl) {
    double Q[NF];
    for (int k = 0; k < NF; ++k) Q[k] = Qin[(int64_t)k * d.ncell + cl];
    const Closure c = closure(d.p, Q);
    double Phi[NF][3], feq[NF][NQ];
    flux(d.p, Q, c, Phi);
    equilibrium(d.c, Q, Phi, feq);
    for (int k = 0; k < NF; ++k)
      for (int i = 0; i < NQ; ++i) d.at(d.f, k, i, cl) = feq[k][i];
  }
  finish_init(d);
  return 0;
}

// Canonical populations f[k][i][cell] (pre-collision state).
void orc_get_populations(void* h, double* out) {
  Domain& d = *static_cast<Domain*>(h);
  std::memcpy(out, d.f.data(), sizeof(double) * d.f.size());
}

// Sets the state; at held x ends the inward population keeps the ghost value.
void orc_set_populations(void* h, const double* in) {
  Domain& d = *static_cast<Domain*>(h);
  std::memcpy(d.f.data(), in, sizeof(double) * d.f.size());
  if (d.p.bc_x == 1 && d.ghost_lo.empty()) record_ghosts(d);
  apply_held_inflow(d);
}

void orc_step(void* h, int n) {
  Domain& d = *static_cast<Domain*>(h);
  for (int s = 0; s < n; ++s) step_once(d);
}

// Zeroth moments Q[k][cell].
void orc_moments(void* h, double* out) {
  Domain& d = *static_cast<Domain*>(h);
#pragma omp parallel for schedule(static)
  for (int64_t cl = 0; cl < d.ncell; ++cl) {
    double Q[NF];
    macroscopic(d, cl, Q);
    for (int k = 0; k < NF; ++k) out[(int64_t)k * d.ncell + cl] = Q[k];
  }
}

// rho, u_x, u_y, u_z, T, p per cell: out[6][cell].
void orc_primitives(void* h, double* out) {
  Domain& d = *static_cast<Domain*>(h);
#pragma omp parallel for schedule(static)
  for (int64_t cl = 0; cl < d.ncell; ++cl) {
    double Q[NF];
    macroscopic(d, cl, Q);
    const Closure c = closure(d.p, Q);
    const double v[6] = {c.rho, c.u[0], c.u[1], c.u[2], c.T, c.p};
    for (int j = 0; j < 6; ++j) out[(int64_t)j * d.ncell + cl] = v[j];
  }
}

// Sensor of the current pre-collision state: theta (div u, physical units), chi
// and the blended rate omega_h, each [cell].
void orc_sensor(void* h, double* theta, double* chi, double* omega_h) {
  Domain& d = *static_cast<Domain*>(h);
#pragma omp parallel for schedule(static)
  for (int64_t cl = 0; cl < d.ncell; ++cl) {
    double f[NF][NQ], fo[NF][NQ];
    gather(d, d.f, cl, f);
    const CellOut o = collide_cell(d, f, fo);
    if (theta) theta[cl] = o.theta;
    if (chi) chi[cl] = o.chi;
    if (omega_h) omega_h[cl] = o.omega_h;
  }
}

// Single-state helpers for unit tests: equilibrium (98), flux (42), closure
// (rho, u, E, p, T, mu_T, kappa_T: 9) of one state Q[14] under this domain's
// parameters, the sensor response chi(s), and the D3Q7 constants.
void orc_equilibrium_of(void* h, const double* Q, double* feq) {
  Domain& d = *static_cast<Domain*>(h);
  const Closure c = closure(d.p, Q);
  double Phi[NF][3], fe[NF][NQ];
  flux(d.p, Q, c, Phi);
  equilibrium(d.c, Q, Phi, fe);
  for (int k = 0; k < NF; ++k)
    for (int i = 0; i < NQ; ++i) feq[k * NQ + i] = fe[k][i];
}

void orc_flux_of(void* h, const double* Q, double* Phi_out) {
  Domain& d = *static_cast<Domain*>(h);
  const Closure c = closure(d.p, Q);
  double Phi[NF][3];
  flux(d.p, Q, c, Phi);
  for (int k = 0; k < NF; ++k)
    for (int a = 0; a < 3; ++a) Phi_out[k * 3 + a] = Phi[k][a];
}

void orc_closure_of(void* h, const double* Q, double* out) {
  Domain& d = *static_cast<Domain*>(h);
  const Closure c = closure(d.p, Q);
  const double v[9] = {c.rho, c.u[0], c.u[1], c.u[2], c.E, c.p, c.T, c.mu_T, c.kappa_T};
  for (int j = 0; j < 9; ++j) out[j] = v[j];
}

double orc_chi_of(void* h, double s) { return sensor_chi(static_cast<Domain*>(h)->p, s); }

// One collision of a given pre-collision population set f[98] -> fout[98].
void orc_collide_of(void* h, const double* f, double* fout, double* theta_chi_omega) {
  Domain& d = *static_cast<Domain*>(h);
  double fi[NF][NQ], fo[NF][NQ];
  for (int k = 0; k < NF; ++k)
    for (int i = 0; i < NQ; ++i) fi[k][i] = f[k * NQ + i];
  const CellOut o = collide_cell(d, fi, fo);
  for (int k = 0; k < NF; ++k)
    for (int i = 0; i < NQ; ++i) fout[k * NQ + i] = fo[k][i];
  if (theta_chi_omega) {
    theta_chi_omega[0] = o.theta;
    theta_chi_omega[1] = o.chi;
    theta_chi_omega[2] = o.omega_h;
  }
}

void orc_lattice(double* w, int* e) {
  for (int i = 0; i < NQ; ++i) {
    w[i] = W[i];
    for (int a = 0; a < 3; ++a) e[i * 3 + a] = E[i][a];
  }
}

// Diagnostics (Sec. 3.2, Eq. 7). Velocity gradients by second-order central
// differences on the grid (periodic; one-sided at held x ends). mu_local follows
// the viscosity law of the domain.
void orc_diag_get(void* h, orc_diag* out) {
  Domain& d = *static_cast<Domain*>(h);
  const int nx = d.p.nx, ny = d.p.ny, nz = d.p.nz;
  std::vector<double> U(3 * (size_t)d.ncell), T(d.ncell);
  double s_rho = 0, s_m[3] = {0, 0, 0}, s_E = 0, s_ek = 0;
  double max_mach = 0, max_cfl = 0, min_rho = INFINITY, min_T = INFINITY, nonfinite = 0;
  for (int64_t cl = 0; cl < d.ncell; ++cl) {
    double Q[NF];
    macroscopic(d, cl, Q);
    bool finite = true;
    for (int k = 0; k < NF; ++k) finite = finite && std::isfinite(Q[k]);
    if (!finite) nonfinite += 1;
    const Closure c = closure(d.p, Q);
    for (int a = 0; a < 3; ++a) U[a * d.ncell + cl] = c.u[a];
    T[cl] = c.T;
    s_rho += Q[RHO];
    for (int a = 0; a < 3; ++a) s_m[a] += Q[MX + a];
    s_E += Q[EN];
    const double u2 = c.u[0] * c.u[0] + c.u[1] * c.u[1] + c.u[2] * c.u[2];
    s_ek += 0.5 * c.rho * u2;
    const double a_snd = std::sqrt(d.p.gamma * c.T);
    max_mach = std::fmax(max_mach, std::sqrt(u2) / a_snd);
    for (int a = 0; a < 3; ++a)
      max_cfl = std::fmax(max_cfl, (std::fabs(c.u[a]) + a_snd) * d.dt / d.p.dx);
    min_rho = std::fmin(min_rho, c.rho);
    min_T = std::fmin(min_T, c.T);
  }
  double s_sol = 0, s_dil = 0;
  for (int z = 0; z < nz; ++z)
    for (int y = 0; y < ny; ++y)
      for (int x = 0; x < nx; ++x) {
        const int64_t cl = d.cell(x, y, z);
        double g[3][3];  // g[a][b] = d_a u_b
        for (int a = 0; a < 3; ++a) {
          int lo[3] = {x, y, z}, hi[3] = {x, y, z};
          const int n = a == 0 ? nx : (a == 1 ? ny : nz);
          double span = 2.0;
          if (a == 0 && d.p.bc_x == 1) {
            lo[0] = x > 0 ? x - 1 : x;
            hi[0] = x < nx - 1 ? x + 1 : x;
            span = (double)(hi[0] - lo[0]);
          } else {
            lo[a] = (lo[a] - 1 + n) % n;
            hi[a] = (hi[a] + 1) % n;
          }
          const int64_t cl_lo = d.cell(lo[0], lo[1], lo[2]);
          const int64_t cl_hi = d.cell(hi[0], hi[1], hi[2]);
          for (int b = 0; b < 3; ++b)
            g[a][b] = span > 0 ? (U[b * d.ncell + cl_hi] - U[b * d.ncell + cl_lo]) / (span * d.p.dx)
                               : 0.0;
        }
        const double wx = g[1][2] - g[2][1], wy = g[2][0] - g[0][2], wz = g[0][1] - g[1][0];
        const double div = g[0][0] + g[1][1] + g[2][2];
        const double mu_loc = d.p.mu * sutherland_ratio(d.p, T[cl]);
        s_sol += mu_loc * (wx * wx + wy * wy + wz * wz);
        s_dil += mu_loc * div * div;
      }
  const double n = (double)d.ncell;
  out->step = (double)d.step;
  out->time = (double)d.step * d.dt;
  out->sum_rho = s_rho;
  out->sum_mx = s_m[0];
  out->sum_my = s_m[1];
  out->sum_mz = s_m[2];
  out->sum_E = s_E;
  out->ek_mean = s_ek / n;
  out->eps_s_raw = s_sol / n;
  out->eps_d_raw = 4.0 / 3.0 * s_dil / n;
  out->max_mach = max_mach;
  out->max_cfl = max_cfl;
  out->min_rho = min_rho;
  out->min_T = min_T;
  out->nonfinite = nonfinite;
}

}  // extern "C"
