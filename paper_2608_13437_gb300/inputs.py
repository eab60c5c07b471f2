"""Seeded, synthetic workloads of the compressible-NSF lattice Boltzmann path.

This module only states problems: grid sizes, physical parameters derived from
the dimensionless groups of each benchmark, initial-state parameters and seeded
random draws. It holds none of the scheme's arithmetic (no equilibrium, flux,
closure, sensor or streaming), so both the CUDA library and the CPU oracle can
take their inputs from it.

Workloads (Sec. 3 of the paper, resized as stated):
  * supersonic Taylor-Green vortex (Sec. 3.2): periodic [0, 2 pi)^3, gamma 1.4,
    Pr 0.71, uniform T0, Sutherland viscosity; C_sigma 40, J_min 1e-2,
    omega_min 1.987, tau_R = tau_q = 5e-3, CFL 0.1.
  * Sod shock tube (Sec. 3.1): gamma 1.4, (rho, u, p) = (1, 0, 1) | (0.125, 0, 0.1),
    constant mu = 1e-6, C_sigma 20, J_min 3e-3, omega_min 1, CFL 0.35,
    tau_R = tau_q = 5 dt, x ends held at the initial states.
  * 64 independent TGV domains with sizes, Mach and Reynolds numbers drawn from
    SplitMix64(seed 0).
"""
from __future__ import annotations

import math

import numpy as np

GAMMA = 1.4

# Background dissipation factor f_mu per grid size. The paper lists 1.8 at 64^3,
# 0.9 at 128^3 and 1e-2 at 256^3 and 512^3 (Sec. 3.2), and 3e-2, 8e-3, 1e-2 at
# 192, 320, 384 (Table 7). Other sizes take the value of the next coarser listed size.
_F_MU_LISTED = {64: 1.8, 128: 0.9, 192: 3e-2, 256: 1e-2, 320: 8e-3, 384: 1e-2, 512: 1e-2}


def tgv_f_mu(n: int) -> float:
    """Listed sizes take their value; sizes below 64 take the 64^3 value and the
    others that of the next listed size up (96 -> 0.9)."""
    if n in _F_MU_LISTED:
        return _F_MU_LISTED[n]
    finer = [k for k in sorted(_F_MU_LISTED) if k >= n]
    return _F_MU_LISTED[finer[0]] if finer else _F_MU_LISTED[max(_F_MU_LISTED)]


def tgv_params(n: int, M0: float = 1.25, Re: float = 1000.0, Pr: float = 0.71,
               U0: float = 1.0, rho0: float = 1.0, L: float = 1.0, tau_relax: float = 5e-3,
               cfl: float = 0.1, C_sigma: float = 40.0, J_min: float = 1e-2,
               omega_min: float = 1.987, f_mu: float | None = None) -> dict:
    """Parameters of the supersonic TGV on an n^3 periodic box of side 2 pi L.

    mu = rho0 U0 L / Re, kappa = gamma mu / ((gamma - 1) Pr) (gas constant 1, since
    T = p / rho), T_ref = T0 = U0^2 / (gamma M0^2). lambda_ref = U0 + a0 = U0 (1 + 1/M0)
    is the largest signal speed of the initial state, used with the CFL number.
    """
    mu = rho0 * U0 * L / Re
    T0 = U0 * U0 / (GAMMA * M0 * M0)
    return dict(
        nx=n, ny=n, nz=n, dx=2.0 * math.pi * L / n, bc_x=0, dt=0.0, cfl=cfl,
        lambda_ref=U0 * (1.0 + 1.0 / M0), gamma=GAMMA, mu=mu,
        kappa=GAMMA * mu / ((GAMMA - 1.0) * Pr), tau_R=tau_relax, tau_q=tau_relax,
        relax_in_dt=0, T_ref=T0, sutherland=1, source_mode=0,
        f_mu=tgv_f_mu(n) if f_mu is None else f_mu, C_sigma=C_sigma, J_min=J_min,
        omega_min=omega_min, sensor_mode=0, collide=1)


def tgv_init(M0: float = 1.25, U0: float = 1.0, rho0: float = 1.0) -> dict:
    return dict(U0=U0, M0=M0, rho0=rho0)


# Sod: left/right states (rho, u, p) (Sec. 3.1).
SOD_LEFT = (1.0, 0.0, 1.0)
SOD_RIGHT = (0.125, 0.0, 0.1)
# Largest |u| + a of the exact Sod solution (star region right of the contact),
# written by tests/golden/gen_golden.py from the oracle's exact Riemann solver.
SOD_LAMBDA_MAX = 2.1915661028007705


def sod_params(n: int, ny: int = 4, nz: int = 4, cfl: float = 0.35, mu: float = 1e-6,
               Pr: float = 0.75, C_sigma: float = 20.0, J_min: float = 3e-3,
               omega_min: float = 1.0, f_mu: float = 0.0, relax_steps: float = 5.0) -> dict:
    """Sod tube on [0, 1] with n cells along x (held ends), periodic y, z.

    The time step follows from the CFL number against the largest signal speed of
    the exact solution; tau_R = tau_q = relax_steps * dt as in Sec. 3.1 (given in
    units of dt, relax_in_dt = 1).
    """
    dx = 1.0 / n
    return dict(
        nx=n, ny=ny, nz=nz, dx=dx, bc_x=1, dt=0.0, cfl=cfl, lambda_ref=SOD_LAMBDA_MAX,
        gamma=GAMMA, mu=mu, kappa=GAMMA * mu / ((GAMMA - 1.0) * Pr),
        tau_R=relax_steps, tau_q=relax_steps, relax_in_dt=1, T_ref=1.0, sutherland=0,
        source_mode=0, f_mu=f_mu, C_sigma=C_sigma, J_min=J_min, omega_min=omega_min,
        sensor_mode=0, collide=1)


def sod_steps(dt: float, t_end: float = 0.2) -> int:
    return int(round(t_end / dt))


# Becker's viscous shock (Sec. 3.1): M_s = 2 into gas at rest (rho, c) = (1, 1), constant
# mu = 2e-3 (Re_s = rho c M_s L / mu = 1000), Pr = 3/4, CFL 0.125, tau_R = tau_q = 5 dt,
# shock centre at x = 0.25 of [0, 1] at t = 0, compared at t = 0.2.
BECKER_MU = 2e-3
BECKER_MACH = 2.0
BECKER_X0 = 0.25
# Largest |u| + a of the exact Becker solution (downstream state), written by
# tests/golden/gen_golden.py from the oracle's Becker solver.
BECKER_LAMBDA_MAX = 2.5490381056766580


def becker_params(n: int, ny: int = 4, nz: int = 4, cfl: float = 0.125,
                  relax_steps: float = 5.0) -> dict:
    """Becker tube on [0, 1] with n cells along x (held ends), periodic y, z."""
    cp = GAMMA / (GAMMA - 1.0)
    return dict(
        nx=n, ny=ny, nz=nz, dx=1.0 / n, bc_x=1, dt=0.0, cfl=cfl, lambda_ref=BECKER_LAMBDA_MAX,
        gamma=GAMMA, mu=BECKER_MU, kappa=BECKER_MU * cp / 0.75, tau_R=relax_steps,
        tau_q=relax_steps, relax_in_dt=1, T_ref=1.0, sutherland=0, source_mode=0, f_mu=0.0,
        C_sigma=20.0, J_min=3e-3, omega_min=1.0, sensor_mode=0, collide=1)


# ---------------------------------------------------------------------------
# Seeded generators
# ---------------------------------------------------------------------------
_MASK = (1 << 64) - 1


class SplitMix64:
    """SplitMix64 (Steele, Lea, Flood 2014): 64-bit state, golden-ratio increment."""

    def __init__(self, seed: int):
        self.state = seed & _MASK

    def next_u64(self) -> int:
        self.state = (self.state + 0x9E3779B97F4A7C15) & _MASK
        z = self.state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _MASK
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _MASK
        return z ^ (z >> 31)

    def uniform(self) -> float:
        """Uniform in [0, 1) from the top 53 bits."""
        return (self.next_u64() >> 11) * (1.0 / (1 << 53))


BATCH_SIZES = (32, 48, 64, 96, 128)
# The TGV initial pressure p0 + rho0 U0^2 / 16 (cos 2x + cos 2y)(cos 2z + 2) has its
# minimum p0 - 3 rho0 U0^2 / 8 at grid nodes (x = y = pi/2, z = 0). With
# p0 = rho0 U0^2 / (gamma M0^2) and uniform T0 the minimum density is
# rho0 (1 - 3 gamma M0^2 / 8): negative for M0 > sqrt(8 / (3 gamma)) = 1.380, and a
# near-vacuum below it. Draws must keep it at or above 5 % of rho0.
TGV_RHO_MIN_FRACTION = 0.05
TGV_M0_ADMISSIBLE = math.sqrt((1.0 - TGV_RHO_MIN_FRACTION) * 8.0 / (3.0 * GAMMA))


def batch_domains(n_domains: int = 64, seed: int = 0, sizes=BATCH_SIZES,
                  m0_range=(0.3, 1.5), re_range=(100.0, 1600.0)) -> list[dict]:
    """Independent periodic TGV domains: per domain, in order, a size index uniform
    in `sizes`, then M0 ~ U[0.3, 1.5], then Re ~ U[100, 1600]. An M0 draw whose
    initial state has (near-)vacuum regions (M0 >= TGV_M0_ADMISSIBLE) is rejected and
    drawn again from the same stream, so M0 is uniform on the admissible part."""
    rng = SplitMix64(seed)
    out = []
    for d in range(n_domains):
        n = sizes[min(int(rng.uniform() * len(sizes)), len(sizes) - 1)]
        redraws = 0
        while True:
            M0 = m0_range[0] + (m0_range[1] - m0_range[0]) * rng.uniform()
            if M0 < TGV_M0_ADMISSIBLE:
                break
            redraws += 1
        Re = re_range[0] + (re_range[1] - re_range[0]) * rng.uniform()
        out.append(dict(index=d, n=n, M0=M0, Re=Re, redraws=redraws))
    return out


def batch_params(domains: list[dict]) -> list[tuple[dict, dict]]:
    return [(tgv_params(d["n"], M0=d["M0"], Re=d["Re"]), tgv_init(M0=d["M0"]))
            for d in domains]


def random_labels(shape, seed: int, dtype=np.float32) -> np.ndarray:
    """Distinct finite values, one per population slot, for permutation tests."""
    rng = np.random.default_rng(seed)
    n = int(np.prod(shape))
    vals = (np.arange(n, dtype=np.float64) + 1.0) * (1.0 + 0.25 * rng.random(n))
    rng.shuffle(vals)
    return vals.astype(dtype).reshape(shape)


def random_smooth_state(nx: int, ny: int, nz: int, seed: int, amp: float = 0.1,
                        modes: int = 3) -> dict:
    """Smooth periodic fields rho, u, p: a few random low Fourier modes on top of
    (1, 0, 1). Returns float64 arrays of shape (nz, ny, nx)."""
    rng = np.random.default_rng(seed)
    z, y, x = np.meshgrid(np.arange(nz) / nz, np.arange(ny) / ny, np.arange(nx) / nx,
                          indexing="ij")

    def field():
        acc = np.zeros((nz, ny, nx))
        for _ in range(modes):
            k = rng.integers(0, 3, size=3)
            ph = rng.random() * 2 * math.pi
            acc += rng.standard_normal() * np.sin(2 * math.pi * (k[0] * x + k[1] * y + k[2] * z) + ph)
        return acc / modes

    rho = 1.0 + amp * field()
    p = 1.0 + amp * field()
    u = [amp * field() for _ in range(3)]
    return dict(rho=rho, ux=u[0], uy=u[1], uz=u[2], p=p)


def tgv_fields(n: int, M0: float = 1.25, U0: float = 1.0, rho0: float = 1.0,
               dtype=np.float32) -> np.ndarray:
    """The TGV initial fields of Sec. 3.2 on the n^3 nodes (i, j, l) * 2 pi / n, as one
    (5, n, n, n) array [z][y][x] of rho, u_x, u_y, u_z, p (input data for callers that
    supply their own initial state)."""
    h = 2.0 * math.pi / n
    x = np.arange(n) * h
    sx, cx, c2x = np.sin(x), np.cos(x), np.cos(2 * x)
    p0 = rho0 * U0 * U0 / (GAMMA * M0 * M0)
    T0 = p0 / rho0
    out = np.empty((5, n, n, n), dtype=dtype)
    for z in range(n):
        cz = math.cos(z * h)
        c2z = math.cos(2 * z * h)
        out[1, z] = U0 * sx[None, :] * cx[:, None] * cz
        out[2, z] = -U0 * cx[None, :] * sx[:, None] * cz
        out[3, z] = 0.0
        p = p0 + rho0 * U0 * U0 / 16.0 * (c2x[None, :] + c2x[:, None]) * (c2z + 2.0)
        out[4, z] = p
        out[0, z] = p / T0
    return out


def separable_wave_fields(nx: int, ny: int, nz: int, A: float, k: int, rho0: float, T0: float,
                          dT: float = 0.0, component: int = 0, T_axis: int = 1) -> dict:
    """A single velocity wave u_component = A sin(k x) on the nodes x_i = 2 pi i / nx
    (component 0: compressive, 1 or 2: shear), uniform density rho0 and a temperature
    T = T0 (1 + dT cos(2 pi j / n_T)) that varies along T_axis (1: y, 2: z) only, so
    the velocity and the temperature are functions of different coordinates. Returns
    float64 rho, ux, uy, uz, p of shape (nz, ny, nx) and the 1-D temperature profile
    T_line (input data for diagnostics with closed forms)."""
    x = np.arange(nx) * 2.0 * math.pi / nx
    n_T = ny if T_axis == 1 else nz
    T_line = T0 * (1.0 + dT * np.cos(2.0 * math.pi * np.arange(n_T) / n_T))
    shape = (nz, ny, nx)
    u = [np.zeros(shape) for _ in range(3)]
    u[component] = np.broadcast_to(A * np.sin(k * x), shape).copy()
    T = np.broadcast_to(T_line[:, None] if T_axis == 1 else T_line[:, None, None], shape)
    rho = np.full(shape, rho0)
    return dict(rho=rho, ux=u[0], uy=u[1], uz=u[2], p=rho * T, T_line=T_line)
