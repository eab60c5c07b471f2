"""Becker's viscous shock (Sec. 3.1): the exact steady profile of a plane shock in a
gas with constant viscosity mu and Prandtl number 3/4.

TEST INFRASTRUCTURE (oracle). Derivation written out here from the 1-D steady
Navier-Stokes-Fourier equations in the shock frame (mass flux m = rho u constant):
  momentum  m u + p - (4/3) mu u' = P,
  energy    m (h + u^2/2) - (4/3) mu u u' - kappa T' = m H,
with h = c_p T, c_p = gamma/(gamma-1) (gas constant 1, T = p/rho). For Pr = mu c_p /
kappa = 3/4 the energy equation is satisfied by h + u^2/2 = H everywhere, so
T = (H - u^2/2)/c_p and p = rho T = (m/u) (gamma-1)/gamma (H - u^2/2). Multiplying the
momentum balance by u gives
  (4/3) mu u u' = m (gamma+1)/(2 gamma) (u - u1)(u - u2),
whose zeros u1 > u2 are the upstream and downstream (Rankine-Hugoniot) speeds.
Partial fractions integrate it to the implicit profile
  x(u) = C [u1 ln(u1 - u) - u2 ln(u - u2)] / (u1 - u2),  C = 8 gamma mu / (3 m (gamma+1)),
monotone for u2 < u < u1 (x increases downstream).
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np


@dataclass(frozen=True)
class BeckerShock:
    gamma: float
    mu: float
    rho1: float   # upstream (pre-shock) state, at rest in the lab frame
    p1: float
    mach: float   # shock Mach number relative to the upstream gas

    @property
    def c1(self) -> float:
        return math.sqrt(self.gamma * self.p1 / self.rho1)

    @property
    def u1(self) -> float:
        """Upstream speed in the shock frame = shock speed in the lab frame."""
        return self.mach * self.c1

    @property
    def u2(self) -> float:
        g, M = self.gamma, self.mach
        return self.u1 * ((g - 1.0) * M * M + 2.0) / ((g + 1.0) * M * M)

    @property
    def m(self) -> float:
        return self.rho1 * self.u1

    @property
    def cp(self) -> float:
        return self.gamma / (self.gamma - 1.0)

    @property
    def H(self) -> float:
        return self.cp * self.p1 / self.rho1 + 0.5 * self.u1 ** 2

    @property
    def kappa(self) -> float:
        """Conductivity giving Pr = mu c_p / kappa = 3/4."""
        return self.mu * self.cp / 0.75

    def x_of_u(self, u):
        u1, u2 = self.u1, self.u2
        C = 8.0 * self.gamma * self.mu / (3.0 * self.m * (self.gamma + 1.0))
        return C * (u1 * np.log(u1 - u) - u2 * np.log(u - u2)) / (u1 - u2)

    def u_of_x(self, x):
        """Shock-frame speed at position x (x = 0 where u = (u1 + u2)/2), by bisection."""
        x = np.asarray(x, dtype=np.float64)
        u1, u2 = self.u1, self.u2
        x0 = self.x_of_u(0.5 * (u1 + u2))
        lo = np.full_like(x, u2)
        hi = np.full_like(x, u1)
        with np.errstate(divide="ignore"):  # far tails reach u1 or u2 to round-off
            for _ in range(100):  # x_of_u decreases from +inf (u -> u2) to -inf (u -> u1)
                mid = 0.5 * (lo + hi)
                right = (self.x_of_u(mid) - x0) > x  # mid lies downstream of x: u(x) > mid
                lo = np.where(right, mid, lo)
                hi = np.where(right, hi, mid)
        return 0.5 * (lo + hi)

    def shock_frame(self, x):
        """rho, u, p, T, tau_xx, q_x at shock-frame positions x (flow in +x)."""
        u = self.u_of_x(x)
        rho = self.m / u
        T = (self.H - 0.5 * u * u) / self.cp
        p = rho * T
        # (4/3) mu u' from the closed form; q = -kappa T' = kappa u u' / c_p
        du = self.m * (self.gamma + 1.0) / (2.0 * self.gamma) * (u - self.u1) * (u - self.u2) / u
        du = du / (4.0 / 3.0 * self.mu)
        tau_xx = 4.0 / 3.0 * self.mu * du
        q_x = self.kappa * u * du / self.cp
        return rho, u, p, T, tau_xx, q_x, du

    def lab(self, x, t, x_shock0):
        """Lab-frame fields of the shock moving in +x into the gas at rest: the shock
        centre is at x_shock0 + u1 t; upstream is to the right. Returns rho, u, p,
        tau_xx, q_x and du/dx (lab)."""
        xi = np.asarray(x, dtype=np.float64) - (x_shock0 + self.u1 * t)
        rho, U, p, T, tau_s, q_s, du_s = self.shock_frame(-xi)
        # shock-frame flow runs in -x in the lab: velocity -U, shifted by the shock speed
        u_lab = self.u1 - U
        # d/dx of u_lab(x) = -d/dx U(-xi) = +U'(-xi): same stress; heat flux flips sign
        return rho, u_lab, p, tau_s, -q_s, du_s

    def downstream(self):
        g = self.gamma
        rho2 = self.m / self.u2
        T2 = (self.H - 0.5 * self.u2 ** 2) / self.cp
        return rho2, self.u1 - self.u2, rho2 * T2

    def max_signal_speed(self) -> float:
        rho2, ul2, p2 = self.downstream()
        return max(abs(ul2) + math.sqrt(self.gamma * p2 / rho2), self.c1)

    def thickness(self, n: int = 200001) -> float:
        """Maximum-slope thickness (rho2 - rho1) / max |d rho/dx| of the profile."""
        rho2, _, _ = self.downstream()
        half = 25.0 * self.mu / (self.rho1 * self.c1)  # several shock widths
        x = np.linspace(-half, half, n)
        rho = self.shock_frame(x)[0]
        return (rho2 - self.rho1) / np.max(np.abs(np.diff(rho)) / (x[1] - x[0]))


def paper_case() -> BeckerShock:
    """Sec. 3.1: M_s = 2, Re_s = rho0 c0 M_s L / mu = 1000 on unit scales (mu = 2e-3),
    gamma = 1.4, Pr = 3/4; upstream rho0 = 1, c0 = 1."""
    g = 1.4
    return BeckerShock(gamma=g, mu=2e-3, rho1=1.0, p1=1.0 / g, mach=2.0)


def initial_moments(b: BeckerShock, n: int, ny: int, nz: int, x_shock0: float) -> np.ndarray:
    """Zeroth moments Q (14, nz, ny, n) of the lab-frame Becker shock at t = 0 on cell
    centres of [0, 1]: rho, rho u, E, and the stress and heat flux at their Newtonian and
    Fourier values of the profile (tau_xx = 4/3 mu u', tau_yy = tau_zz = -2/3 mu u',
    q_x = -kappa T')."""
    x = (np.arange(n) + 0.5) / n
    rho, u, p, tau_xx, q_x, du = b.lab(x, 0.0, x_shock0)
    Q = np.zeros((14, nz, ny, n))
    Q[0] = rho
    Q[1] = rho * u
    Q[4] = p / (b.gamma - 1.0) + 0.5 * rho * u * u
    Q[5] = tau_xx
    Q[6] = -0.5 * tau_xx
    Q[7] = -0.5 * tau_xx
    Q[11] = q_x
    return Q
