"""Linearised relaxed Navier-Stokes-Fourier system of Eq. 2 about a gas at rest.

TEST INFRASTRUCTURE (oracle). A plane perturbation ~ exp(i k x) of the uniform
state (rho0, u = 0, T0, tau = q = 0) obeys d v/dt = M(k) v; the oracle's wave
decay tests compare simulated Fourier amplitudes with exp(M t) v0.

Shear wave, v = (rho u_y, tau_xy):
    d_t(rho u_y) = d_x tau_xy
    d_t tau_xy   = (mu / tau_R) d_x u_y - tau_xy / tau_R
(momentum flux -tau; stress flux -(mu/tau_R) Lambda with Lambda_{xy,x} = u_y).
Eigenvalues satisfy rho0 s (1 + s tau_R) = -mu k^2.

Longitudinal (acoustic) wave, v = (rho, rho u_x, E, tau_xx, q_x):
    d_t rho      = -d_x (rho u_x)
    d_t(rho u_x) = -d_x (p - tau_xx),            p' = (gamma - 1) E'
    d_t E        = -d_x ((E0 + p0) u_x + q_x)
    d_t tau_xx   = (4/3)(mu / tau_R) d_x u_x - tau_xx / tau_R     (Lambda_{xx,x} = 4/3 u_x)
    d_t q_x      = -d_x (K T) / tau_q - q_x / tau_q
with T' = ((gamma - 1) E' - T0 rho') / rho0 and K = d(kappa_T T)/dT at T0 (kappa for a
constant conductivity; kappa (1 + T0 r'(T0)) under Sutherland's law r(T)).
Small-k limits (textbook): sound s = +-i a0 k - Gamma k^2 with
Gamma = ((4/3) mu + (gamma - 1) K / c_p) / (2 rho0), c_p = gamma / (gamma - 1); the
entropy mode s = -K k^2 / (rho0 c_p); shear s = -mu k^2 / rho0.

An extra numerical diffusivity nu_num on every field (Eq. 6) shifts every
eigenvalue by -nu_num k^2.
"""
from __future__ import annotations

import numpy as np
from scipy.linalg import expm

T_SUTHERLAND = 0.4042


def sutherland_slope(T0: float, T_ref: float) -> float:
    """d r / d T at T0 for r(T) = (1 + T_S) t^{3/2} / (t + T_S), t = T / T_ref."""
    t = T0 / T_ref
    num = 1.5 * t ** 0.5 * (t + T_SUTHERLAND) - t ** 1.5
    return (1.0 + T_SUTHERLAND) * num / (t + T_SUTHERLAND) ** 2 / T_ref


def shear_matrix(k: float, rho0: float, mu: float, tau_R: float, nu_num: float = 0.0):
    ik = 1j * k
    M = np.array([[0.0, ik], [ik * mu / (tau_R * rho0), -1.0 / tau_R]], dtype=complex)
    return M - nu_num * k * k * np.eye(2)


def acoustic_matrix(k: float, rho0: float, T0: float, gamma: float, mu: float, kappa: float,
                    tau_R: float, tau_q: float, nu_num: float = 0.0,
                    sutherland: bool = False, T_ref: float | None = None):
    ik = 1j * k
    p0 = rho0 * T0
    E0 = p0 / (gamma - 1.0)
    K = kappa
    if sutherland:
        r = (1.0 + T_SUTHERLAND) * (T0 / T_ref) ** 1.5 / (T0 / T_ref + T_SUTHERLAND)
        mu = mu * r
        K = kappa * (r + T0 * sutherland_slope(T0, T_ref))
    g1 = gamma - 1.0
    M = np.zeros((5, 5), dtype=complex)
    # rho
    M[0, 1] = -ik
    # rho u_x: -(ik)((gamma-1) E - tau)
    M[1, 2] = -ik * g1
    M[1, 3] = ik
    # E: -(ik)((E0 + p0) m / rho0 + q)
    M[2, 1] = -ik * (E0 + p0) / rho0
    M[2, 4] = -ik
    # tau_xx
    M[3, 1] = ik * (4.0 / 3.0) * mu / (tau_R * rho0)
    M[3, 3] = -1.0 / tau_R
    # q_x: -(ik) K T' / tau_q - q / tau_q
    M[4, 0] = -ik * K / tau_q * (-T0 / rho0)
    M[4, 2] = -ik * K / tau_q * (g1 / rho0)
    M[4, 4] = -1.0 / tau_q
    return M - nu_num * k * k * np.eye(5)


def evolve(M: np.ndarray, v0, t: float) -> np.ndarray:
    return expm(M * t) @ np.asarray(v0, dtype=complex)


def fourier_amplitude(field: np.ndarray, k_index: int, axis: int = -1) -> complex:
    """Complex amplitude A of a field A e^{i k x} + c.c. along `axis` (mean over
    the other axes): A = (1/N) sum_x field e^{-i k x}."""
    f = np.moveaxis(np.asarray(field), axis, -1)
    n = f.shape[-1]
    x = np.arange(n)
    c = (f * np.exp(-2j * np.pi * k_index * x / n)).sum(axis=-1) / n
    return complex(np.mean(c))
