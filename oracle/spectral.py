"""Spectral diagnostics of a periodic velocity field (Sec. 3.2): Eq. 7's dissipation
rates with curl and divergence taken spectrally and mu_local applied per cell in
physical space, and the shell-averaged kinetic-energy spectrum normalised so that
sum_k E(k) = <|u|^2> / 2.

TEST INFRASTRUCTURE (oracle): numpy FFTs on FP64 fields of shape (nz, ny, nx) on a
box of side 2 pi L with n points per axis (wavenumbers in units of 1/L).
"""
from __future__ import annotations

import numpy as np

T_SUTHERLAND = 0.4042


def _wavenumbers(shape, L_box):
    nz, ny, nx = shape
    kz = np.fft.fftfreq(nz, d=L_box / nz) * 2 * np.pi
    ky = np.fft.fftfreq(ny, d=L_box / ny) * 2 * np.pi
    kx = np.fft.fftfreq(nx, d=L_box / nx) * 2 * np.pi
    return np.meshgrid(kz, ky, kx, indexing="ij")


def grad_u(u, L_box):
    """g[a][b] = d_a u_b for u = (u_x, u_y, u_z), each (nz, ny, nx)."""
    KZ, KY, KX = _wavenumbers(u[0].shape, L_box)
    ks = (KX, KY, KZ)
    out = np.empty((3, 3) + u[0].shape)
    for b in range(3):
        uh = np.fft.fftn(u[b])
        for a in range(3):
            k = ks[a].copy()
            n_a = u[0].shape[2 - a]
            if n_a % 2 == 0:
                k[np.isclose(np.abs(k), np.pi * n_a / L_box)] = 0.0
            out[a, b] = np.real(np.fft.ifftn(1j * k * uh))
    return out


def mu_local(T, mu, T_ref, sutherland):
    if not sutherland:
        return np.full_like(T, mu)
    t = T / T_ref
    return mu * (1 + T_SUTHERLAND) * t ** 1.5 / (t + T_SUTHERLAND)


def dissipation(u, T, mu, T_ref, sutherland, rho_ref, L_box=2 * np.pi):
    """eps_s = <mu_loc |curl u|^2> / rho_ref, eps_d = 4/3 <mu_loc (div u)^2> / rho_ref."""
    g = grad_u(u, L_box)
    w = (g[1, 2] - g[2, 1], g[2, 0] - g[0, 2], g[0, 1] - g[1, 0])
    div = g[0, 0] + g[1, 1] + g[2, 2]
    m = mu_local(T, mu, T_ref, sutherland)
    eps_s = np.mean(m * (w[0] ** 2 + w[1] ** 2 + w[2] ** 2)) / rho_ref
    eps_d = 4.0 / 3.0 * np.mean(m * div ** 2) / rho_ref
    return float(eps_s), float(eps_d)


def energy_spectrum(u, L_box=2 * np.pi):
    """Shell-averaged E(k), shells of unit width around integer |k| L; returns
    (k, E) with sum(E) = <|u|^2> / 2."""
    n = u[0].size
    KZ, KY, KX = _wavenumbers(u[0].shape, L_box)
    kmag = np.sqrt(KX ** 2 + KY ** 2 + KZ ** 2) * (L_box / (2 * np.pi))
    shell = np.rint(kmag).astype(np.int64)
    e = np.zeros(shell.max() + 1)
    for b in range(3):
        uh = np.fft.fftn(u[b]) / n
        np.add.at(e, shell.ravel(), 0.5 * np.abs(uh.ravel()) ** 2)
    return np.arange(len(e)), e
