"""Spectral diagnostics on the device (Sec. 3.2): Eq. 7's dissipation rates with curl
and divergence taken spectrally (torch.fft, i.e. cuFFT) and mu_local applied per cell in
physical space, and the shell-averaged kinetic-energy spectrum normalised so that
sum_k E(k) = <|u|^2> / 2. Inputs are the primitive fields that lbm_moments(LBM_MOM_PRIM)
writes (rho, u_x, u_y, u_z, T, p), as a device tensor (6, nz, ny, nx), on a periodic box
of side L_box per axis.
"""
from __future__ import annotations

import math

T_SUTHERLAND = 0.4042


def _k(n, L_box, device, dtype):
    import torch
    k = torch.fft.fftfreq(n, d=L_box / n, device=device, dtype=dtype) * (2 * math.pi)
    if n % 2 == 0:  # no derivative of the Nyquist mode of a real field
        k[n // 2] = 0.0
    return k


def gradients(u, L_box=2 * math.pi):
    """g[a][b] = d_a u_b (3, 3, nz, ny, nx) for u (3, nz, ny, nx)."""
    import torch
    nz, ny, nx = u.shape[1:]
    dt = u.dtype
    kx = _k(nx, L_box, u.device, dt).view(1, 1, nx)
    ky = _k(ny, L_box, u.device, dt).view(1, ny, 1)
    kz = _k(nz, L_box, u.device, dt).view(nz, 1, 1)
    uh = torch.fft.fftn(u, dim=(1, 2, 3))
    out = torch.empty((3, 3) + tuple(u.shape[1:]), dtype=dt, device=u.device)
    for a, k in enumerate((kx, ky, kz)):
        out[a] = torch.fft.ifftn(1j * k * uh, dim=(1, 2, 3)).real
    return out


def dissipation(prim, mu, T_ref, sutherland, rho_ref, L_box=2 * math.pi):
    """(eps_s, eps_d) of Eq. 7 from primitive fields (6, nz, ny, nx) (FP64 recommended)."""
    import torch
    g = gradients(prim[1:4], L_box)
    wx, wy, wz = g[1, 2] - g[2, 1], g[2, 0] - g[0, 2], g[0, 1] - g[1, 0]
    div = g[0, 0] + g[1, 1] + g[2, 2]
    T = prim[4]
    if sutherland:
        t = T / T_ref
        m = mu * (1 + T_SUTHERLAND) * t ** 1.5 / (t + T_SUTHERLAND)
    else:
        m = torch.full_like(T, mu)
    eps_s = torch.mean(m * (wx * wx + wy * wy + wz * wz)) / rho_ref
    eps_d = 4.0 / 3.0 * torch.mean(m * div * div) / rho_ref
    return float(eps_s), float(eps_d)


def energy_spectrum(u, L_box=2 * math.pi):
    """(k, E(k)) over unit-width shells of |k| L; sum(E) = <|u|^2> / 2."""
    import torch
    nz, ny, nx = u.shape[1:]
    dt = u.dtype
    kx = _k_full(nx, L_box, u.device, dt).view(1, 1, nx)
    ky = _k_full(ny, L_box, u.device, dt).view(1, ny, 1)
    kz = _k_full(nz, L_box, u.device, dt).view(nz, 1, 1)
    kmag = torch.sqrt(kx * kx + ky * ky + kz * kz) * (L_box / (2 * math.pi))
    shell = torch.round(kmag).to(torch.int64).reshape(-1)
    n = nx * ny * nz
    e = torch.zeros(int(shell.max()) + 1, dtype=dt, device=u.device)
    for b in range(3):
        uh = torch.fft.fftn(u[b]) / n
        e.index_add_(0, shell, (0.5 * uh.abs() ** 2).reshape(-1))
    return torch.arange(len(e), device=u.device), e


def _k_full(n, L_box, device, dtype):
    import torch
    return torch.fft.fftfreq(n, d=L_box / n, device=device, dtype=dtype) * (2 * math.pi)
