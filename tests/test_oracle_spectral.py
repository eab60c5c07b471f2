"""Spectral diagnostics of Sec. 3.2 (oracle side) against closed forms."""
import math

import numpy as np
import pytest

from oracle import spectral


def _tgv(n, U0=1.0):
    x = np.arange(n) * 2 * math.pi / n
    Z, Y, X = np.meshgrid(x, x, x, indexing="ij")
    u = U0 * np.sin(X) * np.cos(Y) * np.cos(Z)
    v = -U0 * np.cos(X) * np.sin(Y) * np.cos(Z)
    return np.stack([u, v, np.zeros_like(u)])


def test_tgv_initial_field_closed_forms():
    """Spectral derivatives are exact for the band-limited TGV field: eps_s = 3/4 mu U0^2
    (uniform T, so mu_local = mu), eps_d = 0; all kinetic energy sits in the shell
    |k| L = sqrt(3) -> 2 and sums to <|u|^2>/2 = U0^2 / 8."""
    n = 16
    u = _tgv(n, U0=1.3)
    T = np.full(u[0].shape, 0.7)
    es, ed = spectral.dissipation(u, T, 2e-3, 0.7, True, 1.0)
    assert es == pytest.approx(0.75 * 2e-3 * 1.3 ** 2, rel=1e-12)
    assert abs(ed) < 1e-25
    k, E = spectral.energy_spectrum(u)
    assert E.sum() == pytest.approx(1.3 ** 2 / 8, rel=1e-12)
    assert E[2] == pytest.approx(E.sum(), rel=1e-12)


def test_parseval_and_random_gradients():
    """Sum of the spectrum equals <|u|^2>/2 for any field; spectral gradients of a
    random band-limited field match its analytic derivatives."""
    rng = np.random.default_rng(4)
    n = 12
    x = np.arange(n) * 2 * math.pi / n
    Z, Y, X = np.meshgrid(x, x, x, indexing="ij")
    u = np.zeros((3, n, n, n))
    du = np.zeros((3, 3, n, n, n))
    for _ in range(6):
        k = rng.integers(-4, 5, size=3)
        a, ph, b = rng.standard_normal(), rng.random() * 6.28, rng.integers(0, 3)
        arg = k[0] * X + k[1] * Y + k[2] * Z + ph
        u[b] += a * np.sin(arg)
        for ax in range(3):
            du[ax, b] += a * k[ax] * np.cos(arg)
    g = spectral.grad_u(u, 2 * math.pi)
    assert np.allclose(g, du, atol=1e-10)
    _, E = spectral.energy_spectrum(u)
    assert E.sum() == pytest.approx(0.5 * np.mean((u ** 2).sum(0)), rel=1e-12)
