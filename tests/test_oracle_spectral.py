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


@pytest.mark.parametrize("component,T_axis", [(0, 1), (0, 2), (1, 2), (2, 1)])
def test_wave_dissipation_closed_forms(component, T_axis):
    """Spectral Eq. 7 on one velocity wave u_c = A sin(k x) with a temperature that
    depends only on y or z (Sutherland viscosity): the spectral derivative is exact,
    <cos^2> = 1/2 on the grid, and mu_local averages over the temperature profile, so
    eps_d = 4/3 mbar A^2 k^2 / 2 / rho_ref for the compressive wave (c = x) and
    eps_s = mbar A^2 k^2 / 2 / rho_ref for a shear wave; the other rate is zero. mbar
    uses the form of Sutherland's law printed with the TGV setup (Sec. 3.2),
    mu (T/T_ref)^{3/2} (T_ref + S)/(T + S), S = 0.4042 T_ref."""
    from paper_2608_13437_gb300 import inputs
    nx, ny, nz, k, A, T0, mu, T_ref, rho_ref = 16, 6, 8, 3, 0.4, 0.9, 0.037, 0.8, 1.7
    f = inputs.separable_wave_fields(nx, ny, nz, A, k, 1.0, T0, 0.35, component, T_axis)
    T = f["p"] / f["rho"]
    S = 0.4042 * T_ref
    mbar = float(np.mean(mu * (f["T_line"] / T_ref) ** 1.5 * (T_ref + S) / (f["T_line"] + S)))
    # dissipation() takes each axis to span 2 pi; only x carries a velocity gradient,
    # so the y and z extents do not enter
    u = np.stack([f["ux"], f["uy"], f["uz"]])
    es, ed = spectral.dissipation(u, T, mu, T_ref, True, rho_ref)
    if component == 0:
        assert ed == pytest.approx(4.0 / 3.0 * mbar * A * A * k * k / 2.0 / rho_ref, rel=1e-12)
        assert abs(es) < 1e-20
    else:
        assert es == pytest.approx(mbar * A * A * k * k / 2.0 / rho_ref, rel=1e-12)
        assert abs(ed) < 1e-20
