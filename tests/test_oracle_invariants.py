"""Invariants of the oracle's full step: conservation, fixed points, streaming as an
exact permutation, axis symmetry, held-boundary consistency, and the TGV initial
diagnostics against their closed forms."""
import math

import numpy as np
import pytest

from conftest import make_oracle
from paper_2608_13437_gb300 import inputs

NF, NQ = 14, 7


def _tgv_like(nx, ny, nz, **kw):
    p = inputs.tgv_params(8)
    p.update(nx=nx, ny=ny, nz=nz, dx=2 * math.pi / max(nx, ny, nz))
    p.update(kw)
    return p


def test_conservation_periodic(oracle_mod):
    """S = 0 for rho, rho u, E (Eq. 2) and streaming only moves populations, so the
    totals stay at their initial values to round-off; the sensor is active."""
    p = _tgv_like(12, 10, 8, f_mu=0.5, C_sigma=40.0, J_min=1e-3, tau_R=0.05, tau_q=0.05)
    o = make_oracle(p)
    s = inputs.random_smooth_state(12, 10, 8, seed=7, amp=0.2)
    o.init_fields(s["rho"], s["ux"], s["uy"], s["uz"], s["p"])
    Q0 = o.moments().reshape(NF, -1).sum(1)
    o.step(50)
    assert np.isfinite(o.moments()).all()
    _, chi, _ = o.sensor()
    assert (chi > 0).any(), "sensor never active: conservation not exercised with blending"
    Q1 = o.moments().reshape(NF, -1).sum(1)
    scale = np.abs(o.moments()[:5]).reshape(5, -1).sum(1)
    assert np.all(np.abs(Q1[:5] - Q0[:5]) <= 1e-13 * scale)
    # stress and heat flux are not conserved: their relaxation must show
    assert np.abs(Q1[5:] - Q0[5:]).max() > 0


@pytest.mark.parametrize("u", [(0.0, 0.0, 0.0), (0.3, -0.2, 0.1)])
def test_uniform_state_is_fixed_point(oracle_mod, u):
    p = _tgv_like(6, 5, 4, f_mu=0.7)
    o = make_oracle(p)
    shape = (4, 5, 6)
    o.init_fields(np.full(shape, 1.1), np.full(shape, u[0]), np.full(shape, u[1]),
                  np.full(shape, u[2]), np.full(shape, 0.9))
    f0 = o.populations()
    o.step(20)
    f1 = o.populations()
    assert np.allclose(f1, f0, rtol=0, atol=1e-14 * np.abs(f0).max())
    th, chi, _ = o.sensor()
    assert np.abs(th).max() < 1e-9 and (chi == 0).all()


@pytest.mark.parametrize("shape,n", [((5, 4, 3), 1), ((5, 4, 3), 7), ((1, 3, 2), 4), ((8, 1, 1), 9)])
def test_streaming_is_exact_permutation(oracle_mod, shape, n):
    """With the collision switched off, n steps move population i of every field
    by n lattice vectors e_i with periodic wrap, and nothing else."""
    nx, ny, nz = shape
    p = _tgv_like(nx, ny, nz, collide=0)
    o = make_oracle(p)
    f0 = inputs.random_labels((NF, NQ, nz, ny, nx), seed=11, dtype=np.float64)
    o.set_populations(f0)
    o.step(n)
    f1 = o.populations()
    _, e = oracle_mod.lattice()
    expect = np.empty_like(f0)
    for i in range(NQ):
        expect[:, i] = np.roll(f0[:, i], shift=(n * e[i, 2], n * e[i, 1], n * e[i, 0]),
                               axis=(1, 2, 3))
    assert np.array_equal(f1, expect)


def test_axis_symmetry(oracle_mod):
    """The same plane wave along x, y or z gives the same solution up to the
    permutation of axes (and of the velocity/stress/heat-flux components)."""
    n = 16
    res = []
    for axis in range(3):
        shape = [1, 1, 1]
        shape[2 - axis] = n
        nz, ny, nx = shape
        p = _tgv_like(nx, ny, nz, f_mu=0.2, C_sigma=40.0, J_min=1e-3)
        p["dx"] = 2 * math.pi / n
        o = make_oracle(p)
        x = np.arange(n) * p["dx"]
        prof = lambda a: a.reshape(shape)
        u = [np.zeros(shape) for _ in range(3)]
        u[axis] = prof(0.3 * np.sin(x))
        u[(axis + 1) % 3] = prof(0.2 * np.cos(x))
        o.init_fields(prof(1 + 0.2 * np.cos(x)), u[0], u[1], u[2], prof(1 + 0.1 * np.sin(2 * x)))
        o.step(30)
        Q = o.moments().reshape(NF, n)
        # map to axis-0 convention: component a -> (a - axis) mod 3
        perm = [(a + axis) % 3 for a in range(3)]
        m = Q[1:4][perm]
        t = np.zeros((3, 3, n))
        pairs = [(0, 0), (1, 1), (2, 2), (0, 1), (0, 2), (1, 2)]
        for s, (b, c) in enumerate(pairs):
            t[b, c] = t[c, b] = Q[5 + s]
        tt = t[np.ix_(perm, perm)]
        res.append(np.concatenate([Q[[0, 4]], m, tt.reshape(9, n), Q[11:14][perm]]))
    assert np.allclose(res[1], res[0], rtol=1e-11, atol=1e-14)
    assert np.allclose(res[2], res[0], rtol=1e-11, atol=1e-14)


def test_held_ends_keep_uniform_state(oracle_mod):
    """A uniform state with x ends held at itself stays uniform."""
    p = inputs.sod_params(12, ny=2, nz=1)
    o = make_oracle(p)
    o.init_riemann(0, 6, (0.7, 0.1, 0.6), (0.7, 0.1, 0.6))
    f0 = o.populations()
    o.step(15)
    assert np.allclose(o.populations(), f0, rtol=0, atol=1e-14)


def test_riemann_mirror_symmetry(oracle_mod):
    """Reflecting the Sod problem (x -> -x, u -> -u) reflects the solution."""
    n = 64
    a = make_oracle(inputs.sod_params(n, ny=1, nz=1))
    a.init_riemann(0, n // 2, inputs.SOD_LEFT, inputs.SOD_RIGHT)
    b = make_oracle(inputs.sod_params(n, ny=1, nz=1))
    b.init_riemann(0, n // 2, inputs.SOD_RIGHT, inputs.SOD_LEFT)
    a.step(40)
    b.step(40)
    Pa = a.primitives()[:, 0, 0, :]
    Pb = b.primitives()[:, 0, 0, ::-1]
    Pb[1] = -Pb[1]
    assert np.allclose(Pa, Pb, rtol=1e-12, atol=1e-13)


def test_tgv_initial_diagnostics(oracle_mod):
    """At t = 0 the TGV field (Sec. 3.2) is solenoidal: central-difference div u is
    zero; <|curl u|^2> = 3/4 U0^2 up to the O(dx^2) error of central differences
    (exactly 3/4 (sin dx / dx)^2 for this field); T is uniform so mu_local = mu;
    <rho |u|^2 / 2> equals the grid average of the analytic field."""
    n = 16
    p = inputs.tgv_params(n)
    o = make_oracle(p)
    o.init_tgv(1.0, 1.25, 1.0)
    d = o.diag()
    h = p["dx"]
    assert abs(d["eps_d_raw"]) < 1e-25
    assert d["eps_s_raw"] == pytest.approx(p["mu"] * 0.75 * (math.sin(h) / h) ** 2, rel=1e-12)
    X = np.arange(n) * h
    Z, Y, Xg = np.meshgrid(X, X, X, indexing="ij")
    u = np.sin(Xg) * np.cos(Y) * np.cos(Z)
    v = -np.cos(Xg) * np.sin(Y) * np.cos(Z)
    p0 = 1.0 / (1.4 * 1.25 ** 2)
    pr = p0 + (np.cos(2 * Xg) + np.cos(2 * Y)) * (np.cos(2 * Z) + 2) / 16
    rho = pr / p0
    assert d["ek_mean"] == pytest.approx(np.mean(0.5 * rho * (u * u + v * v)), rel=1e-13)
    assert d["sum_rho"] == pytest.approx(rho.sum(), rel=1e-13)
    assert d["min_T"] == pytest.approx(p0, rel=1e-12)
    assert d["nonfinite"] == 0


def _sutherland_printed(T, T_ref, mu):
    """Sutherland's law in the form printed with the TGV setup (Sec. 3.2):
    mu (T/T_ref)^{3/2} (T_ref + S) / (T + S) with S = 0.4042 T_ref."""
    S = 0.4042 * T_ref
    return mu * (T / T_ref) ** 1.5 * (T_ref + S) / (T + S)


@pytest.mark.parametrize("sutherland,dT,component,T_axis", [
    (0, 0.0, 0, 1),    # constant viscosity, uniform T, compressive wave u_x(x)
    (1, 0.0, 0, 1),    # Sutherland at a uniform T != T_ref
    (1, 0.35, 0, 1),   # Sutherland with T varying along y, compressive wave
    (1, 0.35, 1, 2),   # shear wave u_y(x), T varying along z
    (1, 0.35, 2, 1),   # shear wave u_z(x), T varying along y
])
def test_wave_diagnostics_closed_forms(oracle_mod, sutherland, dT, component, T_axis):
    """Eq. 7 and the extrema of the diagnostics on a field whose velocity is one wave
    u_c = A sin(k x) and whose temperature depends only on y or z. The central
    difference of sin(k x) is cos(k x) sin(k dx)/dx and the grid mean of cos^2 is 1/2,
    so with mu_local averaged over the temperature profile (mbar):
      compressive (c = x): 4/3 <mu_local (div u)^2> = 2/3 mbar A^2 (sin(k dx)/dx)^2, no curl;
      shear (c = y, z):    <mu_local |curl u|^2>   = 1/2 mbar A^2 (sin(k dx)/dx)^2, no div;
    max Mach = A / sqrt(gamma T_min); max CFL = (A + sqrt(gamma T_max)) dt/dx (|u_c| and
    T peak in different coordinates, so both maxima meet in one cell);
    <rho |u|^2 / 2> = rho0 A^2 / 4. A dropped or doubled 4/3, mu_local applied twice
    (mu = 0.037, so mu^2 != mu), the square of the mean in place of the mean of the
    square, swapped dissipation channels, a missing gamma or a missing sound speed all
    fail here."""
    nx, ny, nz, k, A, rho0, T0, mu, T_ref = 16, 6, 5, 2, 0.3, 1.3, 0.9, 0.037, 0.8
    p = _tgv_like(nx, ny, nz, mu=mu, sutherland=sutherland, T_ref=T_ref)
    o = make_oracle(p)
    f = inputs.separable_wave_fields(nx, ny, nz, A, k, rho0, T0, dT, component, T_axis)
    o.init_fields(f["rho"], f["ux"], f["uy"], f["uz"], f["p"])
    d = o.diag()
    h = p["dx"]
    g2 = (math.sin(k * h) / h) ** 2
    T_line = f["T_line"]
    mbar = float(np.mean(_sutherland_printed(T_line, T_ref, mu))) if sutherland else mu
    n = nx * ny * nz
    if component == 0:
        assert d["eps_d_raw"] == pytest.approx(2.0 / 3.0 * mbar * A * A * g2, rel=1e-12)
        assert abs(d["eps_s_raw"]) < 1e-20
    else:
        assert d["eps_s_raw"] == pytest.approx(0.5 * mbar * A * A * g2, rel=1e-12)
        assert abs(d["eps_d_raw"]) < 1e-20
    gamma = p["gamma"]
    assert d["max_mach"] == pytest.approx(A / math.sqrt(gamma * T_line.min()), rel=1e-12)
    assert d["max_cfl"] == pytest.approx((A + math.sqrt(gamma * T_line.max())) * o.dt / h,
                                         rel=1e-12)
    assert d["ek_mean"] == pytest.approx(rho0 * A * A / 4.0, rel=1e-12)
    assert d["min_T"] == pytest.approx(T_line.min(), rel=1e-12)
    assert d["min_rho"] == pytest.approx(rho0, rel=1e-14)
    assert d["sum_rho"] == pytest.approx(rho0 * n, rel=1e-14)
    E_mean = rho0 * float(np.mean(T_line)) / (gamma - 1.0) + rho0 * A * A / 4.0
    assert d["sum_E"] == pytest.approx(E_mean * n, rel=1e-13)
    for key in ("sum_mx", "sum_my", "sum_mz"):
        assert abs(d[key]) < 1e-12
    assert d["nonfinite"] == 0


@pytest.mark.parametrize("nx", [16, 2])
def test_held_ends_one_sided_differences(oracle_mod, nx):
    """With held x ends the x derivative is one-sided at the two end cells. A linear
    velocity u_x = A x is differentiated exactly by both the central and the one-sided
    differences, so div u = A in every cell and 4/3 <mu (div u)^2> = 4/3 mu A^2 (constant
    viscosity), with no curl. A one-sided difference divided by 2 dx (or 0) at an end
    cell, or a wrapped (periodic) neighbour there, breaks it; nx = 2 has only end
    cells."""
    ny, nz, A, rho0, T0, mu = 3, 2, 0.05, 1.1, 0.8, 0.021
    p = inputs.sod_params(nx, ny=ny, nz=nz)
    p.update(mu=mu, sutherland=0)
    o = make_oracle(p)
    x = (np.arange(nx) + 0.5) / nx
    shape = (nz, ny, nx)
    ux = np.broadcast_to(A * x, shape)
    o.init_fields(np.full(shape, rho0), ux, 0.0, 0.0, np.full(shape, rho0 * T0))
    d = o.diag()
    assert d["eps_d_raw"] == pytest.approx(4.0 / 3.0 * mu * A * A, rel=1e-12)
    assert abs(d["eps_s_raw"]) < 1e-25
