"""The oracle against closed forms and exact solutions:
  * local dilatation recovery (Sec. 2.3) converging to the analytic div u;
  * shear and acoustic waves against the linearised relaxed system (Eq. 2);
  * the numerical viscosity of Eq. 6 (nu_num = f_mu mu / rho on D3Q7);
  * Sod against the exact Riemann solution (Sec. 3.1, Tables 2 and 4).
"""
import json
import math
import os

import numpy as np
import pytest

from conftest import make_oracle
from oracle import linear_modes as lm
from oracle import riemann
from paper_2608_13437_gb300 import inputs

NF, NQ = 14, 7
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _wave_oracle(n, **kw):
    p = dict(nx=n, ny=1, nz=1, dx=1.0 / n, dt=0.05 / n, gamma=1.4, mu=0.01, kappa=0.01,
             tau_R=0.01, tau_q=0.01, T_ref=1.0, sutherland=0, f_mu=0.0, C_sigma=0.0,
             J_min=0.0, omega_min=1.0)
    p.update(kw)
    return make_oracle(p)


# --------------------------------------------------------------------------- dilatation
def test_dilatation_recovery_converges(oracle_mod):
    """One step from equilibrium leaves fneq = -dt D feq (an effective relaxation
    time of 1), so with tau_base = 1/2 (f_mu = 0) the recovered theta is twice
    div u up to O(dx). Fields vary in x and y, with u . grad rho != 0, so the
    density-gradient part of the formula is exercised."""
    errs = []
    for n in (16, 32, 64):
        dx = 1.0 / n
        o = make_oracle(dict(nx=n, ny=n, nz=1, dx=dx, dt=0.1 * dx, mu=1e-3, kappa=1e-3,
                             tau_R=1e-2, tau_q=1e-2, f_mu=0.0, C_sigma=0.0))
        x = (np.arange(n) * dx)[None, None, :]
        y = (np.arange(n) * dx)[None, :, None]
        k = 2 * np.pi
        rho = 1 + 0.2 * np.sin(k * x) * np.ones_like(y)
        ux = 0.1 * np.sin(k * (x + y))
        uy = 0.1 * np.cos(k * y) * np.ones_like(x)
        o.init_fields(rho, ux, uy, np.zeros_like(rho), np.ones_like(rho))
        o.step(1)
        th, _, _ = o.sensor()
        div = 0.1 * k * np.cos(k * (x + y)) - 0.1 * k * np.sin(k * y)
        errs.append(np.abs(0.5 * th - div).max() / np.abs(div).max())
    assert errs[-1] < 0.2
    for a, b in zip(errs, errs[1:]):
        assert 1.8 < a / b < 2.2, errs  # first order
    # without the u . grad rho term the error stalls (the density part matters)
    o = make_oracle(dict(nx=64, ny=64, nz=1, dx=1 / 64, dt=0.1 / 64, mu=1e-3, kappa=1e-3,
                         tau_R=1e-2, tau_q=1e-2, f_mu=0.0, C_sigma=0.0, sensor_mode=1))
    o.init_fields(rho, ux, uy, np.zeros_like(rho), np.ones_like(rho))
    o.step(1)
    th, _, _ = o.sensor()
    assert np.abs(0.5 * th - div).max() / np.abs(div).max() > 1.1 * errs[-1]


def test_compression_has_negative_dilatation(oracle_mod):
    """A converging flow u_x = -U sin(2 pi x) around x = 0 compresses: theta < 0 and
    the sensor fires there; it stays off where the flow expands."""
    n = 64
    o = _wave_oracle(n, C_sigma=20.0, J_min=1e-4)
    x = np.arange(n) / n
    o.init_fields(np.ones((1, 1, n)), (-0.05 * np.sin(2 * np.pi * x))[None, None],
                  np.zeros((1, 1, n)), np.zeros((1, 1, n)), np.ones((1, 1, n)))
    o.step(1)
    th, chi, _ = o.sensor()
    th, chi = th[0, 0], chi[0, 0]
    assert th[0] < 0 and chi[0] > 0
    assert th[n // 2] > 0 and chi[n // 2] == 0


# --------------------------------------------------------------------------- linear waves
def _amp(field):
    return lm.fourier_amplitude(field[0, 0], 1)


@pytest.mark.parametrize("source_mode", [0, 1])
def test_shear_wave_matches_linear_theory(oracle_mod, source_mode):
    """u_y = A sin(2 pi x) decays as the 2x2 relaxed system predicts. With the
    explicit source (default) the amplitude error falls at second order under
    refinement at fixed physical tau_R; the exact-exponential source biases the
    relaxed stress by (dt/tau_R) / (1 - exp(-dt/tau_R)) and converges at first order."""
    t_end = 1.0
    errs = []
    for n in (32, 64, 128):
        o = _wave_oracle(n, source_mode=source_mode)
        x = np.arange(n) / n
        A = 1e-3
        z = np.zeros((1, 1, n))
        o.init_fields(np.ones((1, 1, n)), z, (A * np.sin(2 * np.pi * x))[None, None], z,
                      np.ones((1, 1, n)))
        Q0 = o.moments()
        v0 = [_amp(Q0[2]), _amp(Q0[8])]
        steps = int(round(t_end / o.dt))
        o.step(steps)
        Q = o.moments()
        v = np.array([_amp(Q[2]), _amp(Q[8])])
        M = lm.shear_matrix(2 * np.pi, 1.0, 0.01, 0.01)
        ve = lm.evolve(M, v0, steps * o.dt)
        errs.append(abs(v[0] - ve[0]) / abs(v0[0]))
    decay = abs(ve[0]) / abs(v0[0])
    assert decay < 0.75  # the test sees real decay
    order = 2.0 if source_mode == 0 else 1.0
    assert errs[-1] < (5e-4 if source_mode == 0 else 1e-2), errs
    assert errs[0] / errs[1] > 0.85 * 2 ** order and errs[1] / errs[2] > 0.85 * 2 ** order, errs


@pytest.mark.parametrize("sutherland", [False, True])
def test_acoustic_wave_matches_linear_theory(oracle_mod, sutherland):
    """An isentropic density pulse cos(2 pi x) evolves as exp(M t) of the 5x5
    linearised system (rho, rho u_x, E, tau_xx, q_x). Under Sutherland's law the
    heat-flux flux kappa_T T / tau_q linearises to (kappa_T + T kappa_T') T'."""
    t_end = 1.0
    errs = []
    T_ref = 0.7 if sutherland else 1.0
    for n in (32, 64, 128):
        o = _wave_oracle(n, sutherland=int(sutherland), T_ref=T_ref, mu=0.02, kappa=0.03)
        x = np.arange(n) / n
        eps = 1e-5
        rho = 1 + eps * np.cos(2 * np.pi * x)
        p = 1 + 1.4 * eps * np.cos(2 * np.pi * x)
        z = np.zeros((1, 1, n))
        o.init_fields(rho[None, None], z, z, z, p[None, None])
        Q0 = o.moments()
        idx = [0, 1, 4, 5, 11]
        v0 = [_amp(Q0[k]) for k in idx]
        steps = int(round(t_end / o.dt))
        o.step(steps)
        Q = o.moments()
        v = np.array([_amp(Q[k]) for k in idx])
        M = lm.acoustic_matrix(2 * np.pi, 1.0, 1.0, 1.4, 0.02, 0.03, 0.01, 0.01,
                               sutherland=sutherland, T_ref=T_ref)
        ve = lm.evolve(M, v0, steps * o.dt)
        errs.append(np.abs(v[:3] - ve[:3]).max() / abs(v0[0]))
    # Below N = 128 the error falls with the mesh; from there on an O(dt) part
    # oscillating in time at the 1e-4 level remains (it shrinks with dt at fixed
    # N). The conductivity linearised as kappa_T alone (Fourier form) misses by
    # 5e-2 and a constant conductivity by 1.7e-1, so 2e-3 separates them.
    assert errs[-1] < 2e-3, errs
    assert errs[0] > 3 * errs[-1], errs


def test_linear_system_small_k_limits():
    """The linearised matrices reproduce the textbook small-k limits: shear
    s = -nu k^2, sound s = +-i a k - Gamma k^2 with Gamma = ((4/3) mu + (gamma-1) K
    / c_p) / (2 rho), entropy mode s = -K k^2 / (rho c_p)."""
    rho, T0, g, mu, kap, tR, tq = 1.3, 0.9, 1.4, 0.02, 0.05, 1e-6, 1e-6
    k = 1e-2
    s = np.linalg.eigvals(lm.shear_matrix(k, rho, mu, tR))
    slow = s[np.argmin(abs(s))]
    assert slow.real == pytest.approx(-mu / rho * k * k, rel=1e-6)
    ev = np.linalg.eigvals(lm.acoustic_matrix(k, rho, T0, g, mu, kap, tR, tq))
    ev = ev[np.abs(ev) < 1.0]  # drop the two fast relaxation modes
    cp = g / (g - 1)
    a = math.sqrt(g * T0)
    gam = ((4 / 3) * mu + (g - 1) * kap / cp) / (2 * rho)
    sound = ev[np.abs(ev.imag) > 0.5 * a * k]
    ent = ev[np.abs(ev.imag) <= 0.5 * a * k]
    assert len(sound) == 2 and len(ent) == 1
    assert np.allclose(np.sort(np.abs(sound.imag)), [a * k, a * k], rtol=1e-6)
    assert np.allclose(sound.real, -gam * k * k, rtol=1e-4)
    assert ent.real == pytest.approx(-kap / (rho * cp) * k * k, rel=1e-4)


def test_numerical_viscosity_of_baseline_rate(oracle_mod):
    """Eq. 6: on D3Q7, tau_base = 1/2 + 4 f_mu (mu/rho) dt/dx^2 adds nu_num = f_mu mu/rho.
    A stress component tau_yz(x) with u = 0 has no physical flux divergence and, with
    the relaxation switched off (tau_R huge), only diffuses with nu_num."""
    f_mu, mu = 2.0, 0.005
    rates = []
    k = 2 * np.pi
    for n in (16, 32, 64):
        o = _wave_oracle(n, mu=mu, f_mu=f_mu, tau_R=1e30, tau_q=1e30)
        x = np.arange(n) / n
        f = np.empty((NF, NQ, 1, 1, n))
        for j in range(n):
            Q = np.zeros(NF)
            Q[0], Q[4] = 1.0, 2.5
            Q[10] = 1e-3 * np.sin(k * x[j])
            f[:, :, 0, 0, j] = o.equilibrium_of(Q)
        o.set_populations(f)
        c0 = _amp(o.moments()[10])
        steps = int(round(0.5 / o.dt))
        o.step(steps)
        c1 = _amp(o.moments()[10])
        rates.append(-math.log(abs(c1) / abs(c0)) / (steps * o.dt))
    nu = f_mu * mu / 1.0
    errs = [abs(r / (nu * k * k) - 1) for r in rates]
    assert errs[-1] < 5e-3, (rates, nu * k * k)
    assert errs[0] > errs[1] > errs[2]


# --------------------------------------------------------------------------- Riemann
def test_exact_riemann_solver_invariants():
    """Sod star state satisfies the Rankine-Hugoniot jump conditions across the right
    shock, isentropy and the Riemann invariant across the left fan, continuity of
    u and p across the contact; and it matches the textbook star values
    (Toro, Riemann Solvers and Numerical Methods for Fluid Dynamics, Test 1)."""
    g = 1.4
    L = riemann.State(*inputs.SOD_LEFT)
    R = riemann.State(*inputs.SOD_RIGHT)
    st = riemann.solve_star(L, R, g)
    S = st.sR_head
    assert st.right_shock and not st.left_shock

    def fluxes(rho, u, p):
        E = p / (g - 1) + 0.5 * rho * u * u
        return np.array([rho * (u - S), rho * u * (u - S) + p, E * (u - S) + p * u])

    assert np.allclose(fluxes(R.rho, R.u, R.p), fluxes(st.rho_R, st.u, st.p), rtol=1e-12)
    assert st.p / st.rho_L ** g == pytest.approx(L.p / L.rho ** g, rel=1e-12)
    aL = math.sqrt(g * L.p / L.rho)
    aS = math.sqrt(g * st.p / st.rho_L)
    assert st.u + 2 * aS / (g - 1) == pytest.approx(L.u + 2 * aL / (g - 1), rel=1e-12)
    assert (st.p, st.u, st.rho_L, st.rho_R) == pytest.approx(
        (0.30313, 0.92745, 0.42632, 0.26557), abs=1e-5)
    # sampled profile is continuous through the fan and constant in the star regions
    xi = np.linspace(-2, 2, 4001)
    rho, u, p = riemann.sample(L, R, xi, g)
    fan = (xi > st.sL_head) & (xi < st.sL_tail)
    assert np.all(np.diff(rho[fan]) < 0) and np.all(np.diff(u[fan]) > 0)
    assert riemann.max_signal_speed(L, R) == pytest.approx(inputs.SOD_LAMBDA_MAX, rel=1e-12)


def _sod_run(n):
    o = make_oracle(inputs.sod_params(n, ny=1, nz=1))
    o.init_riemann(0, n // 2, inputs.SOD_LEFT, inputs.SOD_RIGHT)
    steps = inputs.sod_steps(o.dt)
    o.step(steps)
    t = steps * o.dt
    P = o.primitives()[:, 0, 0, :]
    x = (np.arange(n) + 0.5) / n
    return x, t, P


def _shock_metrics(x, t, rho):
    L = riemann.State(*inputs.SOD_LEFT)
    R = riemann.State(*inputs.SOD_RIGHT)
    st = riemann.solve_star(L, R)
    right = x[:-1] > 0.5 + st.u * t + 0.05
    slope = np.abs(np.diff(rho)) / (x[1] - x[0])
    w = (st.rho_R - R.rho) / slope[right].max()
    mid = 0.5 * (st.rho_R + R.rho)
    i = np.where(right & (rho[:-1] >= mid) & (rho[1:] < mid))[0][-1]
    xs = x[i] + (rho[i] - mid) / (rho[i] - rho[i + 1]) * (x[1] - x[0])
    return w, xs, riemann.shock_position(L, R, t, 0.5)


def test_sod_against_exact_solution(oracle_mod):
    """Shock within 1e-3 of its exact position, L1(rho) falling with the mesh, shock
    thickness proportional to dx (first order, Table 2), and the thickness in
    cells of the same order as the paper's w/dx of 4.75-4.92 (Table 2)."""
    with open(os.path.join(GOLDEN, "paper_tables.json")) as fh:
        paper = json.load(fh)
    L = riemann.State(*inputs.SOD_LEFT)
    R = riemann.State(*inputs.SOD_RIGHT)
    res = {}
    for n in (256, 512):
        x, t, P = _sod_run(n)
        assert np.isfinite(P).all()
        re, ue, pe = riemann.sample(L, R, (x - 0.5) / t)
        w, xs, xe = _shock_metrics(x, t, P[0])
        res[n] = dict(l1=np.mean(np.abs(P[0] - re)), w=w, xs=xs, xe=xe)
    assert abs(res[512]["xs"] - res[512]["xe"]) < 1e-3
    assert res[512]["l1"] < 0.75 * res[256]["l1"]
    ratio = res[256]["w"] / res[512]["w"]
    assert 1.6 < ratio < 2.5
    paper_wdx = [r["w_over_dx"] for r in paper["thickness_sod"]]
    for n in (256, 512):
        wdx = res[n]["w"] * n
        assert 0.5 * min(paper_wdx) < wdx < 2.0 * max(paper_wdx)
