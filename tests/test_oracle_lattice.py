"""Pins of the oracle's per-cell pieces against what the paper and mathematics fix.

Each check would fail under a plausible mistake: a wrong weight, a dropped flux
term, a transposed stress index, a sign flip, a wrong Lambda coefficient.
"""
import numpy as np
import pytest

from conftest import make_oracle

NF, NQ = 14, 7


def _domain(oracle_mod, **kw):
    p = dict(nx=4, ny=4, nz=4, dx=0.1, dt=0.01, gamma=1.4, mu=0.02, kappa=0.03,
              tau_R=0.05, tau_q=0.07, T_ref=0.8, sutherland=1, f_mu=0.3, C_sigma=20.0,
              J_min=3e-3, omega_min=1.0)
    p.update(kw)
    return make_oracle(p)


def _random_state(rng):
    Q = np.zeros(NF)
    rho = 0.5 + rng.random()
    u = rng.standard_normal(3) * 0.5
    p = 0.3 + rng.random()
    Q[0] = rho
    Q[1:4] = rho * u
    Q[4] = p / 0.4 + 0.5 * rho * u @ u
    Q[5:] = rng.standard_normal(9) * 0.1
    return Q


def test_d3q7_weights_and_moments(oracle_mod):
    w, e = oracle_mod.lattice()
    assert w.sum() == pytest.approx(1.0, abs=1e-15)
    # isotropy: first and third moments vanish, second = c_s^2 delta with c_s^2 = 1/4 (Sec. 2.2)
    assert np.allclose((w[:, None] * e).sum(0), 0.0)
    second = np.einsum("i,ia,ib->ab", w, e, e)
    assert np.allclose(second, 0.25 * np.eye(3), atol=1e-15)
    assert np.allclose(np.einsum("i,ia,ib,ic->abc", w, e, e, e), 0.0)
    # one rest and six unit vectors along the axes, in +/- pairs
    assert (np.abs(e).sum(1) == np.array([0, 1, 1, 1, 1, 1, 1])).all()
    assert (e[1::2] == -e[2::2]).all()


def test_equilibrium_moments(oracle_mod):
    """Zeroth moment of feq is Q, first moment is the flux (Sec. 2.2), second is c_s^2 Q I."""
    d = _domain(oracle_mod)
    w, e = oracle_mod.lattice()
    c = d.params["dx"] / d.dt
    rng = np.random.default_rng(1)
    for _ in range(5):
        Q = _random_state(rng)
        feq = d.equilibrium_of(Q)
        Phi = d.flux_of(Q)
        assert np.allclose(feq.sum(1), Q, rtol=1e-13, atol=1e-14)
        assert np.allclose(feq @ (c * e), Phi, rtol=1e-12, atol=1e-13)
        m2 = np.einsum("ki,ia,ib->kab", feq, c * e, c * e)
        assert np.allclose(m2, 0.25 * c * c * Q[:, None, None] * np.eye(3), rtol=1e-12, atol=1e-12)


def test_flux_structure_of_eq2(oracle_mod):
    """Structural facts of Eq. 2 that do not restate it term by term: the mass flux
    is the momentum; the momentum flux is symmetric; at rest with zero stress and
    heat flux only the pressure (momentum) and kappa T / tau_q (heat flux) remain
    and both are isotropic; the energy flux at rest equals q."""
    d = _domain(oracle_mod, sutherland=0)
    rng = np.random.default_rng(2)
    Q = _random_state(rng)
    Phi = d.flux_of(Q)
    assert np.allclose(Phi[0], Q[1:4])
    assert np.allclose(Phi[1:4], Phi[1:4].T, rtol=1e-13)
    rest = Q.copy()
    rest[1:4] = 0
    rest[5:] = 0
    P = d.flux_of(rest)
    cl = d.closure_of(rest)
    assert np.allclose(P[1:4], cl["p"] * np.eye(3), rtol=1e-14)
    assert np.allclose(P[11:14], 0.03 / 0.07 * cl["T"] * np.eye(3), rtol=1e-14)
    assert np.allclose(P[[0, 4]], 0.0) and np.allclose(P[5:11], 0.0)
    rest[11:14] = [0.1, -0.2, 0.3]
    assert np.allclose(d.flux_of(rest)[4], [0.1, -0.2, 0.3], rtol=1e-14)


def test_stress_flux_divergence_is_deviatoric_strain(oracle_mod):
    """Sec. 2.1: div Lambda(u) reproduces grad u + grad u^T - 2/3 (div u) I.
    With a quadratic velocity field central differences are exact, so the
    discrete divergence of the oracle's stress flux must equal
    -(mu / tau_R) times the analytic deviatoric strain rate."""
    mu, tau_R = 0.02, 0.05
    d = _domain(oracle_mod, sutherland=0, mu=mu, tau_R=tau_R)
    rng = np.random.default_rng(3)
    A = rng.standard_normal(3)
    B = rng.standard_normal((3, 3))
    C = rng.standard_normal((3, 3, 3))

    def u_of(x):
        return A + B @ x + np.einsum("abc,b,c->a", C, x, x)

    def grad_u(x):  # G[a, b] = d_b u_a
        return B + np.einsum("abc,c->ab", C, x) + np.einsum("acb,c->ab", C, x)

    def state(x):
        u = u_of(x)
        Q = np.zeros(NF)
        Q[0] = 1.0
        Q[1:4] = u
        Q[4] = 1.0 / 0.4 + 0.5 * u @ u  # p = 1 everywhere: T uniform, mu_T constant
        return Q

    h = 1e-3
    x0 = rng.standard_normal(3) * 0.3
    div = np.zeros(6)
    for a in range(3):
        ea = np.zeros(3)
        ea[a] = h
        Pp = d.flux_of(state(x0 + ea))
        Pm = d.flux_of(state(x0 - ea))
        div += (Pp[5:11, a] - Pm[5:11, a]) / (2 * h)
    G = grad_u(x0)
    S = G + G.T - 2.0 / 3.0 * np.trace(G) * np.eye(3)
    pairs = [(0, 0), (1, 1), (2, 2), (0, 1), (0, 2), (1, 2)]
    expect = np.array([-(mu / tau_R) * S[b, c] for b, c in pairs])
    assert np.allclose(div, expect, rtol=1e-6, atol=1e-6)


def test_sutherland_law(oracle_mod):
    """Listing 1 and the form printed in Sec. 3.2 agree: mu(T) = 1.4042 (T/T0)^{3/2}
    / (T/T0 + 0.4042) mu; mu(T_ref) = mu; kappa_T / kappa = mu_T / mu."""
    T_ref = 0.8
    d = _domain(oracle_mod, T_ref=T_ref)
    for T in (0.3, 0.8, 1.7, 5.0):
        Q = np.zeros(NF)
        Q[0] = 1.3
        Q[4] = 1.3 * T / 0.4
        cl = d.closure_of(Q)
        assert cl["T"] == pytest.approx(T, rel=1e-14)
        t = T / T_ref
        assert cl["mu_T"] == pytest.approx(0.02 * 1.4042 * t ** 1.5 / (t + 0.4042), rel=1e-13)
        assert cl["kappa_T"] / 0.03 == pytest.approx(cl["mu_T"] / 0.02, rel=1e-13)
    Q = np.zeros(NF)
    Q[0] = 1.0
    Q[4] = T_ref / 0.4
    assert d.closure_of(Q)["mu_T"] == pytest.approx(0.02, rel=1e-14)


def test_closure_ideal_gas(oracle_mod):
    """Sec. 2.1: p = (gamma - 1)(E - rho |u|^2 / 2), T = p / rho."""
    d = _domain(oracle_mod)
    Q = np.zeros(NF)
    Q[0] = 2.0
    Q[1:4] = [2.0, -4.0, 6.0]          # u = (1, -2, 3), |u|^2 = 14
    Q[4] = 20.0                        # kinetic part 14
    cl = d.closure_of(Q)
    assert cl["p"] == pytest.approx(0.4 * 6.0, rel=1e-14)
    assert cl["T"] == pytest.approx(1.2, rel=1e-14)


def test_sensor_piecewise_response(oracle_mod):
    """Eq. 4 and Table 1: zero up to and at J_min (strict inequality), then C_sigma s,
    saturating at s = 1 / C_sigma."""
    d = _domain(oracle_mod, C_sigma=20.0, J_min=3e-3)
    assert d.chi_of(0.0) == 0.0
    assert d.chi_of(3e-3) == 0.0
    s = 3e-3 * (1 + 1e-9)
    assert d.chi_of(s) == pytest.approx(20.0 * s, rel=1e-12)
    assert d.chi_of(0.025) == pytest.approx(0.5, rel=1e-12)
    assert d.chi_of(1.0 / 20.0) == pytest.approx(1.0, abs=1e-15)
    assert d.chi_of(0.3) == 1.0


def test_single_collision_conserves_and_relaxes(oracle_mod):
    """Collision leaves rho, rho u, E unchanged (S = 0 there, Eq. 2), changes each
    stress/heat-flux moment by exactly its source increment dt S_k (Sec. 2.2), and
    at omega_h = 1 returns feq + w dt S. The exact-exponential switch changes the
    increment to (exp(-dt/tau) - 1) Q_k."""
    rng = np.random.default_rng(5)
    for om_min, f_mu, Cs in ((1.0, 0.3, 20.0), (1.0, 0.0, 1e6)):
        d = _domain(oracle_mod, f_mu=f_mu, C_sigma=Cs, J_min=0.0, omega_min=om_min)
        Q = _random_state(rng)
        f = d.equilibrium_of(Q) + rng.standard_normal((NF, NQ)) * 1e-3
        fo, tco = d.collide_of(f)
        Qin = f.sum(1)
        Qout = fo.sum(1)
        assert np.allclose(Qout[:5], Qin[:5], rtol=1e-14, atol=1e-14)
        dt = d.dt
        dec = np.r_[np.full(6, -dt / 0.05), np.full(3, -dt / 0.07)]
        assert np.allclose(Qout[5:], Qin[5:] * (1 + dec), rtol=1e-12, atol=1e-15)
        if tco[1] == 1.0:
            w, _ = oracle_mod.lattice()
            feq = d.equilibrium_of(Qin)
            dS = np.r_[np.zeros(5), Qin[5:] * dec]
            assert np.allclose(fo, feq + w[None, :] * dS[:, None], rtol=1e-12, atol=1e-14)
        d1 = _domain(oracle_mod, f_mu=f_mu, C_sigma=Cs, J_min=0.0, omega_min=om_min,
                     source_mode=1)
        Qo1 = d1.collide_of(f)[0].sum(1)
        dec1 = np.r_[np.full(6, np.expm1(-dt / 0.05)), np.full(3, np.expm1(-dt / 0.07))]
        assert np.allclose(Qo1[5:], Qin[5:] * (1 + dec1), rtol=1e-12, atol=1e-15)


def test_blend_between_baseline_and_floor(oracle_mod):
    """Eq. 5 and Eq. 6: omega_h = omega - chi (omega - omega_min), omega = 1/tau_base;
    chi = 0 gives the baseline rate, chi = 1 the floor. With f_mu = 0 the baseline
    relaxation time is 1/2 (omega = 2)."""
    d = _domain(oracle_mod, f_mu=0.0, C_sigma=0.0)
    Q = np.zeros(NF)
    Q[0], Q[4] = 1.0, 2.0
    f = d.equilibrium_of(Q)
    _, tco = d.collide_of(f)
    assert tco[1] == 0.0 and tco[2] == pytest.approx(2.0, rel=1e-15)
    d2 = _domain(oracle_mod, f_mu=0.0, C_sigma=1e9, J_min=0.0, omega_min=1.3)
    f2 = f.copy()
    f2[0, 0] -= 1e-3  # a compression in the rest population of rho
    _, tco2 = d2.collide_of(f2)
    assert tco2[0] < 0 and tco2[1] == 1.0 and tco2[2] == pytest.approx(1.3, rel=1e-14)
