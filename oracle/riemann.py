"""Exact solution of the Riemann problem of the 1-D Euler equations (ideal gas).

TEST INFRASTRUCTURE (oracle): the Sod tube of Sec. 3.1 is scored against this
solution. Written from the textbook construction: the star pressure p* is the
root of f_L(p) + f_R(p) + u_R - u_L = 0, where f_K is the velocity jump across a
shock (Rankine-Hugoniot) or a rarefaction (isentropic, Riemann invariant) wave
connecting state K to pressure p; the solution is self-similar in xi = x / t.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np


@dataclass(frozen=True)
class State:
    rho: float
    u: float
    p: float


def _sound(g, s: State) -> float:
    return math.sqrt(g * s.p / s.rho)


def _f_and_df(g: float, p: float, s: State):
    """Velocity change across the wave from s to pressure p, and d/dp."""
    a = _sound(g, s)
    if p > s.p:  # shock
        A = 2.0 / ((g + 1.0) * s.rho)
        B = (g - 1.0) / (g + 1.0) * s.p
        q = math.sqrt(A / (p + B))
        return (p - s.p) * q, q * (1.0 - 0.5 * (p - s.p) / (p + B))
    # rarefaction
    e = (g - 1.0) / (2.0 * g)
    r = (p / s.p) ** e
    return 2.0 * a / (g - 1.0) * (r - 1.0), (p / s.p) ** (-(g + 1.0) / (2.0 * g)) / (s.rho * a)


@dataclass(frozen=True)
class Star:
    p: float
    u: float
    rho_L: float
    rho_R: float
    left_shock: bool
    right_shock: bool
    # wave speeds: left wave (head, tail), right wave (tail, head); equal for shocks
    sL_head: float
    sL_tail: float
    sR_tail: float
    sR_head: float


def solve_star(L: State, R: State, gamma: float = 1.4, tol: float = 1e-14) -> Star:
    g = gamma
    aL, aR = _sound(g, L), _sound(g, R)
    if 2.0 * (aL + aR) / (g - 1.0) <= R.u - L.u:
        raise ValueError("vacuum is generated; no star state")
    # two-rarefaction guess, then Newton on f_L + f_R + du = 0
    e = (g - 1.0) / (2.0 * g)
    p = ((aL + aR - 0.5 * (g - 1.0) * (R.u - L.u)) / (aL / L.p ** e + aR / R.p ** e)) ** (1.0 / e)
    p = max(p, 1e-12)
    for _ in range(100):
        fL, dL = _f_and_df(g, p, L)
        fR, dR = _f_and_df(g, p, R)
        p_new = p - (fL + fR + R.u - L.u) / (dL + dR)
        p_new = max(p_new, 1e-14)
        if abs(p_new - p) <= tol * 0.5 * (p_new + p):
            p = p_new
            break
        p = p_new
    fL, _ = _f_and_df(g, p, L)
    fR, _ = _f_and_df(g, p, R)
    u = 0.5 * (L.u + R.u) + 0.5 * (fR - fL)
    gm = (g - 1.0) / (g + 1.0)

    def rho_star(s: State):
        if p > s.p:
            r = p / s.p
            return s.rho * (r + gm) / (gm * r + 1.0), True
        return s.rho * (p / s.p) ** (1.0 / g), False

    rL, shL = rho_star(L)
    rR, shR = rho_star(R)
    if shL:
        sL = L.u - aL * math.sqrt((g + 1.0) / (2.0 * g) * p / L.p + (g - 1.0) / (2.0 * g))
        sLh = sLt = sL
    else:
        sLh = L.u - aL
        sLt = u - math.sqrt(g * p / rL)
    if shR:
        sR = R.u + aR * math.sqrt((g + 1.0) / (2.0 * g) * p / R.p + (g - 1.0) / (2.0 * g))
        sRh = sRt = sR
    else:
        sRh = R.u + aR
        sRt = u + math.sqrt(g * p / rR)
    return Star(p, u, rL, rR, shL, shR, sLh, sLt, sRt, sRh)


def sample(L: State, R: State, xi, gamma: float = 1.4):
    """rho, u, p at similarity coordinates xi = (x - x0) / t (array)."""
    g = gamma
    st = solve_star(L, R, g)
    xi = np.asarray(xi, dtype=np.float64)
    rho = np.empty_like(xi)
    u = np.empty_like(xi)
    p = np.empty_like(xi)
    aL, aR = _sound(g, L), _sound(g, R)
    for j, s in np.ndenumerate(xi):
        if s <= st.u:  # left of the contact
            if s <= st.sL_head:
                v = (L.rho, L.u, L.p)
            elif s >= st.sL_tail:
                v = (st.rho_L, st.u, st.p)
            else:  # inside the left fan
                uu = 2.0 / (g + 1.0) * (aL + 0.5 * (g - 1.0) * L.u + s)
                a = 2.0 / (g + 1.0) * (aL + 0.5 * (g - 1.0) * (L.u - s))
                v = (L.rho * (a / aL) ** (2.0 / (g - 1.0)), uu,
                     L.p * (a / aL) ** (2.0 * g / (g - 1.0)))
        else:
            if s >= st.sR_head:
                v = (R.rho, R.u, R.p)
            elif s <= st.sR_tail:
                v = (st.rho_R, st.u, st.p)
            else:  # inside the right fan
                uu = 2.0 / (g + 1.0) * (-aR + 0.5 * (g - 1.0) * R.u + s)
                a = 2.0 / (g + 1.0) * (aR - 0.5 * (g - 1.0) * (R.u - s))
                v = (R.rho * (a / aR) ** (2.0 / (g - 1.0)), uu,
                     R.p * (a / aR) ** (2.0 * g / (g - 1.0)))
        rho[j], u[j], p[j] = v
    return rho, u, p


def max_signal_speed(L: State, R: State, gamma: float = 1.4) -> float:
    """Largest |u| + a over the whole self-similar solution. Inside a fan |u| + a
    is monotone in xi, so the constant states bound it."""
    g = gamma
    st = solve_star(L, R, g)
    cands = [abs(L.u) + _sound(g, L), abs(R.u) + _sound(g, R),
             abs(st.u) + math.sqrt(g * st.p / st.rho_L),
             abs(st.u) + math.sqrt(g * st.p / st.rho_R)]
    return max(cands)


def shock_position(L: State, R: State, t: float, x0: float, gamma: float = 1.4) -> float:
    """Position of the right-moving shock at time t (raises if the right wave is a fan)."""
    st = solve_star(L, R, gamma)
    if not st.right_shock:
        raise ValueError("right wave is a rarefaction")
    return x0 + st.sR_head * t
