"""Exact solution of the 1D Riemann problem for an ideal gas.

TEST INFRASTRUCTURE ONLY (part of the oracle).  The paper compares its shock
tube runs with exact solutions (Sec. 4(1), Figs. 6 and 7) without stating a
method; this is the classical exact solver (star-region pressure from the
shock / rarefaction wave curves, solved by Newton's method, then self-similar
sampling), written from the Rankine-Hugoniot and isentropic relations.
States are (rho, u, p); R = 1 so T = p / rho.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np


@dataclasses.dataclass
class Star:
    p: float
    u: float
    rho_l: float
    rho_r: float


def _wave_curve(p, rho_k, p_k, gamma):
    """Velocity jump across the left/right wave as a function of the star
    pressure p, and its derivative: shock branch for p > p_k (Rankine-Hugoniot),
    rarefaction branch otherwise (isentropic, Riemann invariant)."""
    a_k = math.sqrt(gamma * p_k / rho_k)
    if p > p_k:
        A = 2.0 / ((gamma + 1.0) * rho_k)
        B = (gamma - 1.0) / (gamma + 1.0) * p_k
        q = math.sqrt(A / (p + B))
        return (p - p_k) * q, q * (1.0 - 0.5 * (p - p_k) / (p + B))
    e = (gamma - 1.0) / (2.0 * gamma)
    r = p / p_k
    return 2.0 * a_k / (gamma - 1.0) * (r ** e - 1.0), (r ** (-(gamma + 1.0) / (2.0 * gamma))) / (rho_k * a_k)


def star_state(left, right, gamma: float = 1.4, tol: float = 1e-15) -> Star:
    rho_l, u_l, p_l = left
    rho_r, u_r, p_r = right
    a_l = math.sqrt(gamma * p_l / rho_l)
    a_r = math.sqrt(gamma * p_r / rho_r)
    if 2.0 * (a_l + a_r) / (gamma - 1.0) <= u_r - u_l:
        raise ValueError("vacuum is generated")
    # two-rarefaction estimate as the starting point
    e = (gamma - 1.0) / (2.0 * gamma)
    p = ((a_l + a_r - 0.5 * (gamma - 1.0) * (u_r - u_l)) / (a_l / p_l ** e + a_r / p_r ** e)) ** (1.0 / e)
    p = max(p, 1e-12 * min(p_l, p_r))
    for _ in range(200):
        fl, dl = _wave_curve(p, rho_l, p_l, gamma)
        fr, dr = _wave_curve(p, rho_r, p_r, gamma)
        g = fl + fr + (u_r - u_l)
        p_new = p - g / (dl + dr)
        if p_new <= 0.0:
            p_new = 0.5 * p
        if abs(p_new - p) <= tol * 0.5 * (p_new + p):
            p = p_new
            break
        p = p_new
    fl, _ = _wave_curve(p, rho_l, p_l, gamma)
    fr, _ = _wave_curve(p, rho_r, p_r, gamma)
    u = 0.5 * (u_l + u_r) + 0.5 * (fr - fl)
    g1 = (gamma - 1.0) / (gamma + 1.0)
    if p > p_l:
        rl = rho_l * (p / p_l + g1) / (g1 * p / p_l + 1.0)
    else:
        rl = rho_l * (p / p_l) ** (1.0 / gamma)
    if p > p_r:
        rr = rho_r * (p / p_r + g1) / (g1 * p / p_r + 1.0)
    else:
        rr = rho_r * (p / p_r) ** (1.0 / gamma)
    return Star(p=p, u=u, rho_l=rl, rho_r=rr)


def wave_speeds(left, right, gamma: float = 1.4) -> dict:
    """Shock speeds or rarefaction head/tail speeds of both waves."""
    st = star_state(left, right, gamma)
    rho_l, u_l, p_l = left
    rho_r, u_r, p_r = right
    a_l = math.sqrt(gamma * p_l / rho_l)
    a_r = math.sqrt(gamma * p_r / rho_r)
    out = {"contact": st.u}
    if st.p > p_l:
        out["left_shock"] = u_l - a_l * math.sqrt((gamma + 1) / (2 * gamma) * st.p / p_l + (gamma - 1) / (2 * gamma))
    else:
        a_sl = a_l * (st.p / p_l) ** ((gamma - 1) / (2 * gamma))
        out["left_head"] = u_l - a_l
        out["left_tail"] = st.u - a_sl
    if st.p > p_r:
        out["right_shock"] = u_r + a_r * math.sqrt((gamma + 1) / (2 * gamma) * st.p / p_r + (gamma - 1) / (2 * gamma))
    else:
        a_sr = a_r * (st.p / p_r) ** ((gamma - 1) / (2 * gamma))
        out["right_head"] = u_r + a_r
        out["right_tail"] = st.u + a_sr
    return out


def sample(left, right, xi, gamma: float = 1.4):
    """(rho, u, p) at similarity coordinates xi = (x - x0) / t (array)."""
    st = star_state(left, right, gamma)
    sp = wave_speeds(left, right, gamma)
    rho_l, u_l, p_l = left
    rho_r, u_r, p_r = right
    a_l = math.sqrt(gamma * p_l / rho_l)
    a_r = math.sqrt(gamma * p_r / rho_r)
    xi = np.asarray(xi, dtype=np.float64)
    rho = np.empty_like(xi)
    u = np.empty_like(xi)
    p = np.empty_like(xi)
    g = gamma
    for k, s in np.ndenumerate(xi):
        if s <= st.u:  # left of the contact
            if st.p > p_l:
                if s <= sp["left_shock"]:
                    r, v, q = rho_l, u_l, p_l
                else:
                    r, v, q = st.rho_l, st.u, st.p
            else:
                if s <= sp["left_head"]:
                    r, v, q = rho_l, u_l, p_l
                elif s >= sp["left_tail"]:
                    r, v, q = st.rho_l, st.u, st.p
                else:  # inside the left fan
                    c = 2.0 / (g + 1.0) + (g - 1.0) / ((g + 1.0) * a_l) * (u_l - s)
                    r = rho_l * c ** (2.0 / (g - 1.0))
                    v = 2.0 / (g + 1.0) * (a_l + 0.5 * (g - 1.0) * u_l + s)
                    q = p_l * c ** (2.0 * g / (g - 1.0))
        else:
            if st.p > p_r:
                if s >= sp["right_shock"]:
                    r, v, q = rho_r, u_r, p_r
                else:
                    r, v, q = st.rho_r, st.u, st.p
            else:
                if s >= sp["right_head"]:
                    r, v, q = rho_r, u_r, p_r
                elif s <= sp["right_tail"]:
                    r, v, q = st.rho_r, st.u, st.p
                else:  # inside the right fan
                    c = 2.0 / (g + 1.0) - (g - 1.0) / ((g + 1.0) * a_r) * (u_r - s)
                    r = rho_r * c ** (2.0 / (g - 1.0))
                    v = 2.0 / (g + 1.0) * (-a_r + 0.5 * (g - 1.0) * u_r + s)
                    q = p_r * c ** (2.0 * g / (g - 1.0))
        rho[k], u[k], p[k] = r, v, q
    return rho, u, p


def cell_averages(left, right, x_edges, x0: float, t: float, gamma: float = 1.4, sub: int = 16):
    """Exact solution averaged over cells [x_edges[k], x_edges[k+1]] (midpoint
    rule with ``sub`` sub-points per cell), for comparison with cell values."""
    x_edges = np.asarray(x_edges, dtype=np.float64)
    n = len(x_edges) - 1
    w = (np.arange(sub) + 0.5) / sub
    xs = x_edges[:-1, None] + (x_edges[1:] - x_edges[:-1])[:, None] * w[None, :]
    rho, u, p = sample(left, right, (xs - x0) / t, gamma)
    return rho.reshape(n, sub).mean(1), u.reshape(n, sub).mean(1), p.reshape(n, sub).mean(1)
