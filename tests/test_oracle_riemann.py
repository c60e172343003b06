"""Pins of the exact Riemann solver and of the oracle's 1D reduction (Sec. 4(1)-(2)).

* The paper prints the Mach-2 post-shock state (rho = 2.66667, |u| = 1.47902,
  T = 1.6875) and the shock speed D = 2.36643 for a shock into (1, 0, p=1):
  the Rankine-Hugoniot helper of the workloads and the shock branch of the
  exact solver must reproduce them.
* Star states found by the solver satisfy the jump conditions across each
  shock (mass, momentum and energy fluxes) and the isentropic relations
  across each rarefaction, checked directly from the conservation laws.
* The paper's printed initial data: Lax temperatures are p/rho with R = 1,
  and the high-Mach left state has Mach number 10.
* The oracle's 1D reduction of the Lax tube approaches the exact solution:
  NND beats first-order upwind, and halving dx lowers the error.
"""
import math

import numpy as np
import pytest

import oracle
import workloads
from oracle import riemann

G = 1.4


def _digits(x, n):
    return float(f"{x:.{n}g}")


def test_mach2_post_shock_state_matches_paper(golden):
    g = golden("mach2_shock.json")
    rho2, u2, p2, D = workloads.rankine_hugoniot(g["mach"], g["pre_shock"]["rho"], g["pre_shock"]["p"], g["gamma"])
    post = g["post_shock"]
    assert _digits(rho2, 6) == pytest.approx(post["rho"], abs=1e-5)
    assert _digits(u2, 6) == pytest.approx(post["u1_magnitude"], abs=1e-5)
    assert p2 / rho2 == pytest.approx(post["T"], rel=1e-12)
    assert _digits(D, 6) == pytest.approx(g["shock_speed_D"], abs=1e-5)
    # the garbled fifth entry is the product of the two printed values rho * |u|
    assert _digits(post["rho"] * post["u1_magnitude"], 6) == pytest.approx(3.94406, abs=1e-12)
    assert rho2 * u2 == pytest.approx(3.94406, abs=2e-5)
    # shock Mach number as the paper defines it: (D - u)/sqrt(gamma T) ahead of the shock
    assert (D - 0.0) / math.sqrt(G * 1.0) == pytest.approx(2.0, rel=1e-12)


def test_exact_solver_shock_branch_reproduces_single_shock():
    rho2, u2, p2, D = workloads.rankine_hugoniot(2.0)
    st = riemann.star_state((rho2, u2, p2), (1.0, 0.0, 1.0), G)
    assert st.p == pytest.approx(p2, rel=1e-12)
    assert st.u == pytest.approx(u2, rel=1e-12)
    assert st.rho_r == pytest.approx(rho2, rel=1e-12)
    sp = riemann.wave_speeds((rho2, u2, p2), (1.0, 0.0, 1.0), G)
    assert sp["right_shock"] == pytest.approx(D, rel=1e-12)


def _check_shock(pre, post, S):
    """Rankine-Hugoniot: fluxes in the shock frame are continuous."""
    r1, u1, p1 = pre
    r2, u2, p2 = post
    w1, w2 = u1 - S, u2 - S
    e1 = p1 / (G - 1) + 0.5 * r1 * w1 * w1
    e2 = p2 / (G - 1) + 0.5 * r2 * w2 * w2
    assert r1 * w1 == pytest.approx(r2 * w2, rel=1e-10)
    assert r1 * w1 * w1 + p1 == pytest.approx(r2 * w2 * w2 + p2, rel=1e-10)
    assert w1 * (e1 + p1) == pytest.approx(w2 * (e2 + p2), rel=1e-10)


def _check_rarefaction(outer, inner, sign):
    """Isentropic: p / rho^gamma and u -+ 2a/(gamma-1) are unchanged across the fan
    (sign = +1 for a left-facing wave, -1 for a right-facing one)."""
    r1, u1, p1 = outer
    r2, u2, p2 = inner
    a1 = math.sqrt(G * p1 / r1)
    a2 = math.sqrt(G * p2 / r2)
    assert p1 / r1 ** G == pytest.approx(p2 / r2 ** G, rel=1e-10)
    assert u1 + sign * 2 * a1 / (G - 1) == pytest.approx(u2 + sign * 2 * a2 / (G - 1), rel=1e-10)


@pytest.mark.parametrize("left,right", [
    ((0.445, 0.698, 3.528), (0.5, 0.0, 0.571)),     # Lax
    ((5.0, 0.0, 500.0), (1.0, 0.0, 1.0)),           # high-Mach workload
    ((100.0, 10.0, 71.4286), (150.0, 0.0, 7500.0)),  # the paper's high-Mach tube
    ((1.0, 0.0, 1.0), (0.125, 0.0, 0.1)),           # a classical shock tube
    ((1.0, -1.0, 1.0), (1.0, 1.0, 1.0)),            # two rarefactions
    ((1.0, 1.0, 1.0), (1.0, -1.0, 1.0)),            # two shocks
])
def test_star_state_satisfies_jump_conditions(left, right):
    st = riemann.star_state(left, right, G)
    sp = riemann.wave_speeds(left, right, G)
    if "left_shock" in sp:
        _check_shock(left, (st.rho_l, st.u, st.p), sp["left_shock"])
    else:
        _check_rarefaction(left, (st.rho_l, st.u, st.p), +1)
    if "right_shock" in sp:
        _check_shock(right, (st.rho_r, st.u, st.p), sp["right_shock"])
    else:
        _check_rarefaction(right, (st.rho_r, st.u, st.p), -1)
    # the sampled profile is continuous through a fan and equals the star state beside the contact
    r, u, p = riemann.sample(left, right, np.array([st.u - 1e-9, st.u + 1e-9]), G)
    assert r[0] == pytest.approx(st.rho_l, rel=1e-9) and r[1] == pytest.approx(st.rho_r, rel=1e-9)
    assert np.allclose(p, st.p, rtol=1e-9)


def test_printed_initial_states(golden):
    g = golden("shock_tube_states.json")
    lax = g["lax"]
    assert _digits(lax["pressure_left"] / lax["left"][0], 4) == lax["left"][4]
    assert _digits(lax["pressure_right"] / lax["right"][0], 4) == lax["right"][4]
    hm = g["high_mach"]
    mach = hm["left"][1] / math.sqrt(hm["gamma"] * hm["left"][4])
    assert mach == pytest.approx(hm["left_mach"], rel=1e-6)
    # the workloads use the same Lax states
    assert workloads.LAX_LEFT[4] == pytest.approx(lax["left"][4], abs=5e-4)
    assert workloads.LAX_RIGHT[4] == pytest.approx(lax["right"][4], abs=5e-4)


def _lax_error(nx, scheme=oracle.NND, steps_per_200=7000):
    w = workloads.lax_tube(nx=nx, ny=1, nz=1)
    steps = steps_per_200 * nx // 200
    dt = 0.14 / steps
    cfg = oracle.cfg_for(w, dt=dt, tau=dt, scheme=scheme)
    rho, u, T = w.initial_fields()
    f = oracle.run(cfg, oracle.init(cfg, rho, u, T), steps)
    r, _, _ = oracle.macros(cfg, f)
    L = (workloads.LAX_LEFT[0], workloads.LAX_LEFT[1], workloads.LAX_LEFT[0] * workloads.LAX_LEFT[4])
    R = (workloads.LAX_RIGHT[0], workloads.LAX_RIGHT[1], workloads.LAX_RIGHT[0] * workloads.LAX_RIGHT[4])
    edges = np.arange(nx + 1) * w.dx
    re, _, _ = riemann.cell_averages(L, R, edges, 0.5, 0.14, G)
    return np.abs(r[0, 0] - re).sum() / np.abs(re).sum()


def test_lax_tube_1d_reduction_against_exact():
    e_nnd = _lax_error(200)
    e_up1 = _lax_error(200, scheme=oracle.UPWIND1)
    assert 0.03 < e_nnd < 0.065, e_nnd
    assert e_nnd < 0.8 * e_up1, (e_nnd, e_up1)


@pytest.mark.slow
def test_lax_tube_grid_convergence():
    assert _lax_error(400) < 0.75 * _lax_error(200)
