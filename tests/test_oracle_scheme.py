"""Pins of the oracle's convection and dissipation terms (Sec. 3).

With tau = inf (no relaxation) and the dissipation term off, each f_i obeys
the pure advection equation d f_i/dt + v_ia d f_i/dx_a = 0 discretised by
the NND flux and a forward Euler step.  Properties that fix the scheme:

* on linear data the NND flux difference is the exact derivative, so one step
  moves a linear profile by exactly -dt v b (a wrong upwind side, a wrong
  minmod sign or a missing 1/2 breaks it);
* minmod-limited MUSCL fluxes with forward Euler at small Courant number are
  total-variation diminishing and create no new extrema;
* on smooth data the scheme is second-order accurate (first-order upwind is
  first order, the second-order upwind variant second order);
* the dissipation term alone is the heat equation with the printed lambda_i.
"""
import math

import numpy as np
import pytest

import oracle

C1, C2, ETA0 = 2.0, 6.0, 2.0


def _advect_cfg(nx, ny=1, nz=1, dx=0.01, dt=1e-3, scheme=oracle.NND, bc=oracle.PERIODIC):
    return oracle.Cfg(nx=nx, ny=ny, nz=nz, c1=C1, c2=C2, eta0=ETA0, gamma=1.4, tau=math.inf, dt=dt, dx=dx,
                      bc_lo=(bc,) * 3, bc_hi=(bc,) * 3, scheme=scheme, dissipation=0)


def test_linear_profile_moves_exactly():
    """Interior nodes whose stencil is interior: one step gives f - dt v_ix b."""
    nx, dx, dt = 24, 0.01, 1e-3
    cfg = _advect_cfg(nx, 3, 3, dx=dx, dt=dt)
    # data constant in y and z (periodic there); x faces fixed, and only nodes
    # at least three cells from them are checked, so no boundary value enters
    cfg.bc_lo = (oracle.FIXED, oracle.PERIODIC, oracle.PERIODIC)
    cfg.bc_hi = (oracle.FIXED, oracle.PERIODIC, oracle.PERIODIC)
    x = (np.arange(nx) + 0.5) * dx
    f = np.empty((15, 3, 3, nx))
    slopes = np.linspace(-2.0, 3.0, 15)
    for i in range(15):
        f[i] = 1.0 + slopes[i] * x
    v, _ = oracle.velocities(cfg)
    g = oracle.step(cfg, f)
    for i in range(15):
        expect = f[i, 1, 1, 3:-3] - dt * v[i, 0] * slopes[i]
        assert np.max(np.abs(g[i, 1, 1, 3:-3] - expect)) <= 1e-13


@pytest.mark.parametrize("i", [1, 2, 7, 14])
def test_step_profile_is_tvd(i):
    nx, dx = 80, 0.01
    cfg = _advect_cfg(nx, dx=dx, dt=0.4 * dx / C2)
    x = np.arange(nx)
    prof = np.where((x > 20) & (x < 45), 2.0, 0.5) + 0.3 * (x > 60)
    f = np.tile(prof, (15, 1, 1, 1)).astype(float)
    tv0 = np.abs(np.diff(prof, append=prof[:1])).sum()
    lo, hi = prof.min(), prof.max()
    g = f
    for _ in range(60):
        g = oracle.step(cfg, g)
        p = g[i, 0, 0]
        tv = np.abs(np.diff(p, append=p[:1])).sum()
        assert tv <= tv0 * (1 + 1e-12)
        assert p.min() >= lo - 1e-12 and p.max() <= hi + 1e-12
        tv0 = tv


def _sine_error(nx, scheme, i=1):
    """L1 error of advecting one sine period for a quarter domain crossing.
    dt ~ dx^2 so that the first-order time error of forward Euler does not
    mask the spatial order."""
    L = 1.0
    dx = L / nx
    v = C1
    dt = 0.2 * dx / C2 * (32 * dx)
    t_end = 0.25 * L / v
    nsteps = int(round(t_end / dt))
    dt = t_end / nsteps
    cfg = _advect_cfg(nx, dx=dx, dt=dt, scheme=scheme)
    x = (np.arange(nx) + 0.5) * dx
    f = np.tile(np.sin(2 * np.pi * x / L) + 2.0, (15, 1, 1, 1))
    g = oracle.run(cfg, f, nsteps)
    exact = np.sin(2 * np.pi * (x - v * t_end) / L) + 2.0
    return np.abs(g[i, 0, 0] - exact).mean()


@pytest.mark.parametrize("scheme,lo,hi", [(oracle.NND, 1.65, 2.2), (oracle.UPWIND2, 1.85, 2.1),
                                          (oracle.UPWIND1, 0.85, 1.1)])
def test_order_of_accuracy(scheme, lo, hi):
    """Spatial order on smooth data: NND close to 2 (minmod clips the two
    extrema), second-order upwind 2, first-order upwind 1."""
    e1 = _sine_error(64, scheme)
    e2 = _sine_error(128, scheme)
    order = math.log2(e1 / e2)
    assert lo <= order <= hi, order


def test_upwind_direction():
    """f_2 (v = +c1 x) and f_3 (v = -c1 x) carry a bump in opposite directions
    with the speed c1: centroid shift = v t."""
    nx, dx = 200, 0.005
    dt = 0.2 * dx / C2
    n = 400
    cfg = _advect_cfg(nx, dx=dx, dt=dt)
    x = (np.arange(nx) + 0.5) * dx
    bump = np.exp(-((x - 0.5) / 0.05) ** 2)
    f = np.tile(bump, (15, 1, 1, 1))
    g = oracle.run(cfg, f, n)
    t = n * dt
    for i, vx in [(1, C1), (2, -C1), (0, 0.0), (7, C2 / math.sqrt(3)), (14, -C2 / math.sqrt(3))]:
        c = (g[i, 0, 0] * x).sum() / g[i, 0, 0].sum()
        assert abs(c - (0.5 + vx * t)) < 0.05 * dx + 2e-3 * abs(vx * t), (i, c)


def test_dissipation_is_heat_equation():
    """With v_i = 0 (the rest particle) and no relaxation, the extra term of
    Eq. "lp" alone damps a Fourier mode by exactly 1 - 4 lambda dt sin^2(k dx/2)/dx^2
    per step, lambda_1 = c1 dx; the axis particles use c1 dx / 10 (not checked
    here: they also advect); the diagonal particles use 0."""
    nx, dx, dt = 32, 0.01, 1e-4
    cfg = oracle.Cfg(nx=nx, ny=1, nz=1, c1=C1, c2=C2, eta0=ETA0, tau=math.inf, dt=dt, dx=dx, dissipation=1)
    x = np.arange(nx)
    m = 3
    mode = np.cos(2 * np.pi * m * x / nx)
    f = np.tile(mode, (15, 1, 1, 1))
    g = oracle.step(cfg, f)
    lam = C1 * dx
    factor = 1.0 - 4.0 * lam * dt * math.sin(math.pi * m / nx) ** 2 / dx ** 2
    assert np.max(np.abs(g[0, 0, 0] - factor * mode)) <= 1e-14
    # a pure-y axis particle and a diagonal particle see the x mode through
    # advection only when v_x != 0; f_4 (v = +c1 y) has v_x = 0 so only lambda_i acts
    lam4 = C1 * dx / 10.0
    factor4 = 1.0 - 4.0 * lam4 * dt * math.sin(math.pi * m / nx) ** 2 / dx ** 2
    assert np.max(np.abs(g[3, 0, 0] - factor4 * mode)) <= 1e-14


def test_relaxation_with_dt_equal_tau_gives_equilibrium_plus_transport():
    """With dt = tau the BGK term replaces f by f^eq; on a uniform state the
    transport terms vanish, so one step maps any f to f^eq of its moments."""
    cfg = oracle.Cfg(nx=4, ny=3, nz=2, c1=C1, c2=C2, eta0=ETA0, tau=1e-5, dt=1e-5, dx=0.01)
    rng = np.random.default_rng(0)
    f0 = oracle.feq(cfg, 1.2, [0.2, 0.1, -0.3], 1.1) + 0.01 * rng.uniform(-1, 1, 15)
    f = np.broadcast_to(f0[:, None, None, None], (15, 2, 3, 4)).copy()
    g = oracle.step(cfg, f)
    m = oracle.moments(cfg, f0)
    expect = oracle.feq(cfg, m[0], m[1:4], m[4])
    assert np.max(np.abs(g - expect[:, None, None, None])) <= 1e-14
