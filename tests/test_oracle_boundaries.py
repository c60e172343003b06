"""Pins of the oracle's boundary layers (Sec. 4(2)).

The paper defines the two layers outside a face by their macroscopic values:
fixed post-shock values on the right (both layers), linear extrapolation on
the left (rho(1) = 2 rho(2) - rho(3), rho(0) = 2 rho(1) - rho(2), the same
for T and u), and reflection on the side walls (the wall layer copies the
last interior node with u_n = 0; the outer layer copies it with u_n
negated).  The layers hold f = f^eq of those values, so their moments must
return them exactly; periodic faces copy f.
"""
import numpy as np
import pytest

import oracle
import workloads

C = dict(c1=2.0, c2=6.0, eta0=2.0, gamma=1.4, dt=1e-4, tau=1e-4, dx=0.01)


def _ghost_macros(cfg, P, i_axis, pos_ghost, cross):
    """Moments of the padded array's node at ghost coordinate pos_ghost along
    i_axis (interior coordinates), cross = the other two interior coordinates."""
    q = [0, 0, 0]
    others = [a for a in range(3) if a != i_axis]
    q[i_axis] = pos_ghost
    q[others[0]], q[others[1]] = cross
    x, y, z = q
    return oracle.moments(cfg, P[:, z + 2, y + 2, x + 2])


def _field(cfg, seed):
    rho, u, T = workloads.smooth_random_fields(cfg.nx, cfg.ny, cfg.nz, seed, amp=0.2)
    return oracle.init(cfg, rho, u, T), rho, u, T


def test_fixed_layers_hold_given_state():
    left = (2.66667, 1.47902, 0.0, 0.0, 1.6875)
    right = (1.0, 0.0, 0.0, 0.0, 1.0)
    cfg = oracle.Cfg(nx=6, ny=4, nz=3, bc_lo=(1, 0, 0), bc_hi=(1, 0, 0), fixed_lo=(left,) * 3,
                     fixed_hi=(right,) * 3, **C)
    f, *_ = _field(cfg, 1)
    P = oracle.padded(cfg, f)
    for y in range(cfg.ny):
        for z in range(cfg.nz):
            for g in (-1, -2):
                assert np.allclose(_ghost_macros(cfg, P, 0, g, (y, z))[:5], left, rtol=1e-13, atol=1e-13)
            for g in (cfg.nx, cfg.nx + 1):
                assert np.allclose(_ghost_macros(cfg, P, 0, g, (y, z))[:5], right, rtol=1e-13, atol=1e-13)


def test_extrapolation_continues_linear_profiles():
    cfg = oracle.Cfg(nx=7, ny=3, nz=3, bc_lo=(2, 0, 0), bc_hi=(2, 0, 0), **C)
    x = np.arange(cfg.nx, dtype=float)
    shape = (cfg.nz, cfg.ny, cfg.nx)
    rho = (1.0 + 0.05 * x) * np.ones(shape)
    u = np.stack([(0.2 - 0.03 * x) * np.ones(shape), (0.1 + 0.01 * x) * np.ones(shape),
                  (-0.05 + 0.02 * x) * np.ones(shape)])
    T = (1.5 - 0.04 * x) * np.ones(shape)
    f = oracle.init(cfg, rho, u, T)
    P = oracle.padded(cfg, f)
    for g in (-2, -1, cfg.nx, cfg.nx + 1):
        m = _ghost_macros(cfg, P, 0, g, (1, 2))
        expect = [1.0 + 0.05 * g, 0.2 - 0.03 * g, 0.1 + 0.01 * g, -0.05 + 0.02 * g, 1.5 - 0.04 * g]
        assert np.allclose(m[:5], expect, rtol=0, atol=1e-13), (g, m[:5], expect)


def test_extrapolation_formula_on_nonlinear_data():
    """rho(1) = 2 rho(2) - rho(3), rho(0) = 2 rho(1) - rho(2) in the paper's
    numbering, i.e. g1 = 2 m0 - m1 and g2 = 2 g1 - m0 in ours."""
    cfg = oracle.Cfg(nx=5, ny=4, nz=3, bc_lo=(0, 2, 0), bc_hi=(0, 2, 0), **C)
    f, rho, u, T = _field(cfg, 7)
    P = oracle.padded(cfg, f)
    for xz in [(0, 0), (3, 2), (4, 1)]:
        x, z = xz
        m0 = np.array([rho[z, 0, x], *u[:, z, 0, x], T[z, 0, x]])
        m1 = np.array([rho[z, 1, x], *u[:, z, 1, x], T[z, 1, x]])
        g1 = _ghost_macros(cfg, P, 1, -1, (x, z))[:5]
        g2 = _ghost_macros(cfg, P, 1, -2, (x, z))[:5]
        assert np.allclose(g1, 2 * m0 - m1, rtol=1e-12, atol=1e-12)
        assert np.allclose(g2, 2 * (2 * m0 - m1) - m0, rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("axis", [0, 1, 2])
def test_reflection_layers(axis):
    bc = [0, 0, 0]
    bc[axis] = 3
    cfg = oracle.Cfg(nx=5, ny=4, nz=6, bc_lo=tuple(bc), bc_hi=tuple(bc), **C)
    f, rho, u, T = _field(cfg, 11 + axis)
    P = oracle.padded(cfg, f)
    n = (cfg.nx, cfg.ny, cfg.nz)[axis]
    others = [a for a in range(3) if a != axis]
    for hi in (0, 1):
        last = n - 1 if hi else 0
        wall = n if hi else -1
        outer = n + 1 if hi else -2
        for cross in [(0, 0), (1, 2), (2, 3)]:
            q = [0, 0, 0]
            q[axis] = last
            q[others[0]], q[others[1]] = cross
            x, y, z = q
            m0 = np.array([rho[z, y, x], *u[:, z, y, x], T[z, y, x]])
            w = _ghost_macros(cfg, P, axis, wall, cross)[:5]
            o = _ghost_macros(cfg, P, axis, outer, cross)[:5]
            ew = m0.copy()
            ew[1 + axis] = 0.0
            eo = m0.copy()
            eo[1 + axis] = -m0[1 + axis]
            assert np.allclose(w, ew, rtol=1e-12, atol=1e-12)
            assert np.allclose(o, eo, rtol=1e-12, atol=1e-12)


def test_periodic_layers_copy_f():
    cfg = oracle.Cfg(nx=5, ny=4, nz=3, **C)
    f, *_ = _field(cfg, 2)
    P = oracle.padded(cfg, f)
    assert np.array_equal(P[:, 2:-2, 2:-2, 0:2], f[:, :, :, -2:])
    assert np.array_equal(P[:, 2:-2, 2:-2, -2:], f[:, :, :, :2])
    assert np.array_equal(P[:, 2:-2, 0:2, 2:-2], f[:, :, -2:, :])
    assert np.array_equal(P[:, 0:2, 2:-2, 2:-2], f[:, -2:, :, :])


def test_single_cell_periodic_axis_wraps_onto_itself():
    cfg = oracle.Cfg(nx=6, ny=1, nz=1, **C)
    f, *_ = _field(cfg, 3)
    P = oracle.padded(cfg, f)
    for dy in (0, 1, 3, 4):
        assert np.array_equal(P[:, 2, dy, 2:-2], f[:, 0, 0, :])


def test_invalid_configurations_are_rejected():
    f = np.zeros((15, 1, 1, 4))
    with pytest.raises(ValueError):
        oracle.step(oracle.Cfg(nx=4, ny=1, nz=1, bc_lo=(0, 0, 0), bc_hi=(1, 0, 0), **C), f)
    with pytest.raises(ValueError):
        oracle.step(oracle.Cfg(nx=1, ny=1, nz=1, bc_lo=(2, 0, 0), bc_hi=(2, 0, 0), **C), np.zeros((15, 1, 1, 1)))
