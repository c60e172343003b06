"""Pins of the oracle's discrete velocity model and equilibrium (Sec. 2).

The equilibrium is pinned by the five moment relations (e1)-(e5) that the
paper requires of it, which are independent of how A_i, B_i, D_i are written:
a dropped term, a wrong sign or a wrong shell in the coefficients breaks one
of them.  Both transcriptions of the equilibrium (oracle.c and the numpy one
in oracle.vonneumann) are checked.
"""
import numpy as np
import pytest

import oracle
from oracle import vonneumann as vn

PARAM_SETS = [
    # (c1, c2, eta0, gamma): the paper's runs (Sec. 3 and 4) and the workloads
    (2.0, 6.0, 2.0, 1.4),
    (8.0, 24.0, 8.0, 1.4),
    (2.0, 6.0, 4.0, 1.4),
    (4.0, 12.0, 4.0, 1.4),
    (20.0, 60.0, 20.0, 1.4),
    (12.0, 36.0, 20.0, 1.4),
    (3.0, 7.0, 1.5, 5.0 / 3.0),
]


def _states(seed, n=20):
    rng = np.random.default_rng(seed)
    for _ in range(n):
        rho = rng.uniform(0.1, 10.0)
        u = rng.uniform(-3.0, 3.0, size=3)
        T = rng.uniform(0.1, 5.0)
        yield rho, u, T


def _check_relations(f, v, eta, rho, u, T, gamma, tol=1e-13):
    b = 2.0 / (gamma - 1.0)
    P = rho * T
    usq = float(u @ u)
    vsq = (v * v).sum(1) + eta * eta
    scale_e = rho * (b * T + usq) + np.abs(f).sum() * (vsq.max())
    # (e1) mass
    assert abs(f.sum() - rho) <= tol * (rho + np.abs(f).sum())
    # (e2) momentum
    mom = (f[:, None] * v).sum(0)
    assert np.all(np.abs(mom - rho * u) <= tol * (np.abs(f)[:, None] * np.abs(v)).sum(0).max() * 10)
    # (e3) energy
    assert abs((f * vsq).sum() - rho * (b * T + usq)) <= tol * scale_e
    # (e4) pressure tensor
    Pi = np.einsum("i,ia,ib->ab", f, v, v)
    ref = P * np.eye(3) + rho * np.outer(u, u)
    scale4 = np.einsum("i,ia,ib->ab", np.abs(f), np.abs(v), np.abs(v)).max()
    assert np.all(np.abs(Pi - ref) <= tol * 10 * scale4)
    # (e5) energy flux
    q = (f * vsq)[:, None] * v
    lhs = q.sum(0)
    rhs = rho * ((b + 2.0) * T + usq) * u
    scale5 = (np.abs(f * vsq)[:, None] * np.abs(v)).sum(0).max()
    assert np.all(np.abs(lhs - rhs) <= tol * 10 * scale5)


@pytest.mark.parametrize("params", PARAM_SETS)
def test_feq_satisfies_moment_relations(params):
    c1, c2, eta0, gamma = params
    cfg = oracle.Cfg(nx=1, ny=1, nz=1, c1=c1, c2=c2, eta0=eta0, gamma=gamma)
    v, eta = oracle.velocities(cfg)
    for rho, u, T in _states(seed=int(c1 * 100 + eta0)):
        f = oracle.feq(cfg, rho, u, T)
        _check_relations(f, v, eta, rho, u, T, gamma)


@pytest.mark.parametrize("params", PARAM_SETS)
def test_numpy_equilibrium_satisfies_moment_relations(params):
    c1, c2, eta0, gamma = params
    v, eta = vn.velocity_set(c1, c2, eta0)
    for rho, u, T in _states(seed=7 + int(c2)):
        f = vn.equilibrium(rho, u, T, c1, c2, eta0, gamma)
        _check_relations(f, v, eta, rho, u, T, gamma)


def test_two_transcriptions_agree():
    for c1, c2, eta0, gamma in PARAM_SETS:
        cfg = oracle.Cfg(nx=1, ny=1, nz=1, c1=c1, c2=c2, eta0=eta0, gamma=gamma)
        for rho, u, T in _states(seed=3, n=5):
            a = oracle.feq(cfg, rho, u, T)
            b = vn.equilibrium(rho, u, T, c1, c2, eta0, gamma)
            assert np.max(np.abs(a - b)) <= 1e-14 * np.abs(a).max() * 10


def test_velocity_set_structure():
    """Sec. 2: one rest particle with eta0, six axis velocities of speed c1,
    eight diagonal velocities of speed c2 along (+-1,+-1,+-1)."""
    cfg = oracle.Cfg(nx=1, ny=1, nz=1, c1=2.0, c2=6.0, eta0=4.0)
    v, eta = oracle.velocities(cfg)
    speed = np.sqrt((v * v).sum(1))
    assert speed[0] == 0.0 and eta[0] == 4.0 and np.all(eta[1:] == 0.0)
    assert np.allclose(speed[1:7], 2.0, rtol=0, atol=1e-15)
    assert np.allclose(speed[7:], 6.0, rtol=1e-15)
    # axis velocities come in opposite pairs along x, y, z
    for a in range(3):
        assert np.array_equal(v[1 + 2 * a], -v[2 + 2 * a]) and v[1 + 2 * a, a] > 0
    # diagonals: all eight sign patterns, each exactly once, equal magnitude per component
    signs = {tuple(np.sign(row).astype(int)) for row in v[7:]}
    assert len(signs) == 8 and all(0 not in s for s in signs)
    assert np.allclose(np.abs(v[7:]), 6.0 / np.sqrt(3.0), rtol=1e-15)
    # the set is symmetric: sum of v_i and of v_i v_i v_i vanish
    assert np.allclose(v.sum(0), 0.0, atol=1e-14)


def test_moments_invert_equilibrium():
    cfg = oracle.Cfg(nx=1, ny=1, nz=1, c1=2.0, c2=6.0, eta0=2.0)
    for rho, u, T in _states(seed=11):
        m = oracle.moments(cfg, oracle.feq(cfg, rho, u, T))
        assert abs(m[0] - rho) <= 1e-13 * rho * 10
        assert np.allclose(m[1:4], u, rtol=0, atol=1e-12)
        assert abs(m[4] - T) <= 1e-12 * max(1.0, T)


def test_rest_particle_weight_closed_form():
    """f_1^eq = rho (b - 3) T / eta0^2: the rest particle carries no B or D term."""
    cfg = oracle.Cfg(nx=1, ny=1, nz=1, c1=2.0, c2=6.0, eta0=3.0, gamma=1.4)
    f = oracle.feq(cfg, 1.7, [0.4, -0.1, 0.9], 0.8)
    b = 5.0
    assert abs(f[0] - 1.7 * (b - 3.0) * 0.8 / 9.0) <= 1e-15
