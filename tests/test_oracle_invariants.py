"""Invariants of the full oracle step (Secs. 2-3).

* A uniform equilibrium state is a fixed point (all differences vanish and
  f = f^eq), under every boundary kind that is consistent with it.
* Under periodic boundaries the flux form of Eq. "nnd" and the central
  Laplacian telescope, and BGK relaxation conserves rho, rho u and the energy
  (relations e1-e3), so the global sums are constant to rounding.
* The step commutes with the symmetries of the velocity set: exchanging the
  y and z axes, and mirroring y -> -y.
"""
import numpy as np
import pytest

import oracle
import workloads

C = dict(c1=2.0, c2=6.0, eta0=2.0, gamma=1.4)


def _perm(v, fn):
    """Index map i -> j with v_j = fn(v_i)."""
    out = np.empty(15, dtype=int)
    for i in range(15):
        tgt = fn(v[i])
        j = np.where(np.all(np.abs(v - tgt) < 1e-12, axis=1))[0]
        assert len(j) == 1
        out[i] = j[0]
    return out


def _noisy_state(cfg, seed, amp=0.02):
    rho, u, T = workloads.smooth_random_fields(cfg.nx, cfg.ny, cfg.nz, seed)
    f = oracle.init(cfg, rho, u, T)
    return f * (1.0 + workloads.noise(f.shape, seed + 1, amp))


@pytest.mark.parametrize("bcs", [
    ((0, 0, 0), (0, 0, 0)),
    ((1, 0, 0), (1, 0, 0)),
    ((2, 3, 3), (2, 3, 3)),
    ((1, 3, 2), (2, 3, 2)),
])
def test_uniform_state_is_preserved(bcs):
    state = (1.3, 0.4, 0.0, 0.0, 0.9)  # u_n = 0 on the y/z faces so reflection is consistent
    cfg = oracle.Cfg(nx=9, ny=6, nz=5, dt=1e-4, tau=2e-4, dx=0.01, bc_lo=bcs[0], bc_hi=bcs[1],
                     fixed_lo=(state,) * 3, fixed_hi=(state,) * 3, **C)
    n = cfg.ncell
    f = oracle.init(cfg, np.full(n, state[0]), np.repeat(np.array(state[1:4]), n), np.full(n, state[4]))
    g = oracle.run(cfg, f, 10)
    assert np.max(np.abs(g - f)) <= 1e-14 * np.abs(f).max() * 20


def test_periodic_conservation():
    cfg = oracle.Cfg(nx=12, ny=8, nz=6, dt=2e-4, tau=5e-4, dx=0.02, **C)
    f = _noisy_state(cfg, seed=3)
    v, eta = oracle.velocities(cfg)
    before = oracle.conserved(cfg, f)
    g = oracle.run(cfg, f, 20)
    after = oracle.conserved(cfg, g)
    vsq = (v * v).sum(1) + eta * eta
    scale = np.array([np.abs(f).sum(), *(np.abs(f).sum(axis=(1, 2, 3)) @ np.abs(v)), np.abs(f).sum(axis=(1, 2, 3)) @ vsq])
    assert np.all(np.abs(after - before) <= 1e-13 * scale), (after - before) / scale
    # the state did change: the check is not vacuous
    assert np.max(np.abs(g - f)) > 1e-3 * np.abs(f).max()


@pytest.mark.parametrize("scheme", [oracle.NND, oracle.UPWIND2, oracle.UPWIND1])
def test_yz_exchange_symmetry(scheme):
    cfg = oracle.Cfg(nx=7, ny=6, nz=6, dt=2e-4, tau=4e-4, dx=0.02, scheme=scheme, **C)
    v, _ = oracle.velocities(cfg)
    p = _perm(v, lambda w: np.array([w[0], w[2], w[1]]))
    f = _noisy_state(cfg, seed=5)
    fs = np.empty_like(f)
    fs[p] = f.transpose(0, 2, 1, 3)
    g = oracle.step(cfg, f)
    gs = oracle.step(cfg, fs)
    assert np.max(np.abs(gs[p] - g.transpose(0, 2, 1, 3))) <= 1e-14 * np.abs(g).max() * 10


@pytest.mark.parametrize("bc", [oracle.PERIODIC, oracle.REFLECT, oracle.EXTRAPOLATE])
def test_y_mirror_symmetry(bc):
    cfg = oracle.Cfg(nx=6, ny=7, nz=5, dt=2e-4, tau=4e-4, dx=0.02, bc_lo=(0, bc, 0), bc_hi=(0, bc, 0), **C)
    v, _ = oracle.velocities(cfg)
    p = _perm(v, lambda w: np.array([w[0], -w[1], w[2]]))
    f = _noisy_state(cfg, seed=9)
    fm = np.empty_like(f)
    fm[p] = f[:, :, ::-1, :]
    g = oracle.step(cfg, f)
    gm = oracle.step(cfg, fm)
    assert np.max(np.abs(gm[p] - g[:, :, ::-1, :])) <= 1e-14 * np.abs(g).max() * 10


def test_threads_do_not_change_results():
    cfg = oracle.Cfg(nx=10, ny=6, nz=8, dt=2e-4, tau=4e-4, dx=0.02, **C)
    f = _noisy_state(cfg, seed=2)
    a = oracle.run(cfg, f, 3, nthreads=1)
    b = oracle.run(cfg, f, 3, nthreads=4)
    assert np.array_equal(a, b)


def test_step_nodes_matches_full_step():
    """The node-wise evaluation (boundary layers read on the fly) equals the
    full step, bit for bit, including nodes next to every kind of face."""
    state = (1.1, 0.3, 0.0, 0.0, 1.2)
    cfg = oracle.Cfg(nx=8, ny=6, nz=5, dt=2e-4, tau=4e-4, dx=0.02, bc_lo=(1, 3, 0), bc_hi=(2, 3, 0),
                     fixed_lo=(state,) * 3, **C)
    f = _noisy_state(cfg, seed=4)
    g = oracle.step(cfg, f)
    rng = np.random.default_rng(0)
    xyz = np.stack([rng.integers(0, n, 40) for n in (cfg.nx, cfg.ny, cfg.nz)], axis=1)
    xyz = np.concatenate([xyz, [[0, 0, 0], [7, 5, 4], [1, 0, 2], [6, 5, 0]]])
    out = oracle.step_nodes(cfg, f, xyz)
    for k, (x, y, z) in enumerate(xyz):
        assert np.array_equal(out[k], g[:, z, y, x])


@pytest.mark.parametrize("gamma", [1.4, 5.0 / 3.0])
def test_conserved_closed_form_of_uniform_equilibria(gamma):
    """oracle.conserved against the closed form of relations e1-e3 (Sec. 2):
    a cell holding f^eq(rho, u, T) carries mass rho, momentum rho u and
    energy rho (b T + |u|^2) with b = 2 / (gamma - 1).  Two states with
    momentum components of different sizes and signs fill the two halves of
    the grid, so a swapped, dropped or sign-flipped velocity weight, a
    missing eta_0 term or a wrong energy weight changes a sum."""
    cfg = oracle.Cfg(nx=6, ny=4, nz=3, gamma=gamma, c1=2.0, c2=6.0, eta0=3.0)
    b = 2.0 / (gamma - 1.0)
    A = (1.3, 0.4, -0.7, 0.25, 0.9)
    B = (0.6, -1.1, 0.3, 0.8, 2.5)
    left = np.zeros((cfg.nz, cfg.ny, cfg.nx), dtype=bool)
    left[..., : cfg.nx // 2] = True
    rho = np.where(left, A[0], B[0])
    u = np.stack([np.where(left, A[1 + a], B[1 + a]) for a in range(3)])
    T = np.where(left, A[4], B[4])
    got = oracle.conserved(cfg, oracle.init(cfg, rho, u, T))
    half = cfg.ncell // 2

    def cell(s):
        usq = s[1] ** 2 + s[2] ** 2 + s[3] ** 2
        return np.array([s[0], s[0] * s[1], s[0] * s[2], s[0] * s[3], s[0] * (b * s[4] + usq)])

    want = half * (cell(A) + cell(B))
    assert np.all(np.abs(got - want) <= 1e-12 * np.abs(want)), (got, want)
