"""The synthetic workloads: initial fields of the paper's configurations."""
import numpy as np

import workloads


def test_sharp_sphere_reproduces_cell_centre_membership():
    w = workloads.shock_sphere("s", 24, 20, 16, 1.0 / 20, 2.0, 5.0, 0.2, (0.5, 0.5, 0.4), 2.0, 6.0, 4.0, 1e-5, 1e-5,
                               1, width=0.0)
    rho, u, T = w.initial_fields()
    x = (np.arange(24) + 0.5) / 20
    y = (np.arange(20) + 0.5) / 20
    z = (np.arange(16) + 0.5) / 20
    r2 = (x[None, None, :] - 0.5) ** 2 + (y[None, :, None] - 0.5) ** 2 + (z[:, None, None] - 0.4) ** 2
    inside = r2 <= 0.04
    assert inside.any() and (~inside).any()
    assert np.array_equal(rho, np.where(inside, 5.0, 1.0))
    assert np.array_equal(T, np.where(inside, 1.0 / 5.0, 1.0))
    assert not u.any()


def test_smoothed_interfaces_keep_the_pressure_and_the_end_states():
    w = workloads.shock_bubble(64, 32, 32, mach=3.0)  # one-cell tanh surface
    rho, u, T = w.initial_fields()
    assert np.allclose(rho * T, 1.0, rtol=1e-14)            # pressure-matched blend
    assert abs(rho.min() - 0.1) < 1e-3 and rho.max() == 1.0  # both end states (the centre within tanh(4.8))
    mixed = (rho > 0.11) & (rho < 0.99)
    assert 0 < mixed.sum() < rho.size // 4                   # a thin shell
    r2, u2, p2, _ = workloads.rankine_hugoniot(1.5)
    t = workloads.shock_tube("t", 40, 4, 4, 1 / 40, (r2, u2, 0, 0, p2 / r2), (1, 0, 0, 0, 1), 0.5, 2, 6, 2, 1e-5,
                             1e-5, 1, width=1.0)
    rho, u, T = t.initial_fields()
    p = rho * T
    assert np.all(np.diff(rho[0, 0]) <= 0) and np.all(np.diff(u[0, 0, 0]) <= 0) and np.all(np.diff(p[0, 0]) <= 1e-15)
    assert rho[0, 0, 0] == r2 and rho[0, 0, -1] == 1.0


def test_paper_tubes_are_sharp():
    for w in (workloads.lax_tube(), workloads.high_mach_tube()):
        rho, u, T = w.initial_fields()
        assert len(np.unique(rho)) == 2 and len(np.unique(T)) == 2
