"""The on-device von Neumann service (lbm_vn_max_growth, Sec. 3) against the
oracle's amplification matrix (oracle/vonneumann.py: the equilibrium
Jacobian by complex-step differentiation of a second transcription of
Eq. "eq", numpy eigenvalues), at the parameters of the paper's Figs. 2 and 3
with and without the extra dissipation term, along x and along (1, 1, 1),
over 121 wave numbers; a batch of parameter sets and states in one launch;
and the serving parameter rule evaluated on the device against the host."""
import math

import numpy as np
import pytest

from oracle import vonneumann

pytestmark = pytest.mark.gpu

GAMMA = 1.4  # b = 5, as Figs. 2-5 use
TOL = 1e-10  # relative, on max |omega|


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


@pytest.mark.parametrize("direction", [(1.0, 0.0, 0.0), (1.0, 1.0, 1.0)])
@pytest.mark.parametrize("dissipation", [True, False])
@pytest.mark.parametrize("fig", ["fig2", "fig3"])
def test_max_growth_matches_oracle_at_the_papers_parameters(golden, fig, dissipation, direction):
    from paper_1010_4135_gb300 import stability
    g = golden("stability_params.json")[fig]
    st, (c1, c2, eta0) = g["state"], g["c"]
    nk = 121
    kdx = math.pi * np.arange(1, nk + 1) / nk
    want = vonneumann.max_growth(st[0], st[1:4], st[4], c1, c2, eta0, GAMMA, g["dt"], g["tau"], g["dx"], kdx,
                                 direction, dissipation=dissipation)
    got = stability.max_growth_device([st], [(c1, c2, eta0, GAMMA, g["dt"], g["tau"], g["dx"])],
                                      directions=[direction], nk=nk, dissipation=dissipation)[0]
    assert abs(got - want) <= TOL * want, (got, want)


def test_batched_parameter_sets_and_states_match_oracle():
    from paper_1010_4135_gb300 import stability
    rng = np.random.default_rng(12)
    states = [(rng.uniform(0.3, 3.0), rng.uniform(-3, 3), rng.uniform(-1, 1), rng.uniform(-1, 1),
               rng.uniform(0.5, 4.0)) for _ in range(3)]
    params = []
    for _ in range(5):
        c1 = float(rng.integers(3, 8))
        params.append((c1, 3.0 * c1, 2.0 * c1, GAMMA, float(rng.choice([1e-5, 2e-5, 5e-5])), 5e-5, 1.0 / 128))
    dirs = [(1.0, 0.0, 0.0), (1.0, 1.0, 1.0)]
    nk = 24
    kdx = math.pi * np.arange(1, nk + 1) / nk
    got = stability.max_growth_device(states, params, directions=dirs, nk=nk)
    for p, value in zip(params, got):
        want = max(vonneumann.max_growth(s[0], s[1:4], s[4], p[0], p[1], p[2], p[3], p[4], p[5], p[6], kdx, d)
                   for s in states for d in dirs)
        assert abs(value - want) <= TOL * want, (p, value, want)


def test_parameter_rule_on_the_device_equals_the_host_rule():
    import workloads
    from paper_1010_4135_gb300 import stability
    for req in workloads.serving_trace(seed=5, n=6):
        pre, post, other = workloads.request_states(req)
        states = [pre, post, other, *stability.interaction_states(post, other)]
        dx = 1.0 / req["grid"][1]
        assert stability.choose_parameters(states, dx, device=True) == stability.choose_parameters(states, dx)


def test_invalid_arguments_are_rejected():
    import ctypes

    from paper_1010_4135_gb300 import _abi as A
    p = ctypes.c_void_p(256)
    assert A.lbm_vn_max_growth(p, 0, p, 1, p, 1, 8, 1, p, None) == A.LBM_EINVAL
    assert A.lbm_vn_max_growth(None, 1, p, 1, p, 1, 8, 1, p, None) == A.LBM_EINVAL
    assert A.lbm_vn_max_growth(p, 1, p, 1, p, 1, 0, 1, p, None) == A.LBM_EINVAL


def test_clustered_small_eigenvalues_converge():
    """With dt = tau and a small Courant number, ten eigenvalues of G are
    O(Courant) and clustered near 0 (the equilibrium Jacobian is a rank-5
    projector) and five cluster near 1: the QR iteration still deflates them
    and max |omega| matches the oracle (a deflation test relative only to the
    neighbouring diagonal entries would never split the tiny cluster off)."""
    import workloads
    from paper_1010_4135_gb300 import stability
    grids = ((16, 16, 16), (24, 16, 16), (20, 12, 12), (32, 16, 8))
    nk = 24
    kdx = math.pi * np.arange(1, nk + 1) / nk
    for req in workloads.serving_trace(seed=7, n=4, rate=200.0, grids=grids, steps=(20, 70)):
        pre, post, other = workloads.request_states(req)
        states = [pre, post, other, *stability.interaction_states(post, other)]
        dx = 1.0 / req["grid"][1]
        params = [(3.0, 9.0, 6.0, GAMMA, dt, dt, dx) for dt in (5e-6, 2e-6, 5e-7)]
        got = stability.max_growth_device(states, params, nk=nk)
        for p, value in zip(params, got):
            want = max(vonneumann.max_growth(s[0], s[1:4], s[4], *p[:3], GAMMA, p[4], p[5], p[6], kdx, d)
                       for s in states for d in stability.DIRECTIONS)
            assert np.isfinite(value) and abs(value - want) <= TOL * want, (p, value, want)
