"""The product-side von Neumann helper (parameter choice for served runs)
against the oracle's independent construction of the paper's G (Sec. 3)."""
import math

import numpy as np
import pytest

import workloads
from oracle import riemann
from oracle import vonneumann as vn
from paper_1010_4135_gb300 import stability as S


@pytest.mark.parametrize("seed", range(6))
def test_chain_rule_jacobian_matches_complex_step(seed):
    rng = np.random.default_rng(seed)
    rho, u, T = rng.uniform(0.2, 5.0), rng.uniform(-2.0, 2.0, 3), rng.uniform(0.2, 5.0)
    c1 = rng.uniform(1.0, 5.0)
    c2, eta0, gamma = 3.0 * c1, rng.uniform(1.0, 2.0) * c1, rng.choice([1.4, 5.0 / 3.0])
    a = S.equilibrium_jacobian(rho, u, T, c1, c2, eta0, gamma)
    b = vn.feq_jacobian(rho, u, T, c1, c2, eta0, gamma)
    assert np.max(np.abs(a - b)) <= 1e-12 * max(1.0, np.abs(b).max())


@pytest.mark.parametrize("k", [(0.3, 0.0, 0.0), (0.0, 1.7, 0.0), (0.9, -0.4, 2.2)])
@pytest.mark.parametrize("diss", [True, False])
def test_amplification_matrix_matches_oracle(k, diss):
    args = (1.1, [0.5, -0.2, 0.1], 0.9, 2.0, 6.0, 3.0, 1.4, 3e-4, 7e-4, 0.01)
    kv = np.asarray(k) / 0.01
    a = S.amplification(*args, kv, dissipation=diss)
    b = vn.amplification_matrix(*args, kv, dissipation=diss)
    assert np.max(np.abs(a - b)) <= 1e-12


def test_choose_parameters_gives_a_stable_step_and_rejects_a_larger_one():
    r2, u2, p2, _ = workloads.rankine_hugoniot(3.0)
    states = [(1.0, 0.0, 0.0, 0.0, 1.0), (r2, u2, 0.0, 0.0, p2 / r2), (0.1, 0.0, 0.0, 0.0, 10.0)]
    dx = 1.0 / 64
    c1, c2, eta0, dt = S.choose_parameters(states, dx)
    assert c1 >= u2 and c2 == 3 * c1 and eta0 == 2 * c1 and dt is not None
    assert S.max_growth(states, c1, c2, eta0, 1.4, dt, dt, dx, nk=24) <= 1.0 + 1e-3
    assert S.courant(c2, dt, dx) <= S.COURANT_MAX
    bigger = [d for d in S.DT_CANDIDATES if d > dt]
    for d in bigger:
        assert (S.max_growth(states, c1, c2, eta0, 1.4, d, d, dx, nk=24) > 1.0 + 1e-3
                or S.courant(c2, d, dx) > S.COURANT_MAX)
    # no smaller c1 of the rule's ladder has a stable candidate step
    for c in range(2, int(c1)):
        if c < u2:
            continue
        assert all(S.max_growth(states, c, 3 * c, 2 * c, 1.4, d, d, dx, nk=24) > 1.0 + 1e-3
                   or S.courant(3 * c, d, dx) > S.COURANT_MAX for d in S.DT_CANDIDATES)


def test_dissipation_term_lowers_growth_at_fig3_parameters():
    st = [(1.0, 20.0, 0.0, 0.0, 1.0)]
    no = S.max_growth(st, 20.0, 60.0, 20.0, 1.4, 1e-5, 1e-5, 4e-3, directions=((1, 0, 0),), dissipation=False)
    yes = S.max_growth(st, 20.0, 60.0, 20.0, 1.4, 1e-5, 1e-5, 4e-3, directions=((1, 0, 0),))
    assert yes < no and yes <= 1.0 + 1e-3


@pytest.mark.parametrize("left,right", [
    ((1.0, 0.0, 0.0, 0.0, 1.0), (0.125, 0.0, 0.0, 0.0, 0.8)),      # Sod: shock + rarefaction
    ((0.445, 0.698, 0.0, 0.0, 3.528 / 0.445), (0.5, 0.0, 0.0, 0.0, 0.571 / 0.5)),  # Lax
    ((1.0, -2.0, 0.0, 0.0, 0.4), (1.0, 2.0, 0.0, 0.0, 0.4)),        # two rarefactions
    ((1.0, 3.0, 0.0, 0.0, 1.0), (1.0, -3.0, 0.0, 0.0, 1.0)),        # two shocks
])
def test_interaction_states_match_the_exact_riemann_solver(left, right):
    a, b = S.interaction_states(left, right)
    st = riemann.star_state((left[0], left[1], left[0] * left[4]), (right[0], right[1], right[0] * right[4]))
    assert a[1] == pytest.approx(st.u, rel=1e-10, abs=1e-12) and b[1] == a[1]
    assert a[0] == pytest.approx(st.rho_l, rel=1e-10) and b[0] == pytest.approx(st.rho_r, rel=1e-10)
    assert a[0] * a[4] == pytest.approx(st.p, rel=1e-10) and b[0] * b[4] == pytest.approx(st.p, rel=1e-10)


def test_parameter_rule_sees_the_flow_behind_a_shocked_light_bubble():
    """A Mach 5.74 shock into gas ten times lighter: the star velocity (8.25)
    exceeds the post-shock speed (5.49), and c1 follows it."""
    r2, u2, p2, _ = workloads.rankine_hugoniot(5.74)
    post, bubble = (r2, u2, 0.0, 0.0, p2 / r2), (0.1, 0.0, 0.0, 0.0, 10.0)
    star = S.interaction_states(post, bubble)
    assert star[0][1] > 8.2
    c1, _, _, dt = S.choose_parameters([(1.0, 0.0, 0.0, 0.0, 1.0), post, bubble, *star], 1.0 / 128)
    assert c1 >= star[0][1] and dt is not None


def test_request_parameter_candidates():
    """Attempt 0 is the rule; attempt 1 lowers c1 by one (c2 = 3 c1, eta0 =
    2 c1); attempt 2 keeps c1 and takes eta0 = c1."""
    import workloads as W
    from paper_1010_4135_gb300 import serve
    req = {"id": 0, "grid": (64, 64, 64), "mach": 8.4, "ratio": 0.1, "steps": 10, "kind": "sphere"}
    c1, c2, eta0, dt = serve.request_parameters(req)
    assert (c2, eta0) == (3 * c1, 2 * c1)
    assert serve.request_parameters(req, 1) == (c1 - 1, 3 * (c1 - 1), 2 * (c1 - 1), dt)
    assert serve.request_parameters(req, 2) == (c1, c2, c1, dt)
