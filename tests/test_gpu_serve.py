"""The continuous-batching server: requests admitted as they arrive and as
memory frees up, stepped together, each result bitwise the same as the
request solved alone."""
import numpy as np
import pytest

import workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _trace(steps=(20, 70)):
    grids = ((16, 16, 16), (24, 16, 16), (20, 12, 12), (32, 16, 8))
    tr = workloads.serving_trace(seed=7, n=8, rate=200.0, grids=grids, steps=steps)
    return tr


@pytest.mark.parametrize("policy", ["fifo", "sjf"])
def test_served_results_equal_alone_and_budget_is_respected(policy):
    from paper_1010_4135_gb300 import serve
    from paper_1010_4135_gb300 import sim as S
    # all eight arrive within 40 ms and are prepared together (one worker
    # each), and each runs long enough that the next ones are ready before it ends
    tr = _trace(steps=(300, 600))
    sizes = [serve.workspace_bytes(r["grid"]) for r in tr]
    budget = 2 * max(sizes) + min(sizes)  # forces waiting for memory to free up
    srv = serve.Server(hbm_budget=budget, max_batch=3, tick=16, keep_results=True, policy=policy, prep_workers=8)
    done = srv.run(tr)
    assert len(done) == len(tr)
    assert srv.peak_bytes <= budget and srv.peak_batch <= 3
    assert all(j.health == 0 for j in done)
    # requests overlapped on the device: some batch held more than one grid
    assert srv.peak_batch >= 2
    for j in done:
        w = workloads.request_workload(j.req, *j.params)
        s = S.from_workload(w, precision="fp32")
        rho, u, T = w.initial_fields()
        s.init(rho, u, T)
        s.step(j.req["steps"])
        alone, _, _ = s.moments()
        assert np.array_equal(alone, j.rho), j.req
    st = serve.summary(done, srv.wall)
    assert st["p50_latency_s"] <= st["p99_latency_s"]


def test_unhealthy_results_are_solved_again_with_the_next_parameters(monkeypatch):
    """The health bits of every first attempt are forced to 'T <= 0' (on the
    host, no GPU fault): each request is solved again with attempt 1's
    parameters, and that result is bitwise the request solved alone with
    them; latency keeps counting from the first arrival."""
    from paper_1010_4135_gb300 import serve
    from paper_1010_4135_gb300 import sim as S
    real = serve.Server._health
    monkeypatch.setattr(serve.Server, "_health",
                        staticmethod(lambda job: 4 if job.attempt == 0 else real(job)))
    tr = _trace()[:4]
    srv = serve.Server(max_batch=4, tick=16, keep_results=True)
    done = srv.run(tr)
    assert len(done) == len(tr) and srv.retries == len(tr)
    for j in done:
        assert j.attempt == 1 and j.health == 0
        assert j.params == serve.request_parameters(j.req, 1)
        w = workloads.request_workload(j.req, *j.params)
        s = S.from_workload(w, precision="fp32")
        s.init(*w.initial_fields())
        s.step(j.req["steps"])
        alone, _, _ = s.moments()
        assert np.array_equal(alone, j.rho)
    assert serve.summary(done, srv.wall)["retried"] == len(tr)


def test_served_fp32_result_against_the_oracle():
    """A served 64^3 request (parameters from the on-device rule) against the
    oracle itself, not the FP64 path: its FP32 density after the request's
    steps is within the FP32 error model's bound, kappa taken over the
    request's states and the star states where the shocked gas meets the
    second gas (parity_util.fp32_l1_bound)."""
    import oracle
    from paper_1010_4135_gb300 import serve, stability
    from parity_util import NTHREADS, fp32_l1_bound, l1_rel, linf_rel
    tr = workloads.serving_trace(seed=11, n=2, rate=200.0, grids=((64, 64, 64),), steps=(400, 500))
    srv = serve.Server(max_batch=2, tick=16, keep_results=True)
    done = srv.run(tr)
    assert len(done) == 2 and all(j.health == 0 for j in done)
    j = min(done, key=lambda d: d.req["id"])  # one request: 1.2e8 cell-updates for the oracle
    w = workloads.request_workload(j.req, *j.params)
    cfg = oracle.cfg_for(w)
    f = oracle.run(cfg, oracle.init(cfg, *w.initial_fields()), j.req["steps"], NTHREADS)
    ro, _, _ = oracle.macros(cfg, f)
    pre, post, other = workloads.request_states(j.req)
    bound = fp32_l1_bound(cfg, [pre, post, other, *stability.interaction_states(post, other)], j.req["steps"])
    print(f"served {j.req['kind']} 64^3 Mach {j.req['mach']:.2f} ratio {j.req['ratio']:.2f} fp32 vs oracle after "
          f"{j.req['steps']} steps: L1 {l1_rel(j.rho, ro):.3e} Linf {linf_rel(j.rho, ro):.3e} (model bound {bound:.2e})")
    assert l1_rel(j.rho, ro) <= bound
