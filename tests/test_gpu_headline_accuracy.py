"""Stated FP32 density errors of the benchmarked workloads.

* The 256^3 Mach-2 shock-droplet (rho = 5 droplet, (c1, c2, eta0) = (2, 6, 4),
  dt = tau = 5e-5) over its 2000 steps, in the default launch.
* The batched 512x256x256 Mach-3 shock-bubble with eight 128^3 bubbles of
  seeded Mach numbers in [1.5, 6], advanced by one batched launch per step
  replayed from a CUDA graph, over 1000 steps.

The reference is the FP64 path, stepped alone: it equals the oracle to 1e-12
on every parity case and on one full-size step of both grids at sampled
nodes (test_gpu_fullsize).  The oracle itself would need about 1.4 hours of
host time for the droplet's 3.4e10 cell-updates.  Bounds: the FP32 error
model of parity_util.fp32_l1_bound over each grid's states (initial states
and, for the batch, the star states of the shock meeting the bubble).
"""
import numpy as np
import pytest

import oracle
import workloads
from parity_util import fp32_l1_bound, l1_rel, linf_rel

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _rho_after(w, precision, steps):
    from paper_1010_4135_gb300 import sim as S
    s = S.from_workload(w, precision=precision)
    rho, u, T = w.initial_fields()
    s.init(rho, u, T)
    s.step(steps)
    assert s.health() == 0
    r, _, _ = s.moments()
    s.close()
    return r


def test_shock_droplet_256_fp32_error_over_2000_steps():
    w = workloads.shock_droplet(256)
    r32 = _rho_after(w, "fp32", w.steps)
    r64 = _rho_after(w, "fp64", w.steps)
    bound = fp32_l1_bound(oracle.cfg_for(w), (w.meta["ambient"], w.meta["sphere"], w.meta["post"]), w.steps)
    print(f"shock_droplet_256^3 fp32 vs fp64 after {w.steps} steps: L1 {l1_rel(r32, r64):.3e} "
          f"Linf {linf_rel(r32, r64):.3e} (model bound {bound:.2e})")
    assert l1_rel(r32, r64) <= bound


def test_batched_bubbles_fp32_error_over_1000_steps():
    import bench
    from paper_1010_4135_gb300 import sim as S
    from paper_1010_4135_gb300 import stability
    steps = 1000
    ws = bench.batch_workloads()
    sims = []
    for w in ws:
        s = S.from_workload(w, precision="fp32")
        rho, u, T = w.initial_fields()
        s.init(rho, u, T)
        sims.append(s)
    g = S.Graph(sims, 10)
    g.launch(steps // 10)
    for w, s in zip(ws, sims):
        assert s.steps_done == steps and s.health() == 0
        r32, _, _ = s.moments()
        s.close()
        r64 = _rho_after(w, "fp64", steps)
        post, bubble = w.meta["post"], w.meta["sphere"]
        states = (w.meta["ambient"], post, bubble, *stability.interaction_states(post, bubble))
        bound = fp32_l1_bound(oracle.cfg_for(w), states, steps)
        print(f"{w.name} fp32 (batched) vs fp64 after {steps} steps: L1 {l1_rel(r32, r64):.3e} "
              f"Linf {linf_rel(r32, r64):.3e} (model bound {bound:.2e})")
        assert l1_rel(r32, r64) <= bound
