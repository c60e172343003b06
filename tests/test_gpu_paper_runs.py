"""The paper's own runs at the sizes it prints (Sec. 4): the high-Mach tube
of Fig. 7 and the 3D shock-bubble / shock-droplet runs of Figs. 8-10 (the
unprinted domain length, bubble radius and shock position are the readings
in workloads.paper_high_mach_tube / paper_shock_bubble)."""
import numpy as np
import pytest

import oracle
import workloads
from parity_util import NTHREADS, field_errors, fp32_l1_bound, l1_rel, linf_rel

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def test_paper_high_mach_tube():
    """Mach-10 flow into a dense hot gas, (c1, c2, eta0) = (8, 24, 8), dx =
    0.01, to t = 0.25.  FP64 path within 1e-12 of the oracle over 1000 steps;
    the oracle's full run stays physical and within 6% (L1 of rho) of the
    exact Riemann solution (the shocks are smeared over a few cells of 0.01);
    the FP32 path against the oracle itself over all 25,000 steps, within the
    FP32 error model's bound (parity_util.fp32_l1_bound; the cold Mach-10
    stream has kappa_T = 45: 5.9e-3)."""
    from oracle import riemann
    from paper_1010_4135_gb300 import sim as S
    w = workloads.paper_high_mach_tube()
    cfg = oracle.cfg_for(w)
    rho, u, T = w.initial_fields()
    s64 = S.from_workload(w, precision="fp64")
    s64.init(rho, u, T)
    s64.step(1000)
    ref = oracle.run(cfg, oracle.init(cfg, rho, u, T), 1000, NTHREADS)
    assert field_errors(s64.get_f(), ref).max() <= 1e-12
    ref = oracle.run(cfg, ref, w.steps - 1000, NTHREADS)
    s32 = S.from_workload(w, precision="fp32")
    s32.init(rho, u, T)
    s32.step(w.steps)
    assert s32.health() == 0
    r64, _, T64 = oracle.macros(cfg, ref)
    r32, _, _ = s32.moments()
    assert T64.min() > 0
    L, R = workloads.PAPER_HM_LEFT, workloads.PAPER_HM_RIGHT
    exact, _, _ = riemann.cell_averages((L[0], L[1], L[0] * L[4]), (R[0], R[1], R[0] * R[4]),
                                        np.arange(w.nx + 1) * w.dx, 0.5, w.steps * w.dt)
    assert l1_rel(r64[0, 0], exact) < 0.06
    bound = fp32_l1_bound(cfg, (w.meta["left"], w.meta["right"]), w.steps)
    print(f"paper_high_mach_tube fp32 vs oracle after {w.steps} steps: L1 {l1_rel(r32, r64):.3e} "
          f"Linf {linf_rel(r32, r64):.3e} (model bound {bound:.2e}); oracle vs exact L1 {l1_rel(r64[0, 0], exact):.3e}")
    assert l1_rel(r32, r64) <= bound


@pytest.mark.parametrize("kind", ["light", "heavy"])
def test_paper_shock_bubble(kind):
    """300 x 80 x 80, a Mach-2 shock entering from x-hi into a light (0.1358)
    or heavy (4.1538) bubble, reflecting y / z walls, 10,000 steps to t = 0.1
    in FP32: physical throughout; the solution keeps the setup's symmetries
    (mirror in y exactly, y <-> z exchange to rounding, measured 3e-5 of max
    rho); FP32 against the oracle itself over the first 100 steps and
    against the FP64 path (parity-pinned to the oracle) over 2000 steps,
    both within the FP32 error model's bound (parity_util.fp32_l1_bound)."""
    from paper_1010_4135_gb300 import sim as S
    w = workloads.paper_shock_bubble(kind)
    rho, u, T = w.initial_fields()
    cfg = oracle.cfg_for(w)
    states = (w.meta["ambient"], w.meta["sphere"], w.meta["post"])
    # the first 100 steps against the oracle itself (1.9e8 cell-updates on the host)
    s = S.from_workload(w, precision="fp32")
    s.init(rho, u, T)
    s.step(100)
    r100, _, _ = s.moments()
    ro, _, _ = oracle.macros(cfg, oracle.run(cfg, oracle.init(cfg, rho, u, T), 100, NTHREADS))
    print(f"paper_shock_bubble_{kind} fp32 vs oracle after 100 steps: L1 {l1_rel(r100, ro):.3e} "
          f"Linf {linf_rel(r100, ro):.3e} (model bound {fp32_l1_bound(cfg, states, 100):.2e})")
    assert l1_rel(r100, ro) <= fp32_l1_bound(cfg, states, 100)
    s.step(1900)
    r2000, _, _ = s.moments()
    s.step(w.steps - 2000)
    assert s.health() == 0
    r, _, Tf = s.moments()
    assert r.min() > 0 and Tf.min() > 0
    assert np.abs(r - r[:, ::-1, :]).max() <= 1e-6 * r.max()
    assert np.abs(r - r.transpose(1, 0, 2)).max() <= 1e-4 * r.max()
    s64 = S.from_workload(w, precision="fp64")
    s64.init(rho, u, T)
    s64.step(2000)
    r64, _, _ = s64.moments()
    bound = fp32_l1_bound(cfg, states, 2000)
    print(f"paper_shock_bubble_{kind} fp32 vs fp64 path after 2000 steps: L1 {l1_rel(r2000, r64):.3e} "
          f"Linf {linf_rel(r2000, r64):.3e} (model bound {bound:.2e})")
    assert l1_rel(r2000, r64) <= bound
