"""Batched stepping of uneven grids in one persistent launch, and CUDA-graph
replay: every grid's result must be bitwise the one it gets stepped alone."""
import numpy as np
import pytest

import oracle
import workloads
from parity_util import NTHREADS, case_cfg, field_errors, initial_f, sim_for

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


MIX = ["periodic_37x19x11", "fixed_extrap_reflect_33x17x9", "reflect_extrap_fixed_20x12x14", "wide_70x9x5",
       "column_1x5x3", "single_cell_1x1x1"]


def _mix_sims(seed):
    cfgs = [case_cfg(n) for n in MIX]
    f0s = [initial_f(c, seed=seed + k).astype(np.float32) for k, c in enumerate(cfgs)]
    sims = []
    for c, f0 in zip(cfgs, f0s):
        s = sim_for(c, "fp32")
        s.set_f(f0)
        sims.append(s)
    return cfgs, f0s, sims


@pytest.mark.parametrize("variant,zchunk,ztail", [("tiled", 0, 0), ("tiled", 5, 2), ("tiled", 3, 1),
                                                  ("tiled64", 0, 0), ("tiled64", 4, 3), ("split", 0, 0),
                                                  ("split", 5, 2)])
def test_batch_results_equal_alone(variant, zchunk, ztail):
    """Batched (any tile shape and chunking) equals each grid stepped alone
    with the default launch: bitwise."""
    from paper_1010_4135_gb300 import sim as S
    cfgs, f0s, sims = _mix_sims(40)
    for s in sims:
        s.set_launch(variant, zchunk, ztail)
    S.step_batch(sims, 7)
    for c, f0, s in zip(cfgs, f0s, sims):
        alone = sim_for(c, "fp32")
        alone.set_f(f0)
        alone.step(7)
        assert np.array_equal(s.get_f(), alone.get_f()), c
        assert s.steps_done == 7


def test_batch_matches_oracle():
    from paper_1010_4135_gb300 import sim as S
    cfgs, f0s, sims = _mix_sims(50)
    S.step_batch(sims, 5)
    for c, f0, s in zip(cfgs, f0s, sims):
        ref = oracle.run(c, f0.astype(np.float64), 5, NTHREADS)
        assert field_errors(s.get_f(), ref).max() <= 5e-5


def test_batch_of_3d_workloads_with_different_mach_numbers():
    """Grids of the shock-bubble family with seeded Mach numbers, stepped in
    one launch: each equals its own run."""
    from paper_1010_4135_gb300 import sim as S
    machs = workloads.batch_machs(4, 3)
    ws = [workloads.shock_bubble(40, 24, 24, mach=float(mm)) for mm in machs]
    sims, f0s = [], []
    for w in ws:
        s = S.from_workload(w, precision="fp32")
        rho, u, T = w.initial_fields()
        s.init(rho, u, T)
        f0s.append(s.get_f())
        sims.append(s)
    S.step_batch(sims, 6)
    for w, f0, s in zip(ws, f0s, sims):
        a = S.from_workload(w, precision="fp32")
        a.set_f(f0)
        a.step(6)
        assert np.array_equal(a.get_f(), s.get_f())


@pytest.mark.parametrize("batch", [False, True])
def test_graph_replay_equals_stepping(batch):
    from paper_1010_4135_gb300 import sim as S
    cfgs, f0s, sims = _mix_sims(60)
    if not batch:
        cfgs, f0s, sims = cfgs[:1], f0s[:1], sims[:1]
    g = S.Graph(sims, 4)
    g.launch(3)
    for c, f0, s in zip(cfgs, f0s, sims):
        a = sim_for(c, "fp32")
        a.set_f(f0)
        a.step(12)
        assert s.steps_done == 12
        assert np.array_equal(s.get_f(), a.get_f())
    g.close()


def test_graph_of_the_fp64_plain_path():
    from paper_1010_4135_gb300 import sim as S
    c = case_cfg("fixed_extrap_reflect_33x17x9")
    f0 = initial_f(c, seed=3)
    s = sim_for(c, "fp64")
    s.set_f(f0)
    g = S.Graph([s], 2)
    g.launch(5)
    a = sim_for(c, "fp64")
    a.set_f(f0)
    a.step(10)
    assert np.array_equal(s.get_f(), a.get_f())


def test_batch_and_graph_argument_checks():
    from paper_1010_4135_gb300 import _abi as A
    from paper_1010_4135_gb300 import sim as S
    c = case_cfg("wide_70x9x5")
    s32 = sim_for(c, "fp32")
    s64 = sim_for(c, "fp64")
    with pytest.raises(A.LbmError):
        S.step_batch([s32, s64], 1)       # mixed precision
    with pytest.raises(A.LbmError):
        S.step_batch([s32, s32], 1)       # the same sim twice
    with pytest.raises(A.LbmError):
        S.Graph([s32], 3)                 # odd step count
    s32.set_f(initial_f(c, seed=1).astype(np.float32))
    g = S.Graph([s32], 2)
    s32.step(1)                           # buffers swapped outside the graph
    with pytest.raises(A.LbmError):
        g.launch()
    # launch configuration: unknown variant, negative z chunk or tail
    for bad in ((99, 0, 0), (A.LBM_VARIANT_TILED, -1, 0), (A.LBM_VARIANT_TILED, 8, -1)):
        assert A.lbm_set_launch(s32.handle, *bad) == A.LBM_EINVAL


def test_full_descriptor_table_and_one_more():
    """LBM_MAX_BATCH (48) grids of mixed small shapes in one launch equal
    their runs alone; a 49th grid is rejected."""
    from paper_1010_4135_gb300 import _abi as A
    from paper_1010_4135_gb300 import sim as S
    names = ["periodic_37x19x11", "fixed_extrap_reflect_33x17x9", "reflect_extrap_fixed_20x12x14", "column_1x5x3"]
    cfgs = [case_cfg(names[k % len(names)]) for k in range(A.LBM_MAX_BATCH + 1)]
    sims, f0s = [], []
    for k, c in enumerate(cfgs):
        s = sim_for(c, "fp32")
        f0 = initial_f(c, seed=200 + k).astype(np.float32)
        s.set_f(f0)
        sims.append(s)
        f0s.append(f0)
    assert A.lbm_step_batch(S._handles(sims), len(sims), 1) == A.LBM_EINVAL
    S.step_batch(sims[:A.LBM_MAX_BATCH], 3)
    for k in (0, 1, 2, 3, A.LBM_MAX_BATCH - 1):
        alone = sim_for(cfgs[k], "fp32")
        alone.set_f(f0s[k])
        alone.step(3)
        assert np.array_equal(sims[k].get_f(), alone.get_f()), k
