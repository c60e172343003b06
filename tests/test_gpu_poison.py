"""Cells no update may read stay unread: the workspace starts as NaN (every
byte 0xFF), so the edges and corners of the ghost layers (never written:
the stencil is an axis-aligned star), the row padding and the halo columns
beyond the two a step needs hold NaN.  Any read of them would spread NaN
into the interior; the results must equal a run on a zeroed workspace."""
import numpy as np
import pytest

from parity_util import CASES, case_cfg, initial_f, sim_for

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _sim(cfg, precision, fill):
    import torch
    from paper_1010_4135_gb300 import sim as S
    probe = sim_for(cfg, precision)
    ws = torch.full((probe.workspace_bytes,), fill, dtype=torch.uint8, device="cuda")
    probe.close()
    scheme = {0: "nnd", 1: "upwind2", 2: "upwind1"}[cfg.scheme]
    return S.Sim(cfg.nx, cfg.ny, cfg.nz, cfg.c1, cfg.c2, cfg.eta0, cfg.tau, cfg.dt, cfg.dx, gamma=cfg.gamma,
                 precision=precision, bc_lo=cfg.bc_lo, bc_hi=cfg.bc_hi, fixed_lo=cfg.fixed_lo,
                 fixed_hi=cfg.fixed_hi, scheme=scheme, workspace=ws)


@pytest.mark.parametrize("precision,variant", [("fp32", "tiled"), ("fp32", "tiled64"), ("fp32", "split"), ("fp32", "tiled_fill"),
                                               ("fp32", "tiled_single"), ("fp32", "plain"), ("fp64", "plain")])
@pytest.mark.parametrize("name", sorted(CASES))
def test_unread_layers_poisoned_with_nan_do_not_matter(name, precision, variant):
    cfg = case_cfg(name)
    f0 = initial_f(cfg, seed=60)
    if precision == "fp32":
        f0 = f0.astype(np.float32)
    out = []
    for fill in (0xFF, 0x00):
        s = _sim(cfg, precision, fill)
        if precision == "fp32":
            s.set_launch(variant)
        s.set_f(f0)
        s.step(6)
        out.append(s.get_f())
        assert s.health() == 0
    assert np.isfinite(out[0]).all()
    assert np.array_equal(out[0], out[1])


def test_batched_step_on_poisoned_workspaces():
    from paper_1010_4135_gb300 import sim as S
    names = ("periodic_37x19x11", "fixed_extrap_reflect_33x17x9", "reflect_extrap_fixed_20x12x14")
    res = {}
    for fill in (0xFF, 0x00):
        sims = []
        for k, name in enumerate(names):
            cfg = case_cfg(name)
            s = _sim(cfg, "fp32", fill)
            s.set_f(initial_f(cfg, seed=61 + k).astype(np.float32))
            sims.append(s)
        S.step_batch(sims, 5)
        res[fill] = [s.get_f() for s in sims]
    for a, b in zip(res[0xFF], res[0x00]):
        assert np.isfinite(a).all() and np.array_equal(a, b)
