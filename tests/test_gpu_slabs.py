"""x slabs on the GPU: a grid cut into two or three slab sims on one GPU,
whose cut faces are LBM_BC_EXTERNAL and get their neighbours' columns
through lbm_get_halo_source / lbm_set_halo between steps (the host orders
the copies; no kernel waits on another), advances bitwise as the whole
grid's sim, in FP32 (the default tiled kernel) and FP64, with fixed,
extrapolating, reflecting and periodic x faces."""
import ctypes

import numpy as np
import pytest

from parity_util import case_cfg, initial_f, sim_for

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _slab_sims(cfg, world, precision, f0):
    import dataclasses

    from paper_1010_4135_gb300 import slabs
    plans = [slabs.plan(cfg.nx, cfg.bc_lo, cfg.bc_hi, r, world) for r in range(world)]
    sims = []
    for p in plans:
        c = dataclasses.replace(cfg, nx=p.nx, bc_lo=p.bc_lo, bc_hi=p.bc_hi)
        s = sim_for(c, precision)
        s.set_f(f0[..., p.x0:p.x1])
        sims.append(s)
    return sims, plans


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
@pytest.mark.parametrize("name,world", [("fixed_extrap_reflect_33x17x9", 2), ("fixed_extrap_reflect_33x17x9", 3),
                                        ("reflect_extrap_fixed_20x12x14", 2), ("periodic_37x19x11", 2),
                                        ("wide_70x9x5", 3)])
def test_slabs_equal_the_whole_grid(name, world, precision):
    from paper_1010_4135_gb300 import slabs
    cfg = case_cfg(name)
    f0 = initial_f(cfg, seed=41)
    f0 = f0.astype(np.float32) if precision == "fp32" else f0
    whole = sim_for(cfg, precision)
    whole.set_f(f0)
    whole.step(6)
    sims, plans = _slab_sims(cfg, world, precision, f0)
    slabs.advance_local(sims, plans, 6)
    got = np.concatenate([s.get_f() for s in sims], axis=3)
    assert np.array_equal(got, whole.get_f())
    assert all(s.steps_done == 6 for s in sims)


def test_external_faces_need_their_halo_before_each_step():
    from paper_1010_4135_gb300 import _abi as A
    from paper_1010_4135_gb300 import slabs
    cfg = case_cfg("periodic_37x19x11")
    sims, plans = _slab_sims(cfg, 2, "fp32", initial_f(cfg, seed=3).astype(np.float32))
    s = sims[0]
    assert A.lbm_step(s.handle, 1) == A.LBM_EINVAL  # no halo yet
    slabs.exchange_local(sims, plans)
    assert A.lbm_step(s.handle, 2) == A.LBM_EINVAL  # one step per exchange
    assert A.lbm_step(s.handle, 1) == A.LBM_OK
    assert A.lbm_step(s.handle, 1) == A.LBM_EINVAL  # the halo was used up
    # a face that is not EXTERNAL takes no halo; EXTERNAL is an x-face kind only
    whole = sim_for(case_cfg("fixed_extrap_reflect_33x17x9"), "fp32")
    buf = np.zeros((15, 9, 17, 2), dtype=np.float32)
    assert A.lbm_set_halo(whole.handle, 0, ctypes.c_void_p(buf.ctypes.data), 0) == A.LBM_EINVAL
    g = A.make_grid(8, 8, 8, (0, 4, 0), (0, 4, 0))
    assert A.lbm_workspace_bytes(ctypes.byref(g), A.LBM_FP32) == 0
    # slab sims are not batched or captured
    sp = (ctypes.c_void_p * 2)(sims[0].handle, sims[1].handle)
    assert A.lbm_step_batch(sp, 2, 1) == A.LBM_EINVAL


def test_host_halo_paths_match_device_paths():
    from paper_1010_4135_gb300 import slabs
    cfg = case_cfg("fixed_extrap_reflect_33x17x9")
    f0 = initial_f(cfg, seed=5).astype(np.float32)
    a, pa = _slab_sims(cfg, 2, "fp32", f0)
    b, pb = _slab_sims(cfg, 2, "fp32", f0)
    slabs.advance_local(a, pa, 3)
    for _ in range(3):  # the same exchange through host arrays
        src = [(s.halo_source(0).cpu().numpy() if p.left is not None else None,
                s.halo_source(1).cpu().numpy() if p.right is not None else None) for s, p in zip(b, pb)]
        for s, p in zip(b, pb):
            if p.left is not None:
                s.set_halo(0, src[p.left][1])
            if p.right is not None:
                s.set_halo(1, src[p.right][0])
        for s in b:
            s.step(1)
    for x, y in zip(a, b):
        assert np.array_equal(x.get_f(), y.get_f())
