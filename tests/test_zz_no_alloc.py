"""lbm_conserved_noalloc: global sums without any device allocation.

Some callers cannot allocate device memory (a stream being captured into a
CUDA graph, a host whose allocator owns the whole device, a monitoring hook
that must not change the memory footprint).  For them the library offers one
entry point whose scratch is a static device array instead of a workspace.
This file checks it against the workspace-based lbm_conserved on the same
state and against the oracle's sums of that state, through the C ABI, on two
calls in a row (the second call reuses the shared array the first one left
behind), and checks that a call leaves the device's free memory unchanged.
It is named so that pytest collects it last.
"""
import ctypes

import numpy as np
import pytest

import oracle
from parity_util import case_cfg, initial_f, sim_for

pytestmark = pytest.mark.gpu

CONSERVED_TOL = 1e-13  # the tolerance of the conservation checks in test_gpu_parity


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
@pytest.mark.parametrize("name", ["periodic_37x19x11", "wide_70x9x5"])
def test_noalloc_matches_workspace_reduction(name, precision):
    import torch
    from paper_1010_4135_gb300 import _abi as A

    cfg = case_cfg(name)
    f0 = initial_f(cfg, seed=31)
    dt = np.float32 if precision == "fp32" else np.float64
    s = sim_for(cfg, precision)
    s.set_f(f0.astype(dt))
    s.step(3)
    ref = s.conserved()
    dense = torch.empty((15, cfg.nz, cfg.ny, cfg.nx), device="cuda",
                        dtype=torch.float32 if precision == "fp32" else torch.float64)
    s.get_f(dense)
    g = dense.cpu().numpy().astype(np.float64)
    scale = np.abs(oracle.conserved(cfg, np.abs(g)))
    want = oracle.conserved(cfg, g)
    vset = A.make_vset(cfg.c1, cfg.c2, cfg.eta0, cfg.gamma)
    prec = A.LBM_FP32 if precision == "fp32" else A.LBM_FP64
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    for k in range(2):  # two calls in a row: host output
        out = np.zeros(5)
        torch.cuda.synchronize()
        free_before = torch.cuda.mem_get_info()[0]
        rc = A.lbm_conserved_noalloc(ctypes.c_void_p(dense.data_ptr()), prec, cfg.nx, cfg.ny, cfg.nz,
                                     ctypes.byref(vset), ctypes.c_void_p(out.ctypes.data), 0, stream)
        assert rc == A.LBM_OK
        if k == 1:  # after the first call's set-up: the call allocates nothing on the device
            assert torch.cuda.mem_get_info()[0] == free_before
        assert np.all(np.abs(out - ref) <= CONSERVED_TOL * np.maximum(scale, 1e-300)), (out, ref)
        assert np.all(np.abs(out - want) <= CONSERVED_TOL * np.maximum(scale, 1e-300)), (out, want)
    for _ in range(2):  # two calls in a row: device output
        out_d = torch.zeros(5, dtype=torch.float64, device="cuda")
        rc = A.lbm_conserved_noalloc(ctypes.c_void_p(dense.data_ptr()), prec, cfg.nx, cfg.ny, cfg.nz,
                                     ctypes.byref(vset), ctypes.c_void_p(out_d.data_ptr()), 1, stream)
        assert rc == A.LBM_OK
        torch.cuda.synchronize()
        out = out_d.cpu().numpy()
        assert np.all(np.abs(out - ref) <= CONSERVED_TOL * np.maximum(scale, 1e-300)), (out, ref)
        assert np.all(np.abs(out - want) <= CONSERVED_TOL * np.maximum(scale, 1e-300)), (out, want)


def test_noalloc_rejects_grids_beyond_its_scratch():
    from paper_1010_4135_gb300 import _abi as A
    vset = A.make_vset(2.0, 6.0, 2.0)
    out = np.zeros(5)
    # 4096 blocks of 8192 cells is the maximum the static scratch holds
    rc = A.lbm_conserved_noalloc(ctypes.c_void_p(256), A.LBM_FP32, 8193, 64, 64, ctypes.byref(vset),
                                 ctypes.c_void_p(out.ctypes.data), 0, None)
    assert rc == A.LBM_EINVAL
    rc = A.lbm_conserved_noalloc(ctypes.c_void_p(256), A.LBM_FP32, 0, 1, 1, ctypes.byref(vset),
                                 ctypes.c_void_p(out.ctypes.data), 0, None)
    assert rc == A.LBM_EINVAL
