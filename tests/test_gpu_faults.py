"""Failure detection and checkpoint / resume on the GPU, without faulting it.

* A bounded device wait that runs out: the step kernel's copy-barrier wait
  is given a limit of zero polls, so it gives up at once; the kernel drains
  its copies in flight, sets the timeout bit, and the host reads
  LBM_ETIMEOUT.  The device stays usable: the same sim then runs normally.
* Non-physical states raise the health flag (negative temperature, and an
  unstable time step that drives the state non-finite).
* Checkpoint / resume through get_f / set_f is bitwise identical to an
  uninterrupted run (the kernels are deterministic).
"""
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


@pytest.mark.parametrize("variant", ["tiled", "tiled64", "split"])
def test_wait_that_runs_out_reports_timeout_and_device_stays_usable(variant):
    from paper_1010_4135_gb300 import _abi as A
    cfg = case_cfg("periodic_37x19x11")
    f0 = initial_f(cfg, seed=70).astype(np.float32)
    s = sim_for(cfg, "fp32")
    s.set_launch(variant)
    s.set_f(f0)
    A.check(A.lbm_set_wait_limit(s.handle, 0), "lbm_set_wait_limit")
    s.step(1)
    flags = ctypes.c_uint32(0)
    assert A.lbm_health(s.handle, ctypes.byref(flags)) == A.LBM_ETIMEOUT
    assert flags.value & A.LBM_HEALTH_TIMEOUT
    # the context is intact: restore the limit, reload the state, run again
    A.check(A.lbm_set_wait_limit(s.handle, 1 << 22), "lbm_set_wait_limit")
    s.set_f(f0)
    s.step(3)
    assert s.health() == 0
    ref = sim_for(cfg, "fp32")
    ref.set_launch(variant)
    ref.set_f(f0)
    ref.step(3)
    assert np.array_equal(s.get_f(), ref.get_f())


def test_unstable_time_step_raises_the_health_flag():
    from paper_1010_4135_gb300 import _abi as A
    cfg = case_cfg("periodic_37x19x11", dt=5e-2, tau=5e-2)  # Courant numbers far above 1
    s = sim_for(cfg, "fp32")
    s.set_f(initial_f(cfg, seed=71).astype(np.float32))
    s.step(200)
    flags = s.health()
    assert flags & (A.LBM_HEALTH_NONFINITE | A.LBM_HEALTH_RHO | A.LBM_HEALTH_T)


@pytest.mark.parametrize("precision,variant", [("fp32", "tiled"), ("fp32", "tiled_fill"), ("fp64", "plain")])
def test_checkpoint_resume_is_bitwise(precision, variant):
    cfg = case_cfg("fixed_extrap_reflect_33x17x9")
    f0 = initial_f(cfg, seed=72)
    if precision == "fp32":
        f0 = f0.astype(np.float32)
    a = sim_for(cfg, precision)
    if precision == "fp32":
        a.set_launch(variant)
    a.set_f(f0)
    a.step(14)
    b = sim_for(cfg, precision)
    if precision == "fp32":
        b.set_launch(variant)
    b.set_f(f0)
    b.step(6)
    ck = b.get_f()
    b.close()
    c = sim_for(cfg, precision)
    if precision == "fp32":
        c.set_launch(variant)
    c.set_f(ck)
    c.step(8)
    assert np.array_equal(a.get_f(), c.get_f())


def test_stream_ordered_moments_and_health_match_the_synchronising_calls():
    """lbm_moments_async / lbm_health_async queue their work behind the steps
    without synchronising; after an event they equal lbm_moments / lbm_health."""
    import torch
    from paper_1010_4135_gb300 import _abi as A
    cfg = case_cfg("fixed_extrap_reflect_33x17x9")
    s = sim_for(cfg, "fp32")
    s.set_f(initial_f(cfg, seed=73).astype(np.float32))
    s.step(5)
    nz, ny, nx = s.shape
    rho = torch.empty((nz, ny, nx), dtype=torch.float64, device="cuda")
    u = torch.empty((3, nz, ny, nx), dtype=torch.float64, device="cuda")
    T = torch.empty((nz, ny, nx), dtype=torch.float64, device="cuda")
    flags = torch.full((1,), 77, dtype=torch.int32, pin_memory=True)
    A.check(A.lbm_moments_async(s.handle, ctypes.c_void_p(rho.data_ptr()), ctypes.c_void_p(u.data_ptr()),
                                ctypes.c_void_p(T.data_ptr())), "lbm_moments_async")
    A.check(A.lbm_health_async(s.handle, ctypes.c_void_p(flags.data_ptr())), "lbm_health_async")
    ev = torch.cuda.Event()
    ev.record(s.stream)
    ev.synchronize()
    r2, u2, T2 = s.moments()
    assert np.array_equal(rho.cpu().numpy(), r2) and np.array_equal(u.cpu().numpy(), u2)
    assert np.array_equal(T.cpu().numpy(), T2)
    assert int(flags[0]) == s.health() == 0
    assert A.lbm_moments_async(s.handle, None, None, None) == A.LBM_EINVAL
    assert A.lbm_health_async(s.handle, None) == A.LBM_EINVAL
