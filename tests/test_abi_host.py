"""The C-ABI library builds, loads and exports every entry point that
include/lbm.h declares; host-side argument validation works without a GPU
(no compute call is made here)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = []
    for fn in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if fn.endswith(".h"):
            with open(os.path.join(ROOT, "include", fn)) as fh:
                text = fh.read()
            names += re.findall(r"LBM_API\s+[\w\s\*]*?\b(lbm_\w+)\s*\(", text)
    return names


@pytest.fixture(scope="module")
def A():
    from paper_1010_4135_gb300 import _abi
    _abi.lib()
    return _abi


def test_every_declared_symbol_is_exported_and_bound(A):
    names = _declared()
    assert len(names) >= 14
    bound = {n for n, _, _ in A.SIGNATURES}
    for n in names:
        assert hasattr(A.lib(), n), n
        assert n in bound, n


def test_library_is_the_in_tree_build(A):
    path = A.lib()._name
    assert os.path.abspath(path).startswith(os.path.join(ROOT, "paper_1010_4135_gb300", "_build"))


def _grid(A, nx=10, ny=4, nz=3, lo=(0, 0, 0), hi=(0, 0, 0)):
    return A.make_grid(nx, ny, nz, lo, hi)


def test_largest_field_below_2_32_cells_is_accepted(A):
    # rows of 2038 cells pad to 2048 (8 + 2038 + 2), 2044 rows to 2048, 1020 planes to 1024:
    # 2^32 cells, the first field refused; 1019 planes (1023 padded) fit
    assert A.lbm_workspace_bytes(ctypes.byref(_grid(A, 2038, 2044, 1019)), A.LBM_FP32) > 0


def test_workspace_bytes(A):
    small = A.lbm_workspace_bytes(ctypes.byref(_grid(A, 10, 4, 3)), A.LBM_FP64)
    big = A.lbm_workspace_bytes(ctypes.byref(_grid(A, 64, 64, 64)), A.LBM_FP64)
    f32 = A.lbm_workspace_bytes(ctypes.byref(_grid(A, 64, 64, 64)), A.LBM_FP32)
    assert 0 < small < big
    assert f32 < big
    # two padded f buffers of 15 fields at least
    assert big >= 2 * 15 * 64 ** 3 * 8
    assert f32 >= 2 * 15 * 64 ** 3 * 4
    assert A.lbm_workspace_bytes(ctypes.byref(_grid(A)), 7) == 0


@pytest.mark.parametrize("kw", [
    dict(nx=0), dict(ny=-1), dict(lo=(0, 0, 0), hi=(1, 0, 0)), dict(lo=(9, 0, 0), hi=(9, 0, 0)),
    dict(nx=1, lo=(2, 0, 0), hi=(2, 0, 0)),
    # a padded field of 2^32 or more cells (the tiled kernels index a field in 32 bits)
    dict(nx=2038, ny=2044, nz=1020),
])
def test_invalid_grids_have_no_workspace(A, kw):
    args = dict(nx=10, ny=4, nz=3, lo=(0, 0, 0), hi=(0, 0, 0))
    args.update(kw)
    assert A.lbm_workspace_bytes(ctypes.byref(_grid(A, **args)), A.LBM_FP64) == 0


def _create(A, grid=None, vset=None, tau=1e-5, dt=1e-5, dx=0.01, prec=0, ws=4096, nbytes=None):
    grid = grid or _grid(A)
    vset = vset or A.make_vset(2.0, 6.0, 2.0)
    if nbytes is None:
        nbytes = A.lbm_workspace_bytes(ctypes.byref(grid), prec)
    h = ctypes.c_void_p()
    rc = A.lbm_create(ctypes.byref(grid), ctypes.byref(vset), tau, dt, dx, prec, ctypes.c_void_p(ws), nbytes, None,
                      ctypes.byref(h))
    return rc, h


@pytest.mark.parametrize("change", [
    dict(vset=(2.0, 2.0, 1.0)), dict(vset=(2.0, 6.0, 0.0)), dict(vset=(2.0, 6.0, 1.0, 1.0)),
    dict(vset=(-2.0, 6.0, 1.0)), dict(tau=0.0), dict(dt=-1.0), dict(dx=0.0), dict(prec=3),
    dict(ws=0), dict(ws=4100), dict(grid=(0, 1, 1)),
])
def test_create_rejects_invalid_arguments(A, change):
    kw = {}
    if "vset" in change:
        kw["vset"] = A.make_vset(*change["vset"])
    if "grid" in change:
        kw["grid"] = A.make_grid(*change["grid"])
    for k in ("tau", "dt", "dx", "prec", "ws"):
        if k in change:
            kw[k] = change[k]
    if "grid" in change:
        kw["nbytes"] = 1 << 30
    rc, h = _create(A, **kw)
    assert rc == A.LBM_EINVAL and not h.value


def test_create_rejects_small_workspace(A):
    g = _grid(A)
    need = A.lbm_workspace_bytes(ctypes.byref(g), 0)
    rc, h = _create(A, grid=g, nbytes=need - 1)
    assert rc == A.LBM_ENOMEM and not h.value


def test_null_handles_and_status_strings(A):
    assert A.lbm_step(None, 1) == A.LBM_EINVAL
    assert A.lbm_sync(None) == A.LBM_EINVAL
    assert A.lbm_steps_done(None) == -1
    A.lbm_destroy(None)
    for code in range(0, -7, -1):
        assert A.lbm_status_str(code).startswith(b"LBM_")
    assert b"unknown" in A.lbm_status_str(42)


def test_no_cpu_fallback_without_a_device(monkeypatch):
    """The product path refuses to run without a CUDA device instead of
    falling back to anything on the host."""
    import torch
    from paper_1010_4135_gb300 import sim as S
    monkeypatch.setattr(torch.cuda, "is_available", lambda: False)
    with pytest.raises(RuntimeError, match="CUDA device"):
        S.Sim(8, 8, 8, 2.0, 6.0, 4.0, 1e-4, 1e-4, 0.1, precision="fp32")


def test_build_fails_loudly_without_nvcc(monkeypatch):
    from paper_1010_4135_gb300 import build
    monkeypatch.delenv("NVCC", raising=False)
    monkeypatch.setattr(build.shutil, "which", lambda name: None)
    monkeypatch.setattr(build.os.path, "exists", lambda p: False)
    with pytest.raises(RuntimeError, match="nvcc not found"):
        build.nvcc()


def test_external_faces_are_x_faces_of_two_cells_or_more(A):
    g = A.make_grid(8, 6, 5, (A.LBM_BC_EXTERNAL, 0, 3), (A.LBM_BC_EXTERNAL, 0, 3))
    assert A.lbm_workspace_bytes(ctypes.byref(g), A.LBM_FP32) > 0
    for lo, hi in (((0, A.LBM_BC_EXTERNAL, 0), (0, A.LBM_BC_EXTERNAL, 0)),   # y faces: no
                   ((1, 0, A.LBM_BC_EXTERNAL), (1, 0, 3)),                   # z face: no
                   ((5, 0, 0), (1, 0, 0))):                                   # unknown kind
        assert A.lbm_workspace_bytes(ctypes.byref(A.make_grid(8, 6, 5, lo, hi)), A.LBM_FP32) == 0
    assert A.lbm_workspace_bytes(ctypes.byref(A.make_grid(1, 6, 5, (A.LBM_BC_EXTERNAL, 0, 0), (1, 0, 0))),
                                 A.LBM_FP32) == 0


def test_every_bound_entry_point_has_a_forwarder(A):
    for n, _, _ in A.SIGNATURES:
        assert callable(getattr(A, n, None)), n


def test_diagnostic_entry_points_check_their_arguments_before_any_device_call(A):
    p = ctypes.c_void_p(256)
    assert A.lbm_reciprocal_fp32(None, None, 0, None) == A.LBM_OK      # nothing to do, nothing launched
    assert A.lbm_reciprocal_fp32(p, p, -1, None) == A.LBM_EINVAL
    assert A.lbm_reciprocal_fp32(None, p, 4, None) == A.LBM_EINVAL
    assert A.lbm_reciprocal_fp32(p, None, 4, None) == A.LBM_EINVAL
    assert A.lbm_vn_max_growth(p, 0, p, 1, p, 1, 8, 1, p, None) == A.LBM_EINVAL
    assert A.lbm_vn_max_growth(p, 1, p, 1, p, 1, 8, 1, None, None) == A.LBM_EINVAL
    # 2^31 matrices in one call, more than the 2^30 allowed (every call here is
    # refused before anything reaches a device: the pointers are not real)
    assert A.lbm_vn_max_growth(p, 1 << 11, p, 1 << 10, p, 4, 256, 1, p, None) == A.LBM_EINVAL
