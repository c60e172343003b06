"""ctypes binding of include/lbm.h: the same names, argument marshalling only.

Loading compiles the library from csrc/ when it is missing or stale (nvcc
required); there is no fallback implementation: every step of the solver
runs in the CUDA kernels of liblbm.so.
"""
from __future__ import annotations

import ctypes
import threading

from . import build as _build

LBM_OK, LBM_EINVAL, LBM_ENOMEM, LBM_ECUDA, LBM_ENONFINITE, LBM_ETIMEOUT, LBM_ESTATE = 0, -1, -2, -3, -4, -5, -6
LBM_BC_PERIODIC, LBM_BC_FIXED, LBM_BC_EXTRAPOLATE, LBM_BC_REFLECT, LBM_BC_EXTERNAL = 0, 1, 2, 3, 4
LBM_FP64, LBM_FP32 = 0, 1
LBM_SCHEME_NND, LBM_SCHEME_UPWIND2, LBM_SCHEME_UPWIND1 = 0, 1, 2
LBM_HEALTH_NONFINITE, LBM_HEALTH_RHO, LBM_HEALTH_T, LBM_HEALTH_TIMEOUT = 1, 2, 4, 8
LBM_VARIANT_TILED, LBM_VARIANT_PLAIN, LBM_VARIANT_TILED_SINGLE, LBM_VARIANT_TILED_FILL, LBM_VARIANT_TILED64, \
    LBM_VARIANT_TILED_SPLIT = 0, 1, 2, 3, 4, 5
LBM_KERNEL_FILL, LBM_KERNEL_STEP, LBM_KERNEL_REDUCE, LBM_KERNEL_OTHER, LBM_NKERNEL = 0, 1, 2, 3, 4
KERNEL_NAMES = ("fill", "step", "reduce", "other")
LBM_MAX_BATCH = 48


class lbm_grid(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("nz", ctypes.c_int32),
        ("bc_lo", ctypes.c_int32 * 3), ("bc_hi", ctypes.c_int32 * 3),
        ("fixed_lo", (ctypes.c_double * 5) * 3), ("fixed_hi", (ctypes.c_double * 5) * 3),
    ]


class lbm_vset(ctypes.Structure):
    _fields_ = [("c1", ctypes.c_double), ("c2", ctypes.c_double), ("eta0", ctypes.c_double),
                ("gamma", ctypes.c_double)]


_vp = ctypes.c_void_p
_dp = ctypes.POINTER(ctypes.c_double)

# (name, restype, argtypes) of every entry point declared in include/lbm.h
SIGNATURES = [
    ("lbm_workspace_bytes", ctypes.c_size_t, [ctypes.POINTER(lbm_grid), ctypes.c_int32]),
    ("lbm_create", ctypes.c_int, [ctypes.POINTER(lbm_grid), ctypes.POINTER(lbm_vset), ctypes.c_double,
                                  ctypes.c_double, ctypes.c_double, ctypes.c_int32, _vp, ctypes.c_size_t, _vp,
                                  ctypes.POINTER(_vp)]),
    ("lbm_set_scheme", ctypes.c_int, [_vp, ctypes.c_int32, ctypes.c_int32]),
    ("lbm_set_launch", ctypes.c_int, [_vp, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32]),
    ("lbm_set_wait_limit", ctypes.c_int, [_vp, ctypes.c_uint32]),
    ("lbm_set_t_recovery", ctypes.c_int, [_vp, ctypes.c_double]),
    ("lbm_init", ctypes.c_int, [_vp, _vp, _vp, _vp, ctypes.c_int32]),
    ("lbm_step", ctypes.c_int, [_vp, ctypes.c_int64]),
    ("lbm_step_batch", ctypes.c_int, [ctypes.POINTER(_vp), ctypes.c_int32, ctypes.c_int64]),
    ("lbm_graph_capture", ctypes.c_int, [ctypes.POINTER(_vp), ctypes.c_int32, ctypes.c_int64, ctypes.POINTER(_vp)]),
    ("lbm_graph_launch", ctypes.c_int, [_vp]),
    ("lbm_graph_destroy", None, [_vp]),
    ("lbm_moments", ctypes.c_int, [_vp, _vp, _vp, _vp, ctypes.c_int32]),
    ("lbm_moments_async", ctypes.c_int, [_vp, _vp, _vp, _vp]),
    ("lbm_health_async", ctypes.c_int, [_vp, _vp]),
    ("lbm_get_f", ctypes.c_int, [_vp, _vp, ctypes.c_int32]),
    ("lbm_set_f", ctypes.c_int, [_vp, _vp, ctypes.c_int32]),
    ("lbm_conserved", ctypes.c_int, [_vp, _dp]),
    ("lbm_conserved_noalloc", ctypes.c_int, [_vp, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                             ctypes.POINTER(lbm_vset), _vp, ctypes.c_int32, _vp]),
    ("lbm_get_halo_source", ctypes.c_int, [_vp, ctypes.c_int32, _vp, ctypes.c_int32]),
    ("lbm_set_halo", ctypes.c_int, [_vp, ctypes.c_int32, _vp, ctypes.c_int32]),
    ("lbm_vn_max_growth", ctypes.c_int, [_vp, ctypes.c_int32, _vp, ctypes.c_int32, _vp, ctypes.c_int32,
                                         ctypes.c_int32, ctypes.c_int32, _vp, _vp]),
    ("lbm_reciprocal_fp32", ctypes.c_int, [_vp, _vp, ctypes.c_int64, _vp]),
    ("lbm_health", ctypes.c_int, [_vp, ctypes.POINTER(ctypes.c_uint32)]),
    ("lbm_sync", ctypes.c_int, [_vp]),
    ("lbm_steps_done", ctypes.c_int64, [_vp]),
    ("lbm_set_timing", ctypes.c_int, [_vp, ctypes.c_int32]),
    ("lbm_get_timing", ctypes.c_int, [_vp, _dp, ctypes.POINTER(ctypes.c_int64), ctypes.c_int32]),
    ("lbm_status_str", ctypes.c_char_p, [ctypes.c_int]),
    ("lbm_destroy", None, [_vp]),
]

_lock = threading.Lock()
_lib = None


def lib() -> ctypes.CDLL:
    """The loaded liblbm.so (built on first use)."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.build()
            handle = ctypes.CDLL(path)
            for name, res, args in SIGNATURES:
                fn = getattr(handle, name)
                fn.restype = res
                fn.argtypes = args
            _lib = handle
    return _lib


class LbmError(RuntimeError):
    def __init__(self, status: int, where: str = ""):
        self.status = status
        msg = lib().lbm_status_str(status).decode()
        super().__init__(f"{where}: {msg}" if where else msg)


def check(status: int, where: str = "") -> int:
    if status != LBM_OK:
        raise LbmError(status, where)
    return status


def _forward(name):
    def call(*args):
        return getattr(lib(), name)(*args)
    call.__name__ = name
    call.__doc__ = f"{name} of include/lbm.h"
    return call


lbm_workspace_bytes = _forward("lbm_workspace_bytes")
lbm_create = _forward("lbm_create")
lbm_set_scheme = _forward("lbm_set_scheme")
lbm_set_launch = _forward("lbm_set_launch")
lbm_set_wait_limit = _forward("lbm_set_wait_limit")
lbm_set_t_recovery = _forward("lbm_set_t_recovery")
lbm_init = _forward("lbm_init")
lbm_step = _forward("lbm_step")
lbm_step_batch = _forward("lbm_step_batch")
lbm_graph_capture = _forward("lbm_graph_capture")
lbm_graph_launch = _forward("lbm_graph_launch")
lbm_graph_destroy = _forward("lbm_graph_destroy")
lbm_moments = _forward("lbm_moments")
lbm_moments_async = _forward("lbm_moments_async")
lbm_health_async = _forward("lbm_health_async")
lbm_get_f = _forward("lbm_get_f")
lbm_set_f = _forward("lbm_set_f")
lbm_conserved = _forward("lbm_conserved")
lbm_conserved_noalloc = _forward("lbm_conserved_noalloc")
lbm_get_halo_source = _forward("lbm_get_halo_source")
lbm_set_halo = _forward("lbm_set_halo")
lbm_vn_max_growth = _forward("lbm_vn_max_growth")
lbm_reciprocal_fp32 = _forward("lbm_reciprocal_fp32")
lbm_health = _forward("lbm_health")
lbm_sync = _forward("lbm_sync")
lbm_steps_done = _forward("lbm_steps_done")
lbm_set_timing = _forward("lbm_set_timing")
lbm_get_timing = _forward("lbm_get_timing")
lbm_status_str = _forward("lbm_status_str")
lbm_destroy = _forward("lbm_destroy")


def make_grid(nx, ny, nz, bc_lo=(0, 0, 0), bc_hi=(0, 0, 0), fixed_lo=None, fixed_hi=None) -> lbm_grid:
    g = lbm_grid()
    g.nx, g.ny, g.nz = int(nx), int(ny), int(nz)
    for a in range(3):
        g.bc_lo[a] = int(bc_lo[a])
        g.bc_hi[a] = int(bc_hi[a])
        for k in range(5):
            g.fixed_lo[a][k] = float(fixed_lo[a][k]) if fixed_lo is not None else 0.0
            g.fixed_hi[a][k] = float(fixed_hi[a][k]) if fixed_hi is not None else 0.0
    return g


def make_vset(c1, c2, eta0, gamma=1.4) -> lbm_vset:
    v = lbm_vset()
    v.c1, v.c2, v.eta0, v.gamma = float(c1), float(c2), float(eta0), float(gamma)
    return v
