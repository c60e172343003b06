"""Python-side owner of one solver instance.

PyTorch provides the device workspace (one uint8 tensor) and the CUDA stream;
every computation runs in liblbm.so through the C ABI of include/lbm.h.
"""
from __future__ import annotations

import ctypes

import numpy as np
import torch

from . import _abi as A

PRECISIONS = {"fp64": A.LBM_FP64, "fp32": A.LBM_FP32}
SCHEMES = {"nnd": A.LBM_SCHEME_NND, "upwind2": A.LBM_SCHEME_UPWIND2, "upwind1": A.LBM_SCHEME_UPWIND1}


def _ptr(t) -> ctypes.c_void_p:
    return ctypes.c_void_p(t.data_ptr() if isinstance(t, torch.Tensor) else t.ctypes.data)


class Sim:
    """One D3V15 FD-LB grid on one GPU.

    grid: (nx, ny, nz); bc_lo / bc_hi: boundary kinds per axis (LBM_BC_*);
    fixed_lo / fixed_hi: (rho,u1,u2,u3,T) per axis for FIXED faces;
    c1, c2, eta0, gamma: the discrete-velocity constants; tau, dt, dx.
    """

    def __init__(self, nx, ny, nz, c1, c2, eta0, tau, dt, dx, gamma=1.4, precision="fp64",
                 bc_lo=(0, 0, 0), bc_hi=(0, 0, 0), fixed_lo=None, fixed_hi=None, scheme="nnd",
                 dissipation=True, device=None, stream=None, workspace=None):
        if not torch.cuda.is_available():
            raise RuntimeError("paper_1010_4135_gb300.Sim needs a CUDA device (GB300)")
        # constructor arguments, for clone() (the launch configuration is set separately)
        self._config = dict(nx=nx, ny=ny, nz=nz, c1=c1, c2=c2, eta0=eta0, tau=tau, dt=dt, dx=dx, gamma=gamma,
                            precision=precision, bc_lo=bc_lo, bc_hi=bc_hi, fixed_lo=fixed_lo, fixed_hi=fixed_hi,
                            scheme=scheme, dissipation=dissipation, device=device)
        self.launch = ("tiled", 0, 0)  # (variant, zchunk, ztail)
        self.shape = (int(nz), int(ny), int(nx))
        self.prec = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
        self.dtype = np.float64 if self.prec == A.LBM_FP64 else np.float32
        self.device = torch.device("cuda", torch.cuda.current_device() if device is None else
                                   torch.device(device).index or 0)
        self._grid = A.make_grid(nx, ny, nz, bc_lo, bc_hi, fixed_lo, fixed_hi)
        self._vset = A.make_vset(c1, c2, eta0, gamma)
        nbytes = A.lbm_workspace_bytes(ctypes.byref(self._grid), self.prec)
        if nbytes == 0:
            raise A.LbmError(A.LBM_EINVAL, "lbm_workspace_bytes")
        self.workspace_bytes = int(nbytes)
        with torch.cuda.device(self.device):
            if workspace is None:
                workspace = torch.empty(self.workspace_bytes, dtype=torch.uint8, device=self.device)
            self.ws = workspace
            self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
            h = ctypes.c_void_p()
            A.check(A.lbm_create(ctypes.byref(self._grid), ctypes.byref(self._vset), float(tau), float(dt),
                                 float(dx), self.prec, ctypes.c_void_p(self.ws.data_ptr()),
                                 self.ws.numel(), ctypes.c_void_p(self.stream.cuda_stream), ctypes.byref(h)),
                    "lbm_create")
        self._h = h
        if scheme != "nnd" or not dissipation:
            self.set_scheme(scheme, dissipation)

    @property
    def config(self) -> dict:
        return dict(self._config)

    # -- lifetime -------------------------------------------------------------
    def clone(self, stream=None) -> "Sim":
        """A new sim of the same grid, constants, boundaries and scheme (own
        workspace; state undefined until init / set_f)."""
        return Sim(**self._config, stream=stream)

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            A.lbm_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def handle(self) -> ctypes.c_void_p:
        return self._h

    @property
    def ncell(self) -> int:
        return self.shape[0] * self.shape[1] * self.shape[2]

    # -- state ----------------------------------------------------------------
    def set_t_recovery(self, kappa_max: float):
        """FP64 temperature recovery of the FP32 tiled step for cells whose FP32
        T is ill-conditioned (kappa > kappa_max; 0 = off); see lbm_set_t_recovery."""
        A.check(A.lbm_set_t_recovery(self._h, float(kappa_max)), "lbm_set_t_recovery")
        self.t_recovery = float(kappa_max)

    def set_scheme(self, scheme="nnd", dissipation=True):
        s = SCHEMES[scheme] if isinstance(scheme, str) else int(scheme)
        A.check(A.lbm_set_scheme(self._h, s, int(bool(dissipation))), "lbm_set_scheme")

    def set_launch(self, variant="tiled", zchunk: int = 0, ztail: int = 0):
        """FP32 step kernel: "tiled" (32 x 8 TMA plane tiles, cell pairs, boundary layers
        written by the step; default), "tiled64" (the same on 64 x 8 tiles), "split" (the
        32 x 8 tiles with two warp groups, each updating part of the 15 fields), "tiled_fill"
        (boundary layers by a fill launch), "tiled_single" (one cell per thread) or "plain";
        zchunk = z planes per CTA (0 = auto); ztail > 0 (pair kernels): the end of each
        tile column is split into short chunks of ztail planes, launched last."""
        v = {"tiled": A.LBM_VARIANT_TILED, "plain": A.LBM_VARIANT_PLAIN,
             "tiled_single": A.LBM_VARIANT_TILED_SINGLE, "tiled_fill": A.LBM_VARIANT_TILED_FILL,
             "tiled64": A.LBM_VARIANT_TILED64, "split": A.LBM_VARIANT_TILED_SPLIT}[variant] \
            if isinstance(variant, str) else int(variant)
        A.check(A.lbm_set_launch(self._h, v, int(zchunk), int(ztail)), "lbm_set_launch")
        self.launch = (variant, int(zchunk), int(ztail))

    def init(self, rho, u, T):
        """f = f^eq(rho, u, T); arrays shaped [nz,ny,nx] / [3,nz,ny,nx] (numpy or CUDA tensors)."""
        if isinstance(rho, torch.Tensor) and rho.is_cuda:
            r, uu, t = (x.to(torch.float64).contiguous() for x in (rho, u, T))
            assert r.numel() == self.ncell and uu.numel() == 3 * self.ncell and t.numel() == self.ncell
            A.check(A.lbm_init(self._h, _ptr(r), _ptr(uu), _ptr(t), 1), "lbm_init")
            self._keep = (r, uu, t)  # kernels read them asynchronously
        else:
            r, uu, t = (np.ascontiguousarray(x, dtype=np.float64) for x in (rho, u, T))
            assert r.size == self.ncell and uu.size == 3 * self.ncell and t.size == self.ncell
            A.check(A.lbm_init(self._h, _ptr(r), _ptr(uu), _ptr(t), 0), "lbm_init")

    def step(self, n: int = 1):
        A.check(A.lbm_step(self._h, int(n)), "lbm_step")

    def sync(self):
        A.check(A.lbm_sync(self._h), "lbm_sync")

    @property
    def steps_done(self) -> int:
        return int(A.lbm_steps_done(self._h))

    def moments(self, on_device: bool = False):
        """(rho [nz,ny,nx], u [3,nz,ny,nx], T [nz,ny,nx]) in float64."""
        nz, ny, nx = self.shape
        if on_device:
            rho = torch.empty((nz, ny, nx), dtype=torch.float64, device=self.device)
            u = torch.empty((3, nz, ny, nx), dtype=torch.float64, device=self.device)
            T = torch.empty((nz, ny, nx), dtype=torch.float64, device=self.device)
            A.check(A.lbm_moments(self._h, _ptr(rho), _ptr(u), _ptr(T), 1), "lbm_moments")
            return rho, u, T
        rho = np.empty((nz, ny, nx))
        u = np.empty((3, nz, ny, nx))
        T = np.empty((nz, ny, nx))
        A.check(A.lbm_moments(self._h, _ptr(rho), _ptr(u), _ptr(T), 0), "lbm_moments")
        return rho, u, T

    # -- x slabs (slabs.py) ------------------------------------------------------
    def halo_source(self, side: int, out=None) -> torch.Tensor:
        """The two interior x-columns next to x face `side` (0 lo, 1 hi) of the
        current state as a CUDA tensor [15, nz, ny, 2] in the storage precision
        (lbm_get_halo_source; asynchronous on the sim's stream)."""
        nz, ny, _ = self.shape
        if out is None:
            out = torch.empty((15, nz, ny, 2), device=self.device,
                              dtype=torch.float64 if self.dtype == np.float64 else torch.float32)
        A.check(A.lbm_get_halo_source(self._h, int(side), _ptr(out), 1), "lbm_get_halo_source")
        return out

    def set_halo(self, side: int, buf):
        """The two layers outside the EXTERNAL x face `side` from buf
        ([15, nz, ny, 2]; a CUDA tensor: asynchronous on the sim's stream,
        kept alive until the next call; else a host array: synchronous)."""
        if isinstance(buf, torch.Tensor) and buf.is_cuda:
            b = buf.contiguous()
            A.check(A.lbm_set_halo(self._h, int(side), _ptr(b), 1), "lbm_set_halo")
            self._halo_keep = getattr(self, "_halo_keep", {})
            self._halo_keep[int(side)] = b
        else:
            b = np.ascontiguousarray(buf.numpy() if isinstance(buf, torch.Tensor) else buf, dtype=self.dtype)
            A.check(A.lbm_set_halo(self._h, int(side), _ptr(b), 0), "lbm_set_halo")

    def get_f(self, out=None) -> np.ndarray:
        """Interior f, [15, nz, ny, nx], in the storage precision (host copy,
        or into ``out`` when it is a CUDA tensor of that shape and dtype)."""
        if isinstance(out, torch.Tensor):
            A.check(A.lbm_get_f(self._h, _ptr(out), 1), "lbm_get_f")
            return out
        f = np.empty((15,) + self.shape, dtype=self.dtype)
        A.check(A.lbm_get_f(self._h, _ptr(f), 0), "lbm_get_f")
        return f

    def set_f(self, f):
        if isinstance(f, torch.Tensor) and f.is_cuda:
            ff = f.to(torch.float64 if self.dtype == np.float64 else torch.float32).contiguous()
            A.check(A.lbm_set_f(self._h, _ptr(ff), 1), "lbm_set_f")
            self._keep = ff
        else:
            ff = np.ascontiguousarray(f, dtype=self.dtype)
            assert ff.size == 15 * self.ncell
            A.check(A.lbm_set_f(self._h, _ptr(ff), 0), "lbm_set_f")

    def conserved(self, check_health: bool = True) -> np.ndarray:
        """FP64 (mass, momentum x/y/z, energy) over the interior."""
        out = np.zeros(5)
        rc = A.lbm_conserved(self._h, out.ctypes.data_as(A._dp))
        if rc != A.LBM_OK and (check_health or rc != A.LBM_ENONFINITE):
            raise A.LbmError(rc, "lbm_conserved")
        return out

    def set_timing(self, enable: bool = True):
        """Bracket every launch with CUDA events on the sim's stream."""
        A.check(A.lbm_set_timing(self._h, int(bool(enable))), "lbm_set_timing")

    def timing(self, reset: bool = False) -> dict:
        """{kernel class: (device ms summed, launches)} since creation or the last reset."""
        ms = (ctypes.c_double * A.LBM_NKERNEL)()
        n = (ctypes.c_int64 * A.LBM_NKERNEL)()
        A.check(A.lbm_get_timing(self._h, ms, n, int(bool(reset))), "lbm_get_timing")
        return {A.KERNEL_NAMES[k]: (float(ms[k]), int(n[k])) for k in range(A.LBM_NKERNEL)}

    def health(self) -> int:
        flags = ctypes.c_uint32(0)
        rc = A.lbm_health(self._h, ctypes.byref(flags))
        if rc not in (A.LBM_OK, A.LBM_ENONFINITE, A.LBM_ETIMEOUT):
            raise A.LbmError(rc, "lbm_health")
        return int(flags.value)


def _handles(sims):
    arr = (ctypes.c_void_p * len(sims))()
    for k, s in enumerate(sims):
        arr[k] = s.handle
    return arr


def step_batch(sims, steps: int = 1):
    """Advance FP32 sims together: one persistent tile-kernel launch per step
    covers all of them (lbm_step_batch)."""
    A.check(A.lbm_step_batch(_handles(sims), len(sims), int(steps)), "lbm_step_batch")


class Graph:
    """A captured CUDA graph of `steps` (even) steps of one sim or a batch."""

    def __init__(self, sims, steps: int):
        self.sims = list(sims)
        self.steps = int(steps)
        h = ctypes.c_void_p()
        A.check(A.lbm_graph_capture(_handles(self.sims), len(self.sims), self.steps, ctypes.byref(h)),
                "lbm_graph_capture")
        self._h = h

    def launch(self, times: int = 1):
        for _ in range(int(times)):
            A.check(A.lbm_graph_launch(self._h), "lbm_graph_launch")

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            A.lbm_graph_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def from_workload(w, precision="fp64", **kw) -> Sim:
    """A Sim for a ``workloads.Workload`` (grid, constants and boundaries)."""
    return Sim(w.nx, w.ny, w.nz, w.c1, w.c2, w.eta0, w.tau, w.dt, w.dx, gamma=w.gamma, precision=precision,
               bc_lo=w.bc_lo, bc_hi=w.bc_hi, fixed_lo=w.fixed_lo, fixed_hi=w.fixed_hi, **kw)
