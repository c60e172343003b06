"""FP64 CPU oracle of the D3V15 FD-LB step (arXiv:1010.4135).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
the CPU-baseline leg of ``bench.py`` may import this package.  It shares no
code with the CUDA library in ``paper_1010_4135_gb300``; the only module both
sides use is ``workloads`` (seeded initial conditions, no LBM arithmetic).

``oracle.c`` holds the stepper (plain C, double precision, no contraction);
this module compiles it on first use and wraps it with ctypes.  Fields use
the layout f[i][z][y][x] (interior cells only), rho/T [z][y][x], u [3][z][y][x].

Parity status of each function (which passage pins it is listed in the tests):
  feq, moments       Sec. 2 (Eq. "eq", relations e1-e5)   pinned by test_oracle_model
  step / run         Sec. 3 (Eq. "nnd", minmod, Eq. "lp") pinned by test_oracle_scheme,
                     test_oracle_invariants, test_oracle_vonneumann, test_oracle_riemann
  boundary layers    Sec. 4(2)                            pinned by test_oracle_boundaries
  riemann.*          exact solution of the 1D Riemann problem, pinned by the printed
                     Mach-2 state (Sec. 4(2)) and Rankine-Hugoniot / isentropic laws
  vonneumann.*       the amplification matrix G of Sec. 3, pinned against the
                     measured one-step growth of the first-order-upwind oracle
"""
from __future__ import annotations

import ctypes
import dataclasses
import os
import subprocess
import threading

import numpy as np

NV = 15
PERIODIC, FIXED, EXTRAPOLATE, REFLECT = 0, 1, 2, 3
NND, UPWIND2, UPWIND1 = 0, 1, 2

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile oracle.c into oracle/_build/liboracle.so (gcc, -O2, no FP contraction, OpenMP)."""
    os.makedirs(_BUILD, exist_ok=True)
    stale = force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC)
    if stale:
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        cmd = ["gcc", "-std=c99", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp",
               "-shared", "-fPIC", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class _Cfg(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("nz", ctypes.c_int32),
        ("bc_lo", ctypes.c_int32 * 3), ("bc_hi", ctypes.c_int32 * 3),
        ("fixed_lo", (ctypes.c_double * 5) * 3), ("fixed_hi", (ctypes.c_double * 5) * 3),
        ("c1", ctypes.c_double), ("c2", ctypes.c_double), ("eta0", ctypes.c_double),
        ("gamma", ctypes.c_double),
        ("tau", ctypes.c_double), ("dt", ctypes.c_double), ("dx", ctypes.c_double),
        ("scheme", ctypes.c_int32), ("dissipation", ctypes.c_int32),
    ]


@dataclasses.dataclass
class Cfg:
    """Grid, boundary kinds, model constants and scheme of one oracle run."""
    nx: int
    ny: int
    nz: int
    c1: float
    c2: float
    eta0: float
    gamma: float = 1.4
    tau: float = 1e-5
    dt: float = 1e-5
    dx: float = 1e-3
    bc_lo: tuple = (PERIODIC, PERIODIC, PERIODIC)
    bc_hi: tuple = (PERIODIC, PERIODIC, PERIODIC)
    fixed_lo: tuple = ((0.0,) * 5,) * 3
    fixed_hi: tuple = ((0.0,) * 5,) * 3
    scheme: int = NND
    dissipation: int = 1

    def to_c(self) -> _Cfg:
        c = _Cfg()
        c.nx, c.ny, c.nz = self.nx, self.ny, self.nz
        for a in range(3):
            c.bc_lo[a] = int(self.bc_lo[a])
            c.bc_hi[a] = int(self.bc_hi[a])
            for k in range(5):
                c.fixed_lo[a][k] = float(self.fixed_lo[a][k])
                c.fixed_hi[a][k] = float(self.fixed_hi[a][k])
        c.c1, c.c2, c.eta0, c.gamma = self.c1, self.c2, self.eta0, self.gamma
        c.tau, c.dt, c.dx = self.tau, self.dt, self.dx
        c.scheme, c.dissipation = int(self.scheme), int(self.dissipation)
        return c

    @property
    def ncell(self) -> int:
        return self.nx * self.ny * self.nz


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            dp = ctypes.POINTER(ctypes.c_double)
            cp = ctypes.POINTER(_Cfg)
            lib.oracle_velocities.argtypes = [cp, dp, dp]
            lib.oracle_feq.argtypes = [cp, ctypes.c_double, dp, ctypes.c_double, dp]
            lib.oracle_moments.argtypes = [cp, dp, dp]
            lib.oracle_run.argtypes = [cp, dp, ctypes.c_int64, ctypes.c_int]
            lib.oracle_run.restype = ctypes.c_int
            lib.oracle_step.argtypes = [cp, dp, dp, ctypes.c_int]
            lib.oracle_step.restype = ctypes.c_int
            lib.oracle_step_nodes.argtypes = [cp, dp, ctypes.c_int64, ctypes.POINTER(ctypes.c_int32), dp]
            lib.oracle_step_nodes.restype = ctypes.c_int
            lib.oracle_padded.argtypes = [cp, dp, dp]
            lib.oracle_padded.restype = ctypes.c_int
            lib.oracle_init.argtypes = [cp, dp, dp, dp, dp]
            lib.oracle_macros.argtypes = [cp, dp, dp, dp, dp]
            lib.oracle_conserved.argtypes = [cp, dp, dp]
            lib.oracle_max_threads.restype = ctypes.c_int
            _lib = lib
    return _lib


def _dp(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def velocities(cfg: Cfg):
    """(v[15,3], eta[15]) of the D3V15 set (Sec. 2)."""
    v = np.zeros((NV, 3))
    eta = np.zeros(NV)
    _load().oracle_velocities(ctypes.byref(cfg.to_c()), _dp(v), _dp(eta))
    return v, eta


def feq(cfg: Cfg, rho: float, u, T: float) -> np.ndarray:
    """f_i^eq of one node (Eq. "eq")."""
    out = np.zeros(NV)
    uu = _f64(u)
    _load().oracle_feq(ctypes.byref(cfg.to_c()), float(rho), _dp(uu), float(T), _dp(out))
    return out


def moments(cfg: Cfg, f) -> np.ndarray:
    """(rho, u1, u2, u3, T, E) of one node's 15 values."""
    ff = _f64(f)
    out = np.zeros(6)
    _load().oracle_moments(ctypes.byref(cfg.to_c()), _dp(ff), _dp(out))
    return out


def init(cfg: Cfg, rho, u, T) -> np.ndarray:
    """f = f^eq(rho, u, T) on every interior node; returns [15, nz, ny, nx]."""
    r, uu, t = _f64(rho), _f64(u), _f64(T)
    assert r.size == cfg.ncell and uu.size == 3 * cfg.ncell and t.size == cfg.ncell
    f = np.zeros((NV, cfg.nz, cfg.ny, cfg.nx))
    _load().oracle_init(ctypes.byref(cfg.to_c()), _dp(r), _dp(uu), _dp(t), _dp(f))
    return f


def step(cfg: Cfg, f, nthreads: int = 1) -> np.ndarray:
    """One time step; returns a new array."""
    fin = _f64(f)
    assert fin.size == NV * cfg.ncell
    fout = np.empty_like(fin)
    rc = _load().oracle_step(ctypes.byref(cfg.to_c()), _dp(fin), _dp(fout), int(nthreads))
    if rc != 0:
        raise ValueError(f"oracle_step failed ({rc})")
    return fout


def step_nodes(cfg: Cfg, f, xyz) -> np.ndarray:
    """One time step evaluated only at the nodes xyz ([k, 3] of x, y, z);
    returns [k, 15].  Boundary layers are evaluated on the fly."""
    fin = _f64(f)
    assert fin.size == NV * cfg.ncell
    idx = np.ascontiguousarray(xyz, dtype=np.int32).reshape(-1, 3)
    out = np.zeros((idx.shape[0], NV))
    rc = _load().oracle_step_nodes(ctypes.byref(cfg.to_c()), _dp(fin), idx.shape[0],
                                   idx.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), _dp(out))
    if rc != 0:
        raise ValueError(f"oracle_step_nodes failed ({rc})")
    return out


def padded(cfg: Cfg, f) -> np.ndarray:
    """The working copy with two boundary layers per face, [15, nz+4, ny+4, nx+4]
    (interior node (x, y, z) at [.., z+2, y+2, x+2]; edges/corners NaN)."""
    fin = _f64(f)
    out = np.zeros((NV, cfg.nz + 4, cfg.ny + 4, cfg.nx + 4))
    rc = _load().oracle_padded(ctypes.byref(cfg.to_c()), _dp(fin), _dp(out))
    if rc != 0:
        raise ValueError(f"oracle_padded failed ({rc})")
    return out


def run(cfg: Cfg, f, nsteps: int, nthreads: int = 1) -> np.ndarray:
    """nsteps time steps; returns a new array."""
    g = np.array(f, dtype=np.float64, order="C", copy=True)
    assert g.size == NV * cfg.ncell
    rc = _load().oracle_run(ctypes.byref(cfg.to_c()), _dp(g), int(nsteps), int(nthreads))
    if rc != 0:
        raise ValueError(f"oracle_run failed ({rc})")
    return g


def macros(cfg: Cfg, f):
    """(rho [nz,ny,nx], u [3,nz,ny,nx], T [nz,ny,nx]) of every node."""
    ff = _f64(f)
    rho = np.zeros((cfg.nz, cfg.ny, cfg.nx))
    u = np.zeros((3, cfg.nz, cfg.ny, cfg.nx))
    T = np.zeros((cfg.nz, cfg.ny, cfg.nx))
    _load().oracle_macros(ctypes.byref(cfg.to_c()), _dp(ff), _dp(rho), _dp(u), _dp(T))
    return rho, u, T


def conserved(cfg: Cfg, f) -> np.ndarray:
    """(mass, momentum x/y/z, energy) summed over the interior."""
    ff = _f64(f)
    out = np.zeros(5)
    _load().oracle_conserved(ctypes.byref(cfg.to_c()), _dp(ff), _dp(out))
    return out


def cfg_for(w, **over) -> Cfg:
    """Oracle configuration of a ``workloads.Workload`` (keyword overrides allowed)."""
    kw = dict(nx=w.nx, ny=w.ny, nz=w.nz, c1=w.c1, c2=w.c2, eta0=w.eta0, gamma=w.gamma, tau=w.tau,
              dt=w.dt, dx=w.dx, bc_lo=w.bc_lo, bc_hi=w.bc_hi, fixed_lo=w.fixed_lo, fixed_hi=w.fixed_hi)
    kw.update(over)
    return Cfg(**kw)


def max_threads() -> int:
    return int(_load().oracle_max_threads())
