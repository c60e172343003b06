"""Shared helpers of the GPU parity tests: seeded cases and error metrics.

Parity metric (per field): max |a - b| / max(max |b|, 1e-300) over interior
cells, evaluated for each f_i and for rho, rho u and E.  FP64 bar: 1e-12.
"""
from __future__ import annotations

import os

import numpy as np

import oracle
import workloads

NTHREADS = max(1, os.cpu_count() or 1)

STATE_LO = (1.2, 0.3, -0.1, 0.05, 1.1)
STATE_HI = (0.9, 0.1, 0.0, -0.2, 0.8)

# name -> grid, boundary kinds and constants.  Sizes span several 32x8 tiles
# with ragged tails, and the degenerate 1- and 2-cell axes.
CASES = {
    "periodic_37x19x11": dict(n=(37, 19, 11), lo=(0, 0, 0), hi=(0, 0, 0), c=(2.0, 6.0, 3.0)),
    "fixed_extrap_reflect_33x17x9": dict(n=(33, 17, 9), lo=(1, 3, 0), hi=(2, 3, 0), c=(2.0, 6.0, 4.0)),
    "reflect_extrap_fixed_20x12x14": dict(n=(20, 12, 14), lo=(3, 2, 1), hi=(3, 1, 3), c=(3.0, 9.0, 3.0)),
    "single_cell_1x1x1": dict(n=(1, 1, 1), lo=(0, 0, 0), hi=(0, 0, 0), c=(2.0, 6.0, 2.0)),
    "line_2x1x1_extrapolate": dict(n=(2, 1, 1), lo=(2, 0, 0), hi=(2, 0, 0), c=(2.0, 6.0, 2.0)),
    "column_1x5x3": dict(n=(1, 5, 3), lo=(0, 3, 1), hi=(0, 3, 1), c=(2.0, 5.0, 2.5)),
    "wide_70x9x5": dict(n=(70, 9, 5), lo=(1, 0, 3), hi=(1, 0, 3), c=(2.0, 6.0, 2.0)),
    # nx, ny multiples of both tile shapes (32 x 8, 64 x 8): the pair kernels' full-tile form
    "full_tiles_64x16x10": dict(n=(64, 16, 10), lo=(1, 0, 3), hi=(2, 0, 3), c=(2.0, 6.0, 4.0)),
}


def case_cfg(name, scheme=oracle.NND, dissipation=1, dt=2e-4, tau=5e-4, dx=0.02):
    c = CASES[name]
    nx, ny, nz = c["n"]
    c1, c2, eta0 = c["c"]
    return oracle.Cfg(nx=nx, ny=ny, nz=nz, c1=c1, c2=c2, eta0=eta0, gamma=1.4, tau=tau, dt=dt, dx=dx,
                      bc_lo=c["lo"], bc_hi=c["hi"], fixed_lo=(STATE_LO,) * 3, fixed_hi=(STATE_HI,) * 3,
                      scheme=scheme, dissipation=dissipation)


def initial_f(cfg, seed, noise=0.02):
    rho, u, T = workloads.smooth_random_fields(cfg.nx, cfg.ny, cfg.nz, seed, amp=0.1)
    f = oracle.init(cfg, rho, u, T)
    return f * (1.0 + workloads.noise(f.shape, seed + 100, noise))


def sim_for(cfg, precision):
    from paper_1010_4135_gb300 import sim as S
    scheme = {oracle.NND: "nnd", oracle.UPWIND2: "upwind2", oracle.UPWIND1: "upwind1"}[cfg.scheme]
    return S.Sim(cfg.nx, cfg.ny, cfg.nz, cfg.c1, cfg.c2, cfg.eta0, cfg.tau, cfg.dt, cfg.dx, gamma=cfg.gamma,
                 precision=precision, bc_lo=cfg.bc_lo, bc_hi=cfg.bc_hi, fixed_lo=cfg.fixed_lo,
                 fixed_hi=cfg.fixed_hi, scheme=scheme, dissipation=bool(cfg.dissipation))


def field_errors(a, b):
    """Per-field normalised max errors of two [15, ...] arrays."""
    a = np.asarray(a, dtype=np.float64).reshape(15, -1)
    b = np.asarray(b, dtype=np.float64).reshape(15, -1)
    return np.array([np.abs(a[i] - b[i]).max() / max(np.abs(b[i]).max(), 1e-300) for i in range(15)])


def conserved_fields(cfg, f):
    """rho, rho u (3), E per cell from f (oracle velocities), [5, ncell]."""
    v, eta = oracle.velocities(cfg)
    ff = np.asarray(f, dtype=np.float64).reshape(15, -1)
    vsq = (v * v).sum(1) + eta * eta
    return np.stack([ff.sum(0), v[:, 0] @ ff, v[:, 1] @ ff, v[:, 2] @ ff, vsq @ ff])


def moment_errors(cfg, a, b):
    ca, cb = conserved_fields(cfg, a), conserved_fields(cfg, b)
    return np.array([np.abs(ca[k] - cb[k]).max() / max(np.abs(cb[k]).max(), 1e-300) for k in range(5)])


def l1_rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.abs(a - b).sum() / np.abs(b).sum())


# ---------------------------------------------------------------- FP32 error model
#
# The FP32 path stores and updates f in float.  Per time step every stored
# value picks up C_ROUND roundings of relative size U32 = 2^-24, counted along
# the kernel's path of one value: the moment sums (five levels of the
# summation tree), three more for the temperature, five in the equilibrium
# (Eq. "eq" as A + B w + D w^2 and the product with rho) and three fused
# multiply-adds in the update, the last of which is the stored rounding.
# Taken coherent within a step, they put an error of C_ROUND U32 kappa rho
# into a cell's density, where the condition number kappa of a state is the
# larger of
#   kappa_rho = sum_i |f_i^eq| / rho                         (relation e1)
#   kappa_T   = sum_i |f_i^eq| (|v_i|^2 + eta_i^2) / (rho b T)  (e3 for T)
# (the equilibrium's populations are of both signs, so the sums cancel).
# Across steps the errors are independent and the scheme damps them (a single
# perturbation of the initial state shrinks), so they add as a random walk:
#   L1(n) <= C_ROUND U32 kappa_max sqrt(n),
# kappa_max over the states of the workload.  The bound is fixed by the
# model, not by measurement.
U32 = 2.0 ** -24
C_ROUND = 16


def kappa(cfg, state):
    """Condition number (max of kappa_rho, kappa_T) of the macroscopic state
    (rho, u1, u2, u3, T) under the model constants of cfg."""
    v, eta = oracle.velocities(cfg)
    fe = oracle.feq(cfg, state[0], state[1:4], state[4])
    b = 2.0 / (cfg.gamma - 1.0)
    k_rho = np.abs(fe).sum() / state[0]
    k_T = (np.abs(fe) * ((v * v).sum(1) + eta * eta)).sum() / (state[0] * b * state[4])
    return float(max(k_rho, k_T))


def fp32_l1_bound(cfg, states, nsteps):
    """The FP32 model's bound on the L1 relative density error after nsteps."""
    return C_ROUND * U32 * max(kappa(cfg, s) for s in states) * float(np.sqrt(max(1, nsteps)))


def linf_rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.abs(a - b).max() / np.abs(b).max())
