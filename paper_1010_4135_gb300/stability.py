"""Von Neumann stability of the FD-LB step (Sec. 3) for choosing run parameters.

For a perturbation F exp(i k.x) of a uniform state, one step multiplies F by

  G_ij = (1 - dt/tau - sum_a v_ia dt/dx phi_ia) d_ij + dt/tau df^eq_i/df_j
         + lambda_i dt sum_a (2 cos(k_a dx) - 2)/dx^2 d_ij,
  phi_ia = (1 - a~)(1 - e^{-i k_a dx}) for v_ia >= 0,  (1 - b~)(e^{i k_a dx} - 1) otherwise,

with the equilibrium Jacobian evaluated by the chain rule through (rho, u, T)
as the paper writes it:
  d rho/df_j = 1,  d u_a/df_j = (v_ja - u_a)/rho,
  d T/df_j = (|v_j - u|^2 + eta_j^2 - b T)/(b rho),
and the partial derivatives of f^eq_i = rho (A_i + B_i w_i + D_i w_i^2),
w_i = v_i . u, taken from the printed A_i, B_i, D_i.

The scheme is accepted when max |omega| <= 1 + tol over the sampled wave
numbers (the paper's criterion max |omega| <= 1, read to plotting accuracy).
`max_growth` evaluates G on the host (numpy eigenvalues); `max_growth_device`
evaluates a whole batch of parameter sets in one launch of liblbm.so's
lbm_vn_max_growth (G built per thread, Hessenberg QR eigenvalues), and
`choose_parameters(..., device=True)` uses it for every candidate at once.
"""
from __future__ import annotations

import math

import numpy as np

NV = 15


def velocities(c1: float, c2: float, eta0: float):
    s = c2 / math.sqrt(3.0)
    v = np.zeros((NV, 3))
    for a in range(3):
        v[1 + 2 * a, a] = c1
        v[2 + 2 * a, a] = -c1
    signs = np.array([[1, 1, 1], [1, 1, -1], [1, -1, 1], [1, -1, -1],
                      [-1, 1, 1], [-1, 1, -1], [-1, -1, 1], [-1, -1, -1]], dtype=float)
    v[7:] = s * signs
    eta = np.zeros(NV)
    eta[0] = eta0
    return v, eta


def _shell_coefficients(c1, c2, eta0, b):
    """Per-velocity (A0, AT, AU, B0, BT, BU, D) with A = A0 + AT T + AU u^2 etc."""
    c12, c22, e2 = c1 * c1, c2 * c2, eta0 * eta0
    co = np.zeros((NV, 7))
    co[0] = [0.0, (b - 3.0) / e2, 0.0, 0.0, 0.0, 0.0, 0.0]
    ka = 1.0 / (6.0 * (c12 - c22))
    kb = 1.0 / (2.0 * c12 * (c12 - c22))
    co[1:7] = [-c22 * ka, ((b - 3.0) * c22 / e2 + 3.0) * ka, c22 / c12 * ka,
               -c22 * kb, (b + 2.0) * kb, kb, 1.0 / (2.0 * c12 * c12)]
    kd = 1.0 / (8.0 * (c22 - c12))
    ke = 3.0 / (8.0 * c22 * (c22 - c12))
    co[7:] = [-c12 * kd, ((b - 3.0) * c12 / e2 + 3.0) * kd, (3.0 * c12 - c22) / (2.0 * c22) * kd,
              -c12 * ke, (b + 2.0) * ke, ke, 9.0 / (16.0 * c22 * c22)]
    return co


def equilibrium_jacobian(rho, u, T, c1, c2, eta0, gamma):
    """d f^eq_i / d f_j (15 x 15) at the equilibrium of (rho, u, T)."""
    b = 2.0 / (gamma - 1.0)
    u = np.asarray(u, dtype=float)
    v, eta = velocities(c1, c2, eta0)
    co = _shell_coefficients(c1, c2, eta0, b)
    usq = float(u @ u)
    w = v @ u
    A = co[:, 0] + co[:, 1] * T + co[:, 2] * usq
    B = co[:, 3] + co[:, 4] * T + co[:, 5] * usq
    D = co[:, 6]
    dfeq_drho = A + B * w + D * w * w
    dfeq_dT = rho * (co[:, 1] + co[:, 4] * w)
    # d/du_a of rho (A + B w + D w^2): A and B depend on u^2, w on u
    dfeq_du = rho * ((2.0 * co[:, 2] + 2.0 * co[:, 5] * w)[:, None] * u[None, :]
                     + (B + 2.0 * D * w)[:, None] * v)
    drho_df = np.ones(NV)
    du_df = (v - u[None, :]) / rho                      # [j, a]
    rel = v - u[None, :]
    dT_df = ((rel * rel).sum(1) + eta * eta - b * T) / (b * rho)
    return np.outer(dfeq_drho, drho_df) + np.outer(dfeq_dT, dT_df) + dfeq_du @ du_df.T


def amplification(rho, u, T, c1, c2, eta0, gamma, dt, tau, dx, k, alpha_t=0.0, beta_t=0.0,
                  dissipation=True):
    v, _ = velocities(c1, c2, eta0)
    k = np.asarray(k, dtype=float)
    th = k * dx
    lam = np.zeros(NV)
    if dissipation:
        lam[0] = c1 * dx
        lam[1:7] = c1 * dx / 10.0
    phi = np.where(v >= 0.0, (1.0 - alpha_t) * (1.0 - np.exp(-1j * th))[None, :],
                   (1.0 - beta_t) * (np.exp(1j * th) - 1.0)[None, :])
    diag = (1.0 - dt / tau) - (v * phi).sum(1) * dt / dx \
        + lam * dt * (2.0 * np.cos(th) - 2.0).sum() / (dx * dx)
    return np.diag(diag) + (dt / tau) * equilibrium_jacobian(rho, u, T, c1, c2, eta0, gamma)


def max_growth(states, c1, c2, eta0, gamma, dt, tau, dx, nk=48,
               directions=((1.0, 0.0, 0.0), (1.0, 1.0, 1.0)), dissipation=True) -> float:
    """max |omega| over the states (rho, u1, u2, u3, T), directions and nk wave numbers."""
    worst = 0.0
    kdx = np.linspace(math.pi / nk, math.pi, nk)
    for st in states:
        rho, u, T = st[0], np.asarray(st[1:4], dtype=float), st[4]
        for d in directions:
            dd = np.asarray(d, dtype=float)
            dd = dd / np.linalg.norm(dd)
            for q in kdx:
                G = amplification(rho, u, T, c1, c2, eta0, gamma, dt, tau, dx, dd * q / dx,
                                  dissipation=dissipation)
                worst = max(worst, float(np.abs(np.linalg.eigvals(G)).max()))
    return worst


DIRECTIONS = ((1.0, 0.0, 0.0), (1.0, 1.0, 1.0))


def max_growth_device(states, param_sets, directions=DIRECTIONS, nk=48, dissipation=True, stream=None):
    """max |omega| per parameter set (c1, c2, eta0, gamma, dt, tau, dx) over
    the states, directions and the nk wave numbers k dx = pi q / nk, q = 1..nk
    (the same samples as max_growth), in one launch of lbm_vn_max_growth on
    the current CUDA device.  Returns a numpy array (synchronises `stream`)."""
    import ctypes

    import torch

    from . import _abi as A
    dev = torch.device("cuda", torch.cuda.current_device())
    st = torch.tensor([[float(x) for x in s] for s in states], dtype=torch.float64, device=dev)
    ps = torch.tensor([[float(x) for x in p] for p in param_sets], dtype=torch.float64, device=dev)
    ds = torch.tensor([[float(x) for x in d] for d in directions], dtype=torch.float64, device=dev)
    out = torch.empty(len(param_sets), dtype=torch.float64, device=dev)
    stream = stream if stream is not None else torch.cuda.current_stream(dev)
    A.check(A.lbm_vn_max_growth(ctypes.c_void_p(st.data_ptr()), len(states), ctypes.c_void_p(ps.data_ptr()),
                                len(param_sets), ctypes.c_void_p(ds.data_ptr()), len(directions), int(nk),
                                int(bool(dissipation)), ctypes.c_void_p(out.data_ptr()),
                                ctypes.c_void_p(stream.cuda_stream)), "lbm_vn_max_growth")
    stream.synchronize()
    return out.cpu().numpy()


def _velocity_jump(p, rho, pk, gamma):
    """Velocity change across a wave that takes gas (rho, pk) at rest in its
    own frame to pressure p: a shock (Rankine-Hugoniot) when p > pk, an
    isentropic rarefaction otherwise."""
    if p > pk:
        return (p - pk) * math.sqrt(2.0 / ((gamma + 1.0) * rho) / (p + (gamma - 1.0) / (gamma + 1.0) * pk))
    a = math.sqrt(gamma * pk / rho)
    return 2.0 * a / (gamma - 1.0) * ((p / pk) ** ((gamma - 1.0) / (2.0 * gamma)) - 1.0)


def interaction_states(left, right, gamma=1.4):
    """The two states of the star region when gas `left` meets gas `right`
    along x (states (rho, u1, u2, u3, T), R = 1 so p = rho T): the pressure
    p* solves jump_L(p*) + jump_R(p*) = u_L - u_R (bisection on log p), both
    sides move with u*, and each density follows its wave (shock adiabat or
    isentrope).  A shock reaching a bubble or a contact produces these states;
    the flow there can be faster and hotter than behind the incident shock
    (a Mach 5.7 shock into gas ten times lighter drives it to u* = 8.2 with
    T = 27 behind the transmitted shock), so the parameter rule must see them."""
    rl, ul, Tl = float(left[0]), float(left[1]), float(left[4])
    rr, ur, Tr = float(right[0]), float(right[1]), float(right[4])
    pl, pr = rl * Tl, rr * Tr

    def g(p):
        return _velocity_jump(p, rl, pl, gamma) + _velocity_jump(p, rr, pr, gamma) + (ur - ul)

    lo, hi = 1e-12 * min(pl, pr), 1e3 * max(pl, pr) + 1.0
    while g(hi) < 0.0:
        hi *= 10.0
    if g(lo) > 0.0:
        raise ValueError("the two states separate into vacuum")
    for _ in range(200):
        mid = math.sqrt(lo * hi)
        if g(mid) > 0.0:
            hi = mid
        else:
            lo = mid
    p = math.sqrt(lo * hi)
    u = 0.5 * (ul + ur) + 0.5 * (_velocity_jump(p, rr, pr, gamma) - _velocity_jump(p, rl, pl, gamma))
    mu = (gamma - 1.0) / (gamma + 1.0)

    def density(rho, pk):
        return rho * (p / pk + mu) / (mu * p / pk + 1.0) if p > pk else rho * (p / pk) ** (1.0 / gamma)

    dl, dr = density(rl, pl), density(rr, pr)
    return (dl, u, 0.0, 0.0, p / dl), (dr, u, 0.0, 0.0, p / dr)


DT_CANDIDATES = (5e-5, 2e-5, 1e-5, 5e-6, 2e-6, 1e-6, 5e-7, 2e-7)
COURANT_MAX = 0.025


def courant(c2: float, dt: float, dx: float) -> float:
    """Courant number of the diagonal velocities along one axis, (c2/sqrt 3) dt / dx."""
    return c2 / math.sqrt(3.0) * dt / dx


def choose_parameters(states, dx, gamma=1.4, tol=1e-3, candidates=DT_CANDIDATES, courant_max=COURANT_MAX,
                      c1_factors=(1.0, 1.1, 1.2, 1.35, 1.5), device=False, stream=None):
    """(c1, c2, eta0, dt) for a run whose fastest material speed is set by the
    given states, following the paper's advice (c1 near the largest flow
    speed, c2 about 3 c1, eta0 1-2 c1): c2 = 3 c1, eta0 = 2 c1, and c1 the
    smallest of max(2, ceil(f max|u|)) over the factors f for which some dt =
    tau among the candidates has max|omega| <= 1 + tol and a diagonal Courant
    number <= courant_max (the largest such dt).  The smallest stable c1
    matters beyond the linear criterion: at a density jump into cold gas the
    populations of large c1 carry negative energy across (T < 0 near the
    interface within tens of steps once c1^2 / T is near 100), and strong
    shocks need the small Courant numbers of the paper's runs (0.01-0.035):
    1D runs of Mach 2-10 shocks stay positive up to 0.05 and fail for some at
    0.15.  Returns dt = None when no candidate passes.  device=True measures
    every candidate in one batched launch on the current CUDA device and
    applies the same rule to the results."""
    umax = max(math.sqrt(sum(float(x) ** 2 for x in st[1:4])) for st in states)
    order = []  # (c1, dt) in the order the rule tries them
    tried = []
    for f in c1_factors:
        c1 = float(max(2, math.ceil(f * umax)))
        if c1 in tried:
            continue
        tried.append(c1)
        for dt in sorted(candidates, reverse=True):
            if courant(3.0 * c1, dt, dx) <= courant_max:
                order.append((c1, dt))
    if device and order:
        g = max_growth_device(states, [(c1, 3.0 * c1, 2.0 * c1, gamma, dt, dt, dx) for c1, dt in order], nk=24,
                              stream=stream)
        for (c1, dt), growth in zip(order, g):
            if growth <= 1.0 + tol:
                return c1, 3.0 * c1, 2.0 * c1, dt
    elif not device:
        for c1, dt in order:
            if max_growth(states, c1, 3.0 * c1, 2.0 * c1, gamma, dt, dt, dx, nk=24) <= 1.0 + tol:
                return c1, 3.0 * c1, 2.0 * c1, dt
    c1 = tried[-1]
    return c1, 3.0 * c1, 2.0 * c1, None
