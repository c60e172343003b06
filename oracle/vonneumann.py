"""Von Neumann amplification matrix of the FD-LB scheme (Sec. 3).

TEST INFRASTRUCTURE ONLY (part of the oracle).

For a perturbation Delta f_i = F_i exp(i k . x) of a uniform state, one step
maps F^t to F^{t+dt} = G F^t with (Sec. 3, matrix G_ij and the function phi)

  G_ij = (1 - dt/tau - sum_a v_ia dt/dx phi_ia) delta_ij + dt/tau dfeq_i/df_j
         + lambda_i dt sum_a (e^{i k_a dx} - 2 + e^{-i k_a dx}) / dx^2 delta_ij,
  phi_ia = (1 - alpha~)(1 - e^{-i k_a dx})  if v_ia >= 0,
           (1 - beta~)(e^{i k_a dx} - 1)    if v_ia <  0.

The Jacobian dfeq_i/df_j is the chain rule through (rho, u, T) written in the
paper; here it is evaluated by complex-step differentiation of the map
f -> f^eq(moments(f)), which is exact to rounding for this rational map.  The
equilibrium below is a second, independent transcription of Eq. "eq" (numpy,
complex-capable); the tests check it against the moment relations too.

With alpha~ = beta~ = 0 this G is the exact linearisation of the first-order
upwind variant of the oracle stepper, which the tests use to pin both.
"""
from __future__ import annotations

import numpy as np

NV = 15


def velocity_set(c1: float, c2: float, eta0: float):
    """(v[15,3], eta[15]) in the oracle's index order (Sec. 2)."""
    s = c2 / np.sqrt(3.0)
    v = np.zeros((NV, 3))
    for a in range(3):
        v[1 + 2 * a, a] = c1
        v[2 + 2 * a, a] = -c1
    for k in range(8):
        v[7 + k] = [(-s if k & 4 else s), (-s if k & 2 else s), (-s if k & 1 else s)]
    eta = np.zeros(NV)
    eta[0] = eta0
    return v, eta


def equilibrium(rho, u, T, c1, c2, eta0, gamma):
    """f^eq (Eq. "eq") for complex or real (rho, u[3], T)."""
    b = 2.0 / (gamma - 1.0)
    v, _ = velocity_set(c1, c2, eta0)
    u = np.asarray(u)
    usq = u[0] * u[0] + u[1] * u[1] + u[2] * u[2]
    c12, c22 = c1 * c1, c2 * c2
    out = np.zeros(NV, dtype=np.result_type(rho, u, T, np.float64))
    for i in range(NV):
        vu = v[i, 0] * u[0] + v[i, 1] * u[1] + v[i, 2] * u[2]
        if i == 0:
            A, B, D = (b - 3.0) * T / eta0 ** 2, 0.0, 0.0
        elif i <= 6:
            A = (-c22 + ((b - 3.0) * c22 / eta0 ** 2 + 3.0) * T + c22 / c12 * usq) / (6.0 * (c12 - c22))
            B = (-c22 + (b + 2.0) * T + usq) / (2.0 * c12 * (c12 - c22))
            D = 1.0 / (2.0 * c12 ** 2)
        else:
            A = (-c12 + ((b - 3.0) * c12 / eta0 ** 2 + 3.0) * T
                 + (3.0 * c12 - c22) / (2.0 * c22) * usq) / (8.0 * (c22 - c12))
            B = 3.0 * (-c12 + (b + 2.0) * T + usq) / (8.0 * c22 * (c22 - c12))
            D = 9.0 / (16.0 * c22 ** 2)
        out[i] = rho * (A + B * vu + D * vu * vu)
    return out


def macroscopic(f, c1, c2, eta0, gamma):
    """(rho, u[3], T) from 15 values (relations e1-e3, R = 1)."""
    v, eta = velocity_set(c1, c2, eta0)
    b = 2.0 / (gamma - 1.0)
    rho = f.sum()
    u = (f[:, None] * v).sum(0) / rho
    E = (f * ((v * v).sum(1) + eta * eta)).sum()
    T = (E / rho - (u * u).sum()) / b
    return rho, u, T


def feq_jacobian(rho, u, T, c1, c2, eta0, gamma, h: float = 1e-30):
    """d f^eq_i / d f_j at the equilibrium of (rho, u, T) by complex step."""
    f0 = equilibrium(rho, np.asarray(u, float), T, c1, c2, eta0, gamma).astype(complex)
    J = np.zeros((NV, NV))
    for j in range(NV):
        f = f0.copy()
        f[j] += 1j * h
        r, uu, t = macroscopic(f, c1, c2, eta0, gamma)
        J[:, j] = np.imag(equilibrium(r, uu, t, c1, c2, eta0, gamma)) / h
    return J


def amplification_matrix(rho, u, T, c1, c2, eta0, gamma, dt, tau, dx, k,
                         alpha_t: float = 0.0, beta_t: float = 0.0, dissipation: bool = True):
    """G(k) (15x15 complex); k is a 3-vector of wave numbers."""
    v, _ = velocity_set(c1, c2, eta0)
    k = np.asarray(k, dtype=np.float64)
    J = feq_jacobian(rho, u, T, c1, c2, eta0, gamma)
    lam = np.zeros(NV)
    if dissipation:
        lam[0] = c1 * dx
        lam[1:7] = c1 * dx / 10.0
    G = (dt / tau) * J.astype(complex)
    for i in range(NV):
        diag = 1.0 - dt / tau
        for a in range(3):
            th = k[a] * dx
            if v[i, a] >= 0.0:
                phi = (1.0 - alpha_t) * (1.0 - np.exp(-1j * th))
            else:
                phi = (1.0 - beta_t) * (np.exp(1j * th) - 1.0)
            diag = diag - v[i, a] * dt / dx * phi
            diag = diag + lam[i] * dt * (np.exp(1j * th) - 2.0 + np.exp(-1j * th)) / dx ** 2
        G[i, i] += diag
    return G


def max_growth(rho, u, T, c1, c2, eta0, gamma, dt, tau, dx, kdx_values, direction=(1.0, 0.0, 0.0),
               alpha_t: float = 0.0, beta_t: float = 0.0, dissipation: bool = True) -> float:
    """max over the sampled k dx of the spectral radius of G (the paper's
    max|omega|), with k along ``direction``."""
    d = np.asarray(direction, dtype=np.float64)
    d = d / np.linalg.norm(d)
    worst = 0.0
    for kdx in kdx_values:
        G = amplification_matrix(rho, u, T, c1, c2, eta0, gamma, dt, tau, dx, d * (kdx / dx),
                                 alpha_t, beta_t, dissipation)
        worst = max(worst, float(np.abs(np.linalg.eigvals(G)).max()))
    return worst
