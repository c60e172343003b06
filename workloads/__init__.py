"""Seeded synthetic inputs for the D3V15 FD-LB solver.

This module holds the workloads only: grids, model constants, boundary kinds
and initial macroscopic fields (rho, u, T), plus seeded random perturbations
and request traces.  It contains none of the lattice Boltzmann arithmetic
(no equilibrium, moments or fluxes), so both the CUDA path and the CPU oracle
may take their inputs from it.

Conventions: R = 1 (so T = p / rho), gamma = 1.4, cell-centred nodes
x = (i + 1/2) dx on [0, nx dx), fields shaped [nz, ny, nx] and u [3, nz, ny, nx].
Boundary kinds: 0 periodic, 1 fixed, 2 extrapolate, 3 reflect.
Tuples of states are (rho, u1, u2, u3, T) as in the paper's Sec. 4.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

PERIODIC, FIXED, EXTRAPOLATE, REFLECT = 0, 1, 2, 3
GAMMA = 1.4


def rankine_hugoniot(mach: float, rho1: float = 1.0, p1: float = 1.0, gamma: float = GAMMA):
    """Post-shock (rho2, u2, p2) and shock speed D of a normal shock of Mach
    number ``mach`` moving in +x into gas at rest (rho1, p1)."""
    m2 = mach * mach
    rho2 = rho1 * (gamma + 1.0) * m2 / ((gamma - 1.0) * m2 + 2.0)
    p2 = p1 * (1.0 + 2.0 * gamma / (gamma + 1.0) * (m2 - 1.0))
    a1 = math.sqrt(gamma * p1 / rho1)
    D = mach * a1
    u2 = D * (1.0 - rho1 / rho2)
    return rho2, u2, p2, D


def state_from_p(rho, u1, u2, u3, p):
    """(rho, u1, u2, u3, T) with T = p / rho (R = 1)."""
    return (rho, u1, u2, u3, p / rho)


@dataclasses.dataclass
class Workload:
    """One solver run: grid, constants, boundaries and initial fields."""
    name: str
    nx: int
    ny: int
    nz: int
    dx: float
    c1: float
    c2: float
    eta0: float
    dt: float
    tau: float
    steps: int
    gamma: float = GAMMA
    bc_lo: tuple = (PERIODIC, PERIODIC, PERIODIC)
    bc_hi: tuple = (PERIODIC, PERIODIC, PERIODIC)
    fixed_lo: tuple = ((0.0,) * 5,) * 3
    fixed_hi: tuple = ((0.0,) * 5,) * 3
    ic: object = None  # callable(workload) -> (rho, u, T)
    meta: dict = dataclasses.field(default_factory=dict)

    @property
    def ncell(self) -> int:
        return self.nx * self.ny * self.nz

    def initial_fields(self):
        return self.ic(self)

    def with_grid(self, nx, ny, nz, dx=None):
        """Same physics on another grid (dx defaults to the same domain length in x)."""
        d = dataclasses.replace(self, nx=nx, ny=ny, nz=nz, dx=dx if dx is not None else self.dx * self.nx / nx)
        return d


def cell_centres(n: int, dx: float) -> np.ndarray:
    return (np.arange(n, dtype=np.float64) + 0.5) * dx


def _blend(weight, a, b):
    """Fields of state a where weight = 1 and b where weight = 0, blended in
    (rho, u, p) so that a pressure-matched interface keeps its pressure."""
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)

    def pick(va, vb, mixed):  # exact end states where the weight is 0 or 1
        return np.where(weight == 1.0, va, np.where(weight == 0.0, vb, mixed))

    rho_m = b[0] + weight * (a[0] - b[0])
    p_m = b[0] * b[4] + weight * (a[0] * a[4] - b[0] * b[4])
    rho = pick(a[0], b[0], rho_m)
    u = np.stack([pick(a[1 + k], b[1 + k], b[1 + k] + weight * (a[1 + k] - b[1 + k])) for k in range(3)])
    T = pick(a[4], b[4], p_m / rho_m)
    return rho, u, T


def interface_weight(dist, width: float, dx: float):
    """1 on the inside (dist < 0) and 0 outside: a sharp step (the cell
    centre decides) when width = 0, else 0.5 (1 - tanh(dist / (width dx)))."""
    if width <= 0:
        return (dist < 0).astype(np.float64)
    return 0.5 * (1.0 - np.tanh(dist / (width * dx)))


def _two_state_x(w: Workload, left, right, x0: float):
    x = cell_centres(w.nx, w.dx)
    wt = interface_weight(x - x0, w.meta.get("width", 0.0), w.dx)[None, None, :] * np.ones((w.nz, w.ny, w.nx))
    return _blend(wt, left, right)


def shock_tube(name, nx, ny, nz, dx, left, right, x0, c1, c2, eta0, dt, tau, steps, gamma=GAMMA, width=0.0):
    """Riemann problem along x, periodic in y and z, x faces held at the
    initial left/right states (no wave reaches them before the end time).
    width: interface thickness in cells (0 = sharp, see interface_weight)."""
    w = Workload(name=name, nx=nx, ny=ny, nz=nz, dx=dx, c1=c1, c2=c2, eta0=eta0, dt=dt, tau=tau,
                 steps=steps, gamma=gamma,
                 bc_lo=(FIXED, PERIODIC, PERIODIC), bc_hi=(FIXED, PERIODIC, PERIODIC),
                 fixed_lo=(tuple(left), (0.0,) * 5, (0.0,) * 5),
                 fixed_hi=(tuple(right), (0.0,) * 5, (0.0,) * 5),
                 meta={"left": tuple(left), "right": tuple(right), "x0": x0, "width": float(width)})
    w.ic = _tube_ic
    return w


def _tube_ic(w: Workload):
    return _two_state_x(w, w.meta["left"], w.meta["right"], w.meta["x0"])


def _sphere_ic(w: Workload):
    cx, cy, cz = w.meta["centre"]
    R = w.meta["radius"]
    x = cell_centres(w.nx, w.dx)
    y = cell_centres(w.ny, w.dx)
    z = cell_centres(w.nz, w.dx)
    r = np.sqrt((x[None, None, :] - cx) ** 2 + (y[None, :, None] - cy) ** 2 + (z[:, None, None] - cz) ** 2)
    width = w.meta.get("width", 0.0)
    if width <= 0:
        wt = (r * r <= R * R).astype(np.float64)  # the cell centre decides, r = R inside
    else:
        wt = interface_weight(r - R, width, w.dx)
    return _blend(wt, w.meta["sphere"], w.meta["ambient"])


def shock_sphere(name, nx, ny, nz, dx, mach, sphere_rho, radius, centre, c1, c2, eta0, dt, tau, steps,
                 ambient_rho=1.0, ambient_p=1.0, gamma=GAMMA, width=1.0):
    """Planar shock entering at x = 0 into gas at rest holding a sphere of
    another density at the same pressure.  The domain starts all pre-shock;
    the x-lo boundary layers hold the post-shock state, so the boundary
    Riemann problem is exactly the shock of the given Mach number.  x-hi
    extrapolates, y and z are periodic.  Sphere surface: a tanh profile
    `width` cells thick (interface_weight; 0 = sharp, the cell centre
    decides), blended at constant pressure."""
    rho2, u2, p2, D = rankine_hugoniot(mach, ambient_rho, ambient_p, gamma)
    post = state_from_p(rho2, u2, 0.0, 0.0, p2)
    amb = state_from_p(ambient_rho, 0.0, 0.0, 0.0, ambient_p)
    sph = state_from_p(sphere_rho, 0.0, 0.0, 0.0, ambient_p)
    w = Workload(name=name, nx=nx, ny=ny, nz=nz, dx=dx, c1=c1, c2=c2, eta0=eta0, dt=dt, tau=tau,
                 steps=steps, gamma=gamma,
                 bc_lo=(FIXED, PERIODIC, PERIODIC), bc_hi=(EXTRAPOLATE, PERIODIC, PERIODIC),
                 fixed_lo=(post, (0.0,) * 5, (0.0,) * 5),
                 meta={"ambient": amb, "sphere": sph, "post": post, "centre": tuple(centre),
                       "radius": radius, "mach": mach, "shock_speed": D, "width": float(width)})
    w.ic = _sphere_ic
    return w


# ---------------------------------------------------------------- the workloads

LAX_LEFT = state_from_p(0.445, 0.698, 0.0, 0.0, 3.528)
LAX_RIGHT = state_from_p(0.5, 0.0, 0.0, 0.0, 0.571)
HM_LEFT = state_from_p(5.0, 0.0, 0.0, 0.0, 500.0)
HM_RIGHT = state_from_p(1.0, 0.0, 0.0, 0.0, 1.0)


def lax_tube(nx=200, ny=4, nz=4):
    """Lax shock tube: 200x4x4 on [0,1], dx = 0.005, dt = tau = 2e-5, 7000
    steps to t = 0.14, (c1, c2, eta0) = (2, 6, 2) as in the paper's Lax run."""
    return shock_tube("lax_tube_200x4x4", nx, ny, nz, 1.0 / nx, LAX_LEFT, LAX_RIGHT, 0.5,
                      2.0, 6.0, 2.0, 2e-5, 2e-5, 7000)


def high_mach_tube(nx=2000, ny=4, nz=4):
    """High-Mach tube: 2000x4x4 on [0,1], dx = 5e-4, left (5, 0, p=500),
    right (1, 0, p=1); (c1, c2, eta0) = (12, 36, 20), dt = tau = 2e-6, run
    until the shock reaches x = 0.9 (15,980 steps)."""
    return shock_tube("high_mach_tube_2000x4x4", nx, ny, nz, 1.0 / nx, HM_LEFT, HM_RIGHT, 0.5,
                      12.0, 36.0, 20.0, 2e-6, 2e-6, 15980)


# The paper's own runs (Sec. 4) at the sizes it prints.
PAPER_HM_LEFT = (100.0, 10.0, 0.0, 0.0, 0.714286)
PAPER_HM_RIGHT = (150.0, 0.0, 0.0, 0.0, 50.0)


def paper_high_mach_tube():
    """The paper's high-Mach tube (Fig. 7): left (100, 10, 0, 0, 0.714286), a
    Mach-10 flow, right (150, 0, 0, 0, 50); (c1, c2, eta0) = (8, 24, 8), dx =
    0.01, dt = tau = 1e-5, t = 0.25 (25,000 steps).  The domain length is not
    printed: 300 cells on [0, 3] with the interface at x = 0.5 hold the waves
    (left shock -0.55, right shock +9.17 per unit time) until t = 0.25."""
    return shock_tube("paper_high_mach_tube_300x4x4", 300, 4, 4, 0.01, PAPER_HM_LEFT, PAPER_HM_RIGHT, 0.5,
                      8.0, 24.0, 8.0, 1e-5, 1e-5, 25000)


PAPER_BUBBLE_RHO = {"light": 0.1358, "heavy": 4.1538}


def paper_shock_bubble(kind="light", radius_cells=25, shock_cell=250):
    """The paper's 3D run (Sec. 4(2), Figs. 8-10): 300 x 80 x 80 cells of dx =
    0.001, (c1, c2, eta0) = (2, 6, 4), dt = tau = 1e-5, t = 0.1 (10,000
    steps).  Pre-shock gas (1, 0, 0, 0, 1); a Mach-2 shock moving in -x with
    the post-shock state (2.66667, -1.47902, 0, 0, T = 4.5 / 2.66667) behind
    it (x > shock); a bubble of rho 0.1358 (light) or 4.1538 (heavy) at p = 1
    centred at cell (200, 40, 40).  Boundaries as printed: x-hi holds the
    post-shock state, x-lo extrapolates, the four y / z faces reflect.  The
    bubble radius and the initial shock position are not printed: radius 25
    cells, shock at cell 250.  The bubble surface is one cell thick."""
    nx, ny, nz, dx = 300, 80, 80, 0.001
    r2, u2, p2, D = rankine_hugoniot(2.0)
    post = state_from_p(r2, -u2, 0.0, 0.0, p2)
    amb = state_from_p(1.0, 0.0, 0.0, 0.0, 1.0)
    sph = state_from_p(PAPER_BUBBLE_RHO[kind], 0.0, 0.0, 0.0, 1.0)
    w = Workload(name=f"paper_shock_bubble_{kind}_300x80x80", nx=nx, ny=ny, nz=nz, dx=dx, c1=2.0, c2=6.0, eta0=4.0,
                 dt=1e-5, tau=1e-5, steps=10000, gamma=GAMMA,
                 bc_lo=(EXTRAPOLATE, REFLECT, REFLECT), bc_hi=(FIXED, REFLECT, REFLECT),
                 fixed_hi=(post, (0.0,) * 5, (0.0,) * 5),
                 meta={"ambient": amb, "sphere": sph, "post": post, "centre": ((200 + 0.5) * dx, 40 * dx, 40 * dx),
                       "radius": radius_cells * dx, "mach": 2.0, "shock_speed": D, "width": 1.0,
                       "shock_x": shock_cell * dx})
    w.ic = _paper_bubble_ic
    return w


def _paper_bubble_ic(w: Workload):
    rho, u, T = _sphere_ic(w)
    post = w.meta["post"]
    behind = (cell_centres(w.nx, w.dx) >= w.meta["shock_x"])[None, None, :] & np.ones(rho.shape, dtype=bool)
    rho = np.where(behind, post[0], rho)
    u = np.stack([np.where(behind, post[1 + a], u[a]) for a in range(3)])
    T = np.where(behind, post[4], T)
    return rho, u, T


def shock_droplet(n=256):
    """Mach-2 shock into a rho = 5 droplet (radius 0.1, centre (0.3, 0.5, 0.5))
    on the unit cube, n^3 cells; (c1, c2, eta0) = (2, 6, 4), dt = tau = 5e-5,
    2000 steps."""
    return shock_sphere(f"shock_droplet_{n}^3", n, n, n, 1.0 / n, 2.0, 5.0, 0.1, (0.3, 0.5, 0.5),
                        2.0, 6.0, 4.0, 5e-5, 5e-5, 2000)


def shock_bubble(nx=512, ny=256, nz=256, mach=3.0, c=(4.0, 12.0, 8.0), dt=2e-5):
    """Mach-3 shock into a rho = 0.1 bubble (radius 0.15, centre (0.35, 0.5,
    0.5)), 512x256x256 cells of 1/256; (c1, c2, eta0) = (4, 12, 8), dt = tau = 2e-5
    unless given."""
    dx = 1.0 / ny
    return shock_sphere(f"shock_bubble_{nx}x{ny}x{nz}", nx, ny, nz, dx, mach, 0.1, 0.15, (0.35, 0.5, 0.5),
                        c[0], c[1], c[2], dt, dt, 2000)


def batch_machs(seed: int = 4, n: int = 8):
    """Seeded Mach numbers of the concurrent 128^3 copies, uniform in [1.5, 6]."""
    return np.random.default_rng(seed).uniform(1.5, 6.0, size=n)


def noise(shape, seed: int, amplitude: float = 1.0) -> np.ndarray:
    """Seeded uniform noise in [-amplitude, amplitude]."""
    return np.random.default_rng(seed).uniform(-amplitude, amplitude, size=shape)


def smooth_random_fields(nx, ny, nz, seed: int, rho0=1.0, u0=(0.3, -0.2, 0.1), T0=1.0, amp=0.1):
    """Smooth periodic random (rho, u, T): a few seeded Fourier modes on top of a
    uniform state, small enough to keep rho and T positive."""
    rng = np.random.default_rng(seed)
    z, y, x = np.meshgrid(np.arange(nz) / nz, np.arange(ny) / ny, np.arange(nx) / nx, indexing="ij")

    def field():
        out = np.zeros((nz, ny, nx))
        for _ in range(3):
            kx, ky, kz = rng.integers(0, 3, size=3)
            ph = rng.uniform(0, 2 * np.pi)
            out += rng.uniform(-1, 1) * np.cos(2 * np.pi * (kx * x + ky * y + kz * z) + ph)
        return out / 3.0

    rho = rho0 * (1.0 + amp * field())
    u = np.stack([u0[a] + amp * field() for a in range(3)])
    T = T0 * (1.0 + amp * field())
    return rho, u, T


# ---------------------------------------------------------------- serving trace

SERVING_GRIDS = ((64, 64, 64), (96, 96, 96), (128, 128, 128), (192, 128, 128), (256, 256, 256))


def serving_trace(seed: int = 5, n: int = 200, rate: float = 20.0, grids=SERVING_GRIDS,
                  steps=(500, 3000), mach=(1.2, 10.0), ratio=(0.1, 10.0)):
    """Seeded request stream: exponential inter-arrival times of mean 1/rate,
    grid uniform over `grids`, Mach uniform, density ratio log-uniform, step
    count uniform in [steps[0], steps[1]], kind 50/50 shock tube or shock
    sphere.  Returns a list of dicts sorted by arrival time (seconds)."""
    rng = np.random.default_rng(seed)
    t = np.cumsum(rng.exponential(1.0 / rate, size=n))
    out = []
    for k in range(n):
        g = grids[int(rng.integers(0, len(grids)))]
        out.append({
            "id": k,
            "arrival": float(t[k]),
            "grid": tuple(int(v) for v in g),
            "mach": float(rng.uniform(*mach)),
            "ratio": float(10.0 ** rng.uniform(math.log10(ratio[0]), math.log10(ratio[1]))),
            "steps": int(rng.integers(steps[0], steps[1] + 1)),
            "kind": "tube" if rng.uniform() < 0.5 else "sphere",
        })
    return out


def request_states(req):
    """Pre-shock, post-shock and second-gas states (rho, u1, u2, u3, T) of a
    request: a shock of the request's Mach number into gas at rest (1, 0, p=1),
    and gas of density `ratio` at the same pressure (the tube's right state or
    the sphere)."""
    r2, u2, p2, _ = rankine_hugoniot(req["mach"])
    pre = state_from_p(1.0, 0.0, 0.0, 0.0, 1.0)
    post = state_from_p(r2, u2, 0.0, 0.0, p2)
    other = state_from_p(req["ratio"], 0.0, 0.0, 0.0, 1.0)
    return pre, post, other


def request_workload(req, c1, c2, eta0, dt, width=3.0):
    """The Workload of a request with the given model constants.  Tube: the
    post-shock state (x < 0.3 of the domain) against gas of the request's
    density ratio; sphere: the shock entering at x = 0 into ambient gas holding
    a sphere of that density (radius 0.1 L_y, centre (0.3 L_x, 0.5, 0.5)).
    Both interfaces are `width` cells thick (interface_weight): served
    requests reach Mach 10 into gas ten times lighter or heavier, where a
    one-cell jump can drive T below zero at the interface."""
    nx, ny, nz = req["grid"]
    dx = 1.0 / ny
    pre, post, other = request_states(req)
    if req["kind"] == "tube":
        w = shock_tube(f"req{req['id']}_tube", nx, ny, nz, dx, post, other, 0.3 * nx * dx, c1, c2, eta0, dt, dt,
                       req["steps"], width=width)
    else:
        w = shock_sphere(f"req{req['id']}_sphere", nx, ny, nz, dx, req["mach"], req["ratio"], 0.1,
                         (0.3 * nx * dx, 0.5, 0.5), c1, c2, eta0, dt, dt, req["steps"], width=width)
    return w
