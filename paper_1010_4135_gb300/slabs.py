"""x-slab decomposition of one grid over several ranks (one GPU each).

The grid's nx cells along x are cut into contiguous slabs (`partition`);
rank r owns slab r as its own solver instance, whose faces at the cuts are of
kind LBM_BC_EXTERNAL.  Before every step each rank sends the two boundary
x-columns of its state to its neighbours and writes the two columns it
receives into the two layers outside its cut faces (`exchange`).  The global
x faces keep the grid's own boundary kinds; for a periodic x axis the first
and the last slab are neighbours (a ring).  The scheme's stencil (Sec. 3:
NND convection and the dissipation Laplacian) reaches two cells along an
axis and no further, so with the halos in place every slab advances exactly
as the same cells of the whole grid: one exchange of 2 x 15 x ny x nz values
per cut face and step.

The exchange is torch.distributed point-to-point messaging (NCCL between
GPUs; gloo between host processes).  A stepper is anything with
`halo_source(side)` (the two interior columns next to x face `side`, 0 = lo,
1 = hi, as a [15, nz, ny, 2] tensor), `set_halo(side, buf)` and `step(n)`;
`Sim` is the GPU one.
"""
from __future__ import annotations

import dataclasses

import torch
import torch.distributed as dist

BC_PERIODIC, BC_EXTERNAL = 0, 4  # lbm.h boundary kinds
TAG_LO, TAG_HI = 11, 12  # message tags: a rank's lo / hi boundary columns


def partition(nx: int, world: int):
    """[(x0, x1)] of the world's slabs: contiguous, sizes differing by at most
    one (the first nx % world slabs one cell longer), each at least two cells
    (the two columns a neighbour needs)."""
    if world < 1 or nx < 2 * world:
        raise ValueError(f"cannot cut {nx} cells into {world} slabs of at least two cells")
    base, extra = divmod(nx, world)
    out, x0 = [], 0
    for r in range(world):
        x1 = x0 + base + (1 if r < extra else 0)
        out.append((x0, x1))
        x0 = x1
    return out


@dataclasses.dataclass
class SlabPlan:
    """One rank's slab: its x range and x-face kinds, and its neighbours
    (None at a global face)."""
    rank: int
    world: int
    x0: int
    x1: int
    bc_lo: tuple
    bc_hi: tuple
    left: int | None
    right: int | None

    @property
    def nx(self) -> int:
        return self.x1 - self.x0


def plan(nx: int, bc_lo, bc_hi, rank: int, world: int) -> SlabPlan:
    """The slab of `rank`: x faces at cuts become EXTERNAL; a periodic x axis
    links the last slab to the first (with one rank, to itself)."""
    x0, x1 = partition(nx, world)[rank]
    periodic = bc_lo[0] == BC_PERIODIC
    left = rank - 1 if rank > 0 else (world - 1 if periodic else None)
    right = rank + 1 if rank < world - 1 else (0 if periodic else None)
    lo = list(bc_lo)
    hi = list(bc_hi)
    if left is not None:
        lo[0] = BC_EXTERNAL
    if right is not None:
        hi[0] = BC_EXTERNAL
    return SlabPlan(rank, world, x0, x1, tuple(lo), tuple(hi), left, right)


def exchange(stepper, p: SlabPlan, group=None):
    """Halo exchange of one step: send this slab's lo columns to the left
    neighbour and its hi columns to the right one; the right neighbour's lo
    columns become this slab's hi layers and the left one's hi columns its lo
    layers.  Messages are tagged by the face they come from, and posted in
    the same order on every rank (sends lo, hi; receives from the right,
    from the left), which also pairs them when both neighbours are one rank
    (two slabs in a ring) and the transport ignores tags."""
    lo_src = stepper.halo_source(0) if p.left is not None else None
    hi_src = stepper.halo_source(1) if p.right is not None else None
    if p.world == 1:  # a periodic ring of one slab: its own columns wrap around
        if p.left is not None:
            stepper.set_halo(1, lo_src)
            stepper.set_halo(0, hi_src)
        return
    ref = lo_src if lo_src is not None else hi_src
    if ref is None:
        return
    lo_halo = torch.empty_like(ref) if p.left is not None else None
    hi_halo = torch.empty_like(ref) if p.right is not None else None
    ops = []
    if p.left is not None:
        ops.append(dist.P2POp(dist.isend, lo_src, p.left, group=group, tag=TAG_LO))
    if p.right is not None:
        ops.append(dist.P2POp(dist.isend, hi_src, p.right, group=group, tag=TAG_HI))
    if p.right is not None:
        ops.append(dist.P2POp(dist.irecv, hi_halo, p.right, group=group, tag=TAG_LO))
    if p.left is not None:
        ops.append(dist.P2POp(dist.irecv, lo_halo, p.left, group=group, tag=TAG_HI))
    for req in dist.batch_isend_irecv(ops):
        req.wait()
    if lo_halo is not None:
        stepper.set_halo(0, lo_halo)
    if hi_halo is not None:
        stepper.set_halo(1, hi_halo)


def advance(stepper, p: SlabPlan, steps: int, group=None):
    """`steps` time steps of this rank's slab, each after its halo exchange."""
    for _ in range(int(steps)):
        exchange(stepper, p, group)
        stepper.step(1)


def slab_workload(w, p: SlabPlan):
    """The rank's part of a workloads.Workload: its x range of the grid with
    the slab's x-face kinds (other faces and constants unchanged); its
    initial fields are that x range of the whole grid's."""
    return dataclasses.replace(w, name=f"{w.name}_slab{p.rank}of{p.world}", nx=p.nx, bc_lo=p.bc_lo, bc_hi=p.bc_hi,
                               ic=lambda _w: slab_fields(w.initial_fields(), p))


def slab_fields(fields, p: SlabPlan):
    """The rank's x range of initial fields (rho [nz,ny,nx], u [3,nz,ny,nx], T)."""
    rho, u, T = fields
    return rho[..., p.x0:p.x1].copy(), u[..., p.x0:p.x1].copy(), T[..., p.x0:p.x1].copy()


def exchange_local(steppers, plans):
    """The halo exchange of slabs held by one process (their sims on one or
    several GPUs): every slab's source columns are taken before any halo is
    written, then each cut face gets its neighbour's columns.  With sims on
    one stream the copies are ordered by that stream."""
    src = [(st.halo_source(0) if p.left is not None else None, st.halo_source(1) if p.right is not None else None)
           for st, p in zip(steppers, plans)]
    for st, p in zip(steppers, plans):
        if p.left is not None:
            st.set_halo(0, src[p.left][1])
        if p.right is not None:
            st.set_halo(1, src[p.right][0])


def advance_local(steppers, plans, steps: int):
    """`steps` time steps of all slabs held by one process."""
    for _ in range(int(steps)):
        exchange_local(steppers, plans)
        for st in steppers:
            st.step(1)
