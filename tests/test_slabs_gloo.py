"""The x-slab decomposition of slabs.py as gloo ranks on the CPU.

Each rank owns one slab of the grid and steps it with the oracle: the two
columns it receives from each neighbour are placed as two extra interior
columns beside the cut face, and the oracle steps the widened slab (its x
faces there extrapolate; the extra columns' own new values are discarded).
Own cells read at most two columns across a face (the stencil of Sec. 3), so
when the partition, the plan and the halo exchange are right, the slabs put
together equal the unsplit oracle run bit for bit.  Cases: two ranks with
fixed / extrapolating x faces, two ranks on a periodic x axis (both
neighbours are the same rank), three ranks with reflecting x faces.
"""
import os
import socket

import numpy as np
import pytest
import torch
import torch.multiprocessing as mp

import oracle
import workloads

STEPS = 6


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


STATE_LO = (1.2, 0.3, -0.1, 0.05, 1.1)
STATE_HI = (0.9, 0.1, 0.0, -0.2, 0.8)


def _cfg(nx, bcx):
    return oracle.Cfg(nx=nx, ny=6, nz=5, c1=2.0, c2=6.0, eta0=3.0, gamma=1.4, tau=5e-4, dt=2e-4, dx=0.02,
                      bc_lo=(bcx[0], 0, 3), bc_hi=(bcx[1], 0, 3), fixed_lo=(STATE_LO,) * 3, fixed_hi=(STATE_HI,) * 3)


def _f0(cfg):
    rho, u, T = workloads.smooth_random_fields(cfg.nx, cfg.ny, cfg.nz, 7, amp=0.1)
    f = oracle.init(cfg, rho, u, T)
    return f * (1.0 + workloads.noise(f.shape, 8, 0.02))


class OracleSlab:
    """A slab stepped by the oracle on the widened slab (see the module text)."""

    def __init__(self, cfg, plan, f):
        self.cfg, self.p, self.f = cfg, plan, f
        self.halo = {}

    def halo_source(self, side):
        return torch.from_numpy(np.ascontiguousarray(self.f[..., :2] if side == 0 else self.f[..., -2:]))

    def set_halo(self, side, buf):
        self.halo[side] = buf.numpy().copy()

    def step(self, n):
        import dataclasses
        assert n == 1
        parts, lo_bc, hi_bc, off = [], self.cfg.bc_lo[0], self.cfg.bc_hi[0], 0
        if self.p.left is not None:
            parts.append(self.halo.pop(0))
            lo_bc, off = oracle.EXTRAPOLATE, 2
        parts.append(self.f)
        if self.p.right is not None:
            parts.append(self.halo.pop(1))
            hi_bc = oracle.EXTRAPOLATE
        wide = np.concatenate(parts, axis=3)
        cw = dataclasses.replace(self.cfg, nx=wide.shape[3], bc_lo=(lo_bc,) + tuple(self.cfg.bc_lo[1:]),
                                 bc_hi=(hi_bc,) + tuple(self.cfg.bc_hi[1:]))
        self.f = oracle.step(cw, wide)[..., off:off + self.p.nx].copy()


def _worker(rank, world, port, nx, bcx, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import torch.distributed as dist
    from paper_1010_4135_gb300 import slabs
    dist.init_process_group("gloo", rank=rank, world_size=world)
    cfg = _cfg(nx, bcx)
    p = slabs.plan(cfg.nx, cfg.bc_lo, cfg.bc_hi, rank, world)
    stepper = OracleSlab(cfg, p, _f0(cfg)[..., p.x0:p.x1].copy())
    slabs.advance(stepper, p, STEPS)
    q.put((rank, p.x0, p.x1, stepper.f))
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("world,nx,bcx", [(2, 13, (oracle.FIXED, oracle.EXTRAPOLATE)),
                                          (2, 12, (oracle.PERIODIC, oracle.PERIODIC)),
                                          (3, 14, (oracle.REFLECT, oracle.REFLECT))])
def test_slabs_equal_the_whole_grid(world, nx, bcx):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, nx, bcx, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = sorted((q.get(timeout=180) for _ in procs), key=lambda o: o[0])
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    cfg = _cfg(nx, bcx)
    ref = oracle.run(cfg, _f0(cfg), STEPS)
    assert [(o[1], o[2]) for o in out] == [(a, b) for a, b in __import__(
        "paper_1010_4135_gb300.slabs", fromlist=["partition"]).partition(nx, world)]
    got = np.concatenate([o[3] for o in out], axis=3)
    assert np.array_equal(got, ref)
    # the run moved the state: the comparison is not vacuous
    assert np.abs(ref - _f0(cfg)).max() > 1e-4 * np.abs(ref).max()


def test_partition_and_plan():
    from paper_1010_4135_gb300 import slabs
    assert slabs.partition(10, 3) == [(0, 4), (4, 7), (7, 10)]
    assert slabs.partition(4, 2) == [(0, 2), (2, 4)]
    with pytest.raises(ValueError):
        slabs.partition(5, 3)  # a slab of one cell cannot give its neighbour two columns
    p = slabs.plan(10, (1, 0, 0), (2, 0, 0), 0, 3)
    assert (p.left, p.right, p.bc_lo[0], p.bc_hi[0]) == (None, 1, 1, slabs.BC_EXTERNAL)
    p = slabs.plan(10, (1, 0, 0), (2, 0, 0), 2, 3)
    assert (p.left, p.right, p.bc_lo[0], p.bc_hi[0]) == (1, None, slabs.BC_EXTERNAL, 2)
    p = slabs.plan(10, (0, 0, 0), (0, 0, 0), 0, 2)  # periodic x: a ring
    assert (p.left, p.right, p.bc_lo[0], p.bc_hi[0]) == (1, 1, slabs.BC_EXTERNAL, slabs.BC_EXTERNAL)
    p = slabs.plan(10, (0, 0, 0), (0, 0, 0), 0, 1)  # one slab on a periodic axis: its own neighbour
    assert (p.left, p.right) == (0, 0)
