"""Continuous-batching solve server.

Requests (shock tubes and shock-sphere solves of different grids, Mach
numbers and density ratios) arrive over time.  The server admits a request
when it has arrived, a batch slot is free and its workspace fits the HBM
budget; admitted grids stay resident and advance together, one batched tile
kernel launch per time step covering every resident grid (lbm_step_batch).
A request retires after its own number of steps: its moments are copied to
the host, its workspace is released, and waiting requests are admitted in
arrival order.  Latency is measured from arrival to retirement.
"""
from __future__ import annotations

import collections
import ctypes
import dataclasses
import time

import numpy as np
import torch

import workloads
from . import _abi as A
from . import autotune
from . import sim as S
from . import stability


@dataclasses.dataclass
class Job:
    req: dict
    params: tuple
    sim: object = None
    nbytes: int = 0
    remaining: int = 0
    admitted: float = 0.0
    finished: float = 0.0
    health: int = 0
    rho: object = None


def request_parameters(req):
    """(c1, c2, eta0, dt) of a request from the von Neumann rule, applied to
    its initial states and to the star states where the shocked gas meets
    the second gas (the tube's contact, the sphere's surface)."""
    nx, ny, nz = req["grid"]
    pre, post, other = workloads.request_states(req)
    states = [pre, post, other, *stability.interaction_states(post, other)]
    c1, c2, eta0, dt = stability.choose_parameters(states, 1.0 / ny)
    if dt is None:
        dt = min(stability.DT_CANDIDATES)
    return c1, c2, eta0, dt


def workspace_bytes(grid, precision=A.LBM_FP32) -> int:
    g = A.make_grid(*grid)
    return int(A.lbm_workspace_bytes(ctypes.byref(g), precision))


class Server:
    """hbm_budget: bytes of workspace the resident grids may hold together
    (default: 80% of the device's free memory); tick: most steps launched
    between two retirement checks; tune: give each admitted grid the z chunk
    the autotuner measured for its shape (once per shape, then cached)."""

    def __init__(self, hbm_budget=None, max_batch=A.LBM_MAX_BATCH, tick=50, keep_results=False, tune=True):
        if hbm_budget is None:
            free, _ = torch.cuda.mem_get_info()
            hbm_budget = int(0.8 * free)
        self.budget = int(hbm_budget)
        self.max_batch = int(max_batch)
        self.tick = int(tick)
        self.keep_results = keep_results
        self.tune = tune
        self.peak_bytes = 0
        self.peak_batch = 0
        self.launches = 0

    def _admit(self, job: Job):
        w = workloads.request_workload(job.req, *job.params)
        s = S.from_workload(w, precision="fp32")
        rho, u, T = w.initial_fields()
        s.init(rho, u, T)
        if self.tune:
            autotune.tune(s)
        job.sim = s
        job.remaining = job.req["steps"]

    def run(self, trace, time_scale: float = 1.0):
        """Serve `trace` (arrival times scaled by time_scale) in real time; returns the finished jobs."""
        pending = collections.deque(sorted(trace, key=lambda r: r["arrival"]))
        jobs_waiting: collections.deque = collections.deque()
        active: list = []
        done: list = []
        used = 0
        t0 = time.perf_counter()
        while pending or jobs_waiting or active:
            now = time.perf_counter() - t0
            while pending and pending[0]["arrival"] * time_scale <= now:
                r = pending.popleft()
                jobs_waiting.append(Job(req=r, params=request_parameters(r), nbytes=workspace_bytes(r["grid"])))
            # admission in arrival order, by footprint and batch slots
            while jobs_waiting and len(active) < self.max_batch and used + jobs_waiting[0].nbytes <= self.budget:
                j = jobs_waiting.popleft()
                self._admit(j)
                j.admitted = time.perf_counter() - t0
                used += j.nbytes
                active.append(j)
            if jobs_waiting and not active and jobs_waiting[0].nbytes > self.budget:
                raise RuntimeError(f"request {jobs_waiting[0].req['id']} exceeds the HBM budget")
            self.peak_bytes = max(self.peak_bytes, used)
            self.peak_batch = max(self.peak_batch, len(active))
            if not active:
                if pending:
                    time.sleep(max(0.0, pending[0]["arrival"] * time_scale - (time.perf_counter() - t0)))
                continue
            n = min(self.tick, min(j.remaining for j in active))
            S.step_batch([j.sim for j in active], n)
            self.launches += n
            for j in active:
                j.remaining -= n
            still = []
            for j in active:
                if j.remaining > 0:
                    still.append(j)
                    continue
                j.health = j.sim.health()
                rho, _, _ = j.sim.moments()  # synchronises
                j.finished = time.perf_counter() - t0
                if self.keep_results:
                    j.rho = rho
                j.sim.close()
                j.sim = None
                used -= j.nbytes
                done.append(j)
            active = still
        self.wall = time.perf_counter() - t0
        return done


def summary(done, wall, time_scale=1.0):
    lat = np.array([j.finished - j.req["arrival"] * time_scale for j in done])
    cells = sum(int(np.prod(j.req["grid"])) * j.req["steps"] for j in done)
    return {
        "requests": len(done),
        "p50_latency_s": float(np.percentile(lat, 50)),
        "p99_latency_s": float(np.percentile(lat, 99)),
        "mean_latency_s": float(lat.mean()),
        "solves_per_s": len(done) / wall,
        "cell_updates_per_s": cells / wall,
        "wall_s": wall,
        "unhealthy": int(sum(1 for j in done if j.health)),
    }
