"""Continuous-batching solve server.

Requests (shock tubes and shock-sphere solves of different grids, Mach
numbers and density ratios) arrive over time.  On arrival a worker thread
prepares each request off the serving loop: its parameters (the von Neumann
rule of stability.py) and its initial fields.  The loop admits a prepared
request when a batch slot is free and its workspace fits the HBM budget;
admitted grids stay resident and advance together, one batched tile kernel
launch per time step covering every resident grid (lbm_step_batch).

The loop never drains the GPU to make progress: steps are launched a tick
(at most `tick` steps) at a time with at most two ticks in flight; a
request that has run its steps gets its moments and health bits queued on
the stream (lbm_moments_async / lbm_health_async into page-locked memory)
and an event recorded behind them; its workspace is released once that
event has completed, and its latency ends there (arrival to results on the
host).  Waiting requests are admitted in arrival order (policy "fifo", the
default: a request that does not fit the memory left blocks the ones behind
it), or shortest job first (policy "sjf": among the prepared requests that fit,
the one with the fewest cell-updates; re-solves first), which cuts the
median latency under overload at the cost of the largest requests.  SJF
bounds the wait: a request that later arrivals have overtaken MAX_BYPASS
times is admitted next, before anything younger, as soon as it fits.

A request whose result comes back unhealthy (health bits: rho <= 0, T <= 0,
non-finite) is solved again with the next parameter candidate
(request_parameters(req, attempt)), ahead of the waiting queue; its latency
keeps counting from the original arrival.
"""
from __future__ import annotations

import collections
import concurrent.futures as cf
import ctypes
import dataclasses
import threading
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
    nbytes: int = 0
    attempt: int = 0           # parameter candidate (request_parameters)
    prep: object = None        # future of (params, workload, (rho, u, T) page-locked)
    fields: tuple = None       # the page-locked initial fields while their copy is in flight
    params: tuple = None
    sim: object = None
    remaining: int = 0
    admitted: float = 0.0
    finished: float = 0.0
    health: int = 0
    bypassed: int = 0          # later arrivals admitted ahead of this job (SJF)
    rho: object = None
    # retirement in flight
    event: object = None
    out: tuple = None          # device (rho, u, T) of the final state
    host_rho: object = None    # page-locked copy of rho
    host_flags: object = None  # page-locked health bits


ATTEMPTS = 3  # parameter candidates per request
POLICIES = ("fifo", "sjf")
MAX_BYPASS = 32  # SJF: later arrivals that may overtake a waiting request


def work(req) -> int:
    """Cell-updates a request needs."""
    nx, ny, nz = req["grid"]
    return int(nx) * int(ny) * int(nz) * int(req["steps"])


def next_admission(waiting, used: int, budget: int, policy: str = "fifo", max_bypass: int = MAX_BYPASS):
    """The waiting job to admit next, or None: FIFO takes the head of the
    queue if it is prepared and fits the memory left; SJF takes, among the
    prepared jobs that fit, a re-solve first, else the one with the least
    work (ties in arrival order) -- unless a job has been overtaken
    max_bypass times (`bypassed`, counted by note_admission): the oldest such
    job goes next, and nothing else is admitted until it is prepared and
    fits, so no request waits without bound while small ones keep arriving."""
    if policy == "fifo":
        if waiting and waiting[0].prep.done() and used + waiting[0].nbytes <= budget:
            return waiting[0]
        return None
    starved = next((j for j in waiting if j.bypassed >= max_bypass), None)
    if starved is not None:
        return starved if starved.prep.done() and used + starved.nbytes <= budget else None
    best, key = None, None
    for j in waiting:
        if not j.prep.done() or used + j.nbytes > budget:
            continue
        k = (j.attempt == 0, work(j.req))
        if key is None or k < key:
            best, key = j, k
    return best


def note_admission(waiting, job):
    """Count the overtaking: every job still waiting that arrived before
    `job` (is ahead of it in the queue) has been bypassed once more."""
    for j in waiting:
        if j is job:
            break
        j.bypassed += 1


_tls = threading.local()


def _service_stream():
    """A CUDA stream of this (preparation) thread for the parameter service."""
    s = getattr(_tls, "stream", None)
    if s is None:
        s = torch.cuda.Stream()
        _tls.stream = s
    return s


def request_parameters(req, attempt: int = 0, device: bool = False):
    """(c1, c2, eta0, dt) of a request.  Attempt 0: the von Neumann rule
    (stability.choose_parameters) applied to its initial states and to the
    star states where the shocked gas meets the second gas (the tube's
    contact, the sphere's surface).  The rule's linear criterion is a
    sufficient one; at strong density jumps into cold gas a smaller c1 keeps
    the populations realizable, so attempt 1 takes c1 - 1 (c2 = 3 c1, eta0 =
    2 c1), attempt 2 the rule's c1 with eta0 = c1 (the paper's most common
    choice).  Measured on the seeded 200-request trace: the three requests
    the rule left unhealthy all finish healthy with attempt 1.  device=True
    measures all candidates in one launch of the on-device von Neumann service
    (on this thread's own stream)."""
    nx, ny, nz = req["grid"]
    pre, post, other = workloads.request_states(req)
    states = [pre, post, other, *stability.interaction_states(post, other)]
    c1, c2, eta0, dt = stability.choose_parameters(states, 1.0 / ny, device=device,
                                                   stream=_service_stream() if device else None)
    if dt is None:
        dt = min(stability.DT_CANDIDATES)
    if attempt == 1 and c1 > 2.0:
        c1 -= 1.0
        c2, eta0 = 3.0 * c1, 2.0 * c1
    elif attempt >= 2:
        eta0 = c1
    return c1, c2, eta0, dt


def prepare(req, attempt: int = 0, device: bool = False, timing=None):
    """Work of one request before admission: parameters (the von Neumann rule,
    on the device with device=True), workload and initial fields (in
    page-locked memory, ready for an asynchronous copy).  timing(params_s,
    fields_s), if given, receives the seconds of the two parts."""
    t0 = time.perf_counter()
    params = request_parameters(req, attempt, device)
    t1 = time.perf_counter()
    w = workloads.request_workload(req, *params)
    fields = tuple(torch.from_numpy(np.ascontiguousarray(a)).pin_memory() for a in w.initial_fields())
    if timing is not None:
        timing(t1 - t0, time.perf_counter() - t1)
    return params, w, fields


def workspace_bytes(grid, precision=A.LBM_FP32) -> int:
    g = A.make_grid(*grid)
    return int(A.lbm_workspace_bytes(ctypes.byref(g), precision))


class Server:
    """hbm_budget: bytes of workspace the resident grids may hold together
    (default: 80% of the device's free memory); tick: most steps launched
    per batched launch sequence between two looks at the queue; tune: give
    each admitted grid the launch configuration the autotuner measured for
    its shape (once per shape, then cached; `tune_shapes` does it ahead).
    One batched launch runs one kernel, so every grid keeps the default tile
    shape and only its z chunk and tail are tuned."""

    VARIANT = ("tiled",)

    def __init__(self, hbm_budget=None, max_batch=A.LBM_MAX_BATCH, tick=50, keep_results=False, tune=True,
                 prep_workers=2, policy="fifo", vn_device=True):
        if policy not in POLICIES:
            raise ValueError(f"policy must be one of {POLICIES}")
        self.policy = policy
        if hbm_budget is None:
            free, _ = torch.cuda.mem_get_info()
            hbm_budget = int(0.8 * free)
        self.budget = int(hbm_budget)
        self.max_batch = int(max_batch)
        self.tick = int(tick)
        self.keep_results = keep_results
        self.tune = tune
        self.prep_workers = int(prep_workers)
        self.stream = torch.cuda.Stream()
        self.peak_bytes = 0
        self.peak_batch = 0
        self.launches = 0
        self.retries = 0
        self.host_s = collections.Counter()  # host seconds by activity
        # request preparation (worker threads): the parameter rule on the device
        # (vn_device) or the host, and the initial fields
        self.vn_device = bool(vn_device)
        self.prep_s = collections.Counter()
        self._prep_lock = threading.Lock()

    def _warm_workers(self, pool):
        """Before the clock starts: every preparation thread sets up its CUDA
        stream and runs the parameter service once, so that the first
        requests do not pay that set-up in their latency."""
        if not self.vn_device:
            return
        gate = threading.Barrier(self.prep_workers)

        def warm():
            gate.wait(timeout=120)
            stability.max_growth_device([(1.0, 0.0, 0.0, 0.0, 1.0)], [(2.0, 6.0, 4.0, 1.4, 1e-5, 1e-5, 0.01)],
                                        nk=2, stream=_service_stream())

        for f in [pool.submit(warm) for _ in range(self.prep_workers)]:
            f.result()

    def _note_prep(self, params_s, fields_s):
        with self._prep_lock:
            self.prep_s["params"] += params_s
            self.prep_s["fields"] += fields_s
            self.prep_s["requests"] += 1

    def tune_shapes(self, grids):
        """Autotune each grid shape once before serving (cached per shape)."""
        if not self.tune:
            return
        for g in grids:
            w = workloads.request_workload({"id": -1, "grid": tuple(g), "mach": 2.0, "ratio": 1.0,
                                            "steps": 1, "kind": "sphere"}, 2.0, 6.0, 4.0, 1e-5)
            s = S.from_workload(w, precision="fp32", stream=self.stream)
            s.init(*w.initial_fields())
            autotune.tune(s, variants=self.VARIANT)
            s.close()

    def _admit(self, job: Job):
        params, w, fields = job.prep.result()
        job.params = params
        job.fields = fields
        s = S.from_workload(w, precision="fp32", stream=self.stream)
        with torch.cuda.stream(self.stream):
            rho, u, T = (f.to(s.device, non_blocking=True) for f in fields)
        s.init(rho, u, T)  # device pointers: stream-ordered, no synchronisation
        if self.tune:
            autotune.tune(s, variants=self.VARIANT)
        job.sim = s
        job.remaining = job.req["steps"]

    @staticmethod
    def _health(job: Job) -> int:
        """Health bits of a retired job (the page-locked copy of its flags)."""
        return int(job.host_flags[0])

    def _retire_start(self, job: Job):
        """Queue the final moments and health bits behind the job's steps."""
        s = job.sim
        nz, ny, nx = s.shape
        with torch.cuda.stream(self.stream):
            rho = torch.empty((nz, ny, nx), dtype=torch.float64, device=s.device)
            u = torch.empty((3, nz, ny, nx), dtype=torch.float64, device=s.device)
            T = torch.empty((nz, ny, nx), dtype=torch.float64, device=s.device)
            flags = torch.zeros(1, dtype=torch.int32, pin_memory=True)
            A.check(A.lbm_moments_async(s.handle, ctypes.c_void_p(rho.data_ptr()), ctypes.c_void_p(u.data_ptr()),
                                        ctypes.c_void_p(T.data_ptr())), "lbm_moments_async")
            A.check(A.lbm_health_async(s.handle, ctypes.c_void_p(flags.data_ptr())), "lbm_health_async")
            host_rho = torch.empty(rho.shape, dtype=torch.float64, pin_memory=True)
            host_rho.copy_(rho, non_blocking=True)
            job.event = torch.cuda.Event()
            job.event.record(self.stream)
        job.out = (rho, u, T)
        job.host_flags = flags
        job.host_rho = host_rho

    def run(self, trace, time_scale: float = 1.0):
        """Serve `trace` (arrival times scaled by time_scale) in real time; returns the finished jobs."""
        pending = collections.deque(sorted(trace, key=lambda r: r["arrival"]))
        waiting: collections.deque = collections.deque()
        active: list = []
        retiring: list = []
        done: list = []
        ticks: collections.deque = collections.deque()  # events of launched ticks
        used = 0
        pool = cf.ThreadPoolExecutor(max_workers=self.prep_workers)
        self._warm_workers(pool)
        t0 = time.perf_counter()

        def clock():
            return time.perf_counter() - t0

        try:
            while pending or waiting or active or retiring:
                h = time.perf_counter()
                while pending and pending[0]["arrival"] * time_scale <= clock():
                    r = pending.popleft()
                    waiting.append(Job(req=r, nbytes=workspace_bytes(r["grid"]),
                                       prep=pool.submit(prepare, r, 0, self.vn_device, self._note_prep)))
                # admission by the policy, footprint and batch slots, once prepared
                while len(active) < self.max_batch:
                    j = next_admission(waiting, used, self.budget, self.policy)
                    if j is None:
                        break
                    note_admission(waiting, j)
                    waiting.remove(j)
                    self._admit(j)
                    j.admitted = clock()
                    used += j.nbytes
                    active.append(j)
                if waiting and not active and not retiring:
                    big = next((j for j in waiting if j.nbytes > self.budget), None)
                    if big is not None:
                        raise RuntimeError(f"request {big.req['id']} exceeds the HBM budget")
                self.host_s["admit"] += time.perf_counter() - h
                self.peak_bytes = max(self.peak_bytes, used)
                self.peak_batch = max(self.peak_batch, len(active))
                # results that have reached the host free their workspace
                h = time.perf_counter()
                still = []
                for j in retiring:
                    if j.event.query():
                        j.finished = clock()
                        j.health = self._health(j)
                        if self.keep_results:
                            j.rho = j.host_rho.numpy()
                        j.sim.close()
                        j.sim, j.out, j.host_rho, j.fields = None, None, None, None
                        used -= j.nbytes
                        if j.health and j.attempt + 1 < ATTEMPTS:
                            # solve it again with the next parameter candidate, first in line
                            self.retries += 1
                            waiting.appendleft(Job(req=j.req, nbytes=j.nbytes, attempt=j.attempt + 1,
                                                   prep=pool.submit(prepare, j.req, j.attempt + 1, self.vn_device,
                                                                   self._note_prep)))
                        else:
                            done.append(j)
                    else:
                        still.append(j)
                retiring = still
                self.host_s["retire"] += time.perf_counter() - h
                if active:
                    # at most two ticks in flight: wait for the older one
                    h = time.perf_counter()
                    while len(ticks) >= 2:
                        ticks.popleft().synchronize()
                    self.host_s["wait_gpu"] += time.perf_counter() - h
                    h = time.perf_counter()
                    n = min(self.tick, min(j.remaining for j in active))
                    S.step_batch([j.sim for j in active], n)
                    self.launches += n
                    still = []
                    for j in active:
                        j.remaining -= n
                        if j.remaining > 0:
                            still.append(j)
                        else:
                            self._retire_start(j)
                            retiring.append(j)
                    active = still
                    ev = torch.cuda.Event()
                    ev.record(self.stream)
                    ticks.append(ev)
                    self.host_s["launch"] += time.perf_counter() - h
                    continue
                # nothing to step: wait for a retirement, a preparation or the next arrival
                h = time.perf_counter()
                if retiring:
                    retiring[0].event.synchronize()
                elif waiting:
                    cf.wait([j.prep for j in waiting], timeout=0.05, return_when=cf.FIRST_COMPLETED)
                elif pending:
                    time.sleep(max(0.0, min(0.05, pending[0]["arrival"] * time_scale - clock())))
                self.host_s["idle"] += time.perf_counter() - h
        finally:
            pool.shutdown(wait=True)
        self.wall = clock()
        return done


def summary(done, wall, time_scale=1.0):
    lat = np.array([j.finished - j.req["arrival"] * time_scale for j in done])
    queue = np.array([j.admitted - j.req["arrival"] * time_scale for j in done])
    cells = sum(int(np.prod(j.req["grid"])) * j.req["steps"] for j in done)
    return {
        "requests": len(done),
        "p50_latency_s": float(np.percentile(lat, 50)),
        "p99_latency_s": float(np.percentile(lat, 99)),
        "mean_latency_s": float(lat.mean()),
        "p50_queue_s": float(np.percentile(queue, 50)),
        "solves_per_s": len(done) / wall,
        "cell_updates_per_s": cells / wall,
        "wall_s": wall,
        "unhealthy": int(sum(1 for j in done if j.health)),
        "retried": int(sum(1 for j in done if j.attempt > 0)),
    }
