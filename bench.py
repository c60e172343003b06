#!/usr/bin/env python3
"""Throughput benchmark of the D3V15 FD-LB solver on one GB300 (or N replicas).

Workload (default): the 256^3 Mach-2 shock-droplet grid (rho = 5 droplet of
radius 0.1 at (0.3, 0.5, 0.5), (c1, c2, eta0) = (2, 6, 4), dt = tau = 5e-5),
f stored and updated in FP32.  One bench step = one time step of the whole
path (boundary fill + fused moments / equilibrium / NND / dissipation / BGK /
update kernel, health flag).  Inputs are resident in HBM; the two f buffers
(2 x 1.0 GB) exceed the 129 MB L2, so no flush is needed between steps.

Prints one JSON line (rank 0).  `--impl reference` times the FP64 CPU oracle
on a bounded slab of the same workload instead.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "D3V15 cell-updates/s & % HBM roofline; served-solve p50/p99 at stated L1 error"
UNIT = "cell-updates/s"
FALLBACK_HBM_GBS = 6800.0


def parse():
    p = argparse.ArgumentParser(description=__doc__)
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=1000)
    p.add_argument("--warmup", type=int, default=10)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--precision", default="fp32", choices=["fp32", "fp64"])
    p.add_argument("--requests", type=int, default=200, help="serve: number of requests in the trace")
    p.add_argument("--rate", type=float, default=20.0, help="serve: mean arrival rate (requests/s)")
    p.add_argument("--hbm-budget-gb", type=float, default=0.0, help="serve: workspace budget (0 = 80%% of free)")
    p.add_argument("--policy", default="fifo", choices=["fifo", "sjf"], help="serve: admission order")
    p.add_argument("--l1-sample", type=float, default=0.1,
                   help="serve: fraction of the finished requests (seeded) checked against the FP64 path")
    p.add_argument("--serve-requests", type=int, default=30,
                   help="default line: requests of the compact serving summary (0 = none)")
    p.add_argument("--serve-rate", type=float, default=2.0,
                   help="default line: arrival rate of the compact serving summary (the sustainable rate)")
    p.add_argument("--workload", default="droplet", choices=["droplet", "bubble", "batch", "batch_small", "serve"],
                   help="droplet: 256^3 Mach-2 shock-droplet; bubble: 512x256x256 Mach-3 shock-bubble; "
                        "batch: the bubble grid plus 8 128^3 copies with seeded Mach numbers, one launch per "
                        "step, replayed as a CUDA graph; batch_small: the 8 128^3 copies alone (a profiling "
                        "size); serve: the seeded request stream through the continuous-batching server")
    p.add_argument("--cpu-steps", type=int, default=3, help="oracle steps of the CPU baseline sample")
    p.add_argument("--variant", default="tiled", choices=["tiled", "tiled64", "split", "tiled_fill", "tiled_single", "plain"], help="FP32 step kernel")
    p.add_argument("--zchunk", type=int, default=0, help="z planes per CTA of the tiled kernel (0 = auto)")
    p.add_argument("--ztail", type=int, default=0,
                   help="with --zchunk: short chunks of this many planes end each tile column (0 = none)")
    p.add_argument("--no-cpu", action="store_true")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-accuracy", action="store_true",
                   help="skip the FP64 reference run behind the line's accuracy object")
    return p.parse_args()


def workload(name):
    import workloads
    if name == "droplet":
        return workloads.shock_droplet(256)
    return workloads.shock_bubble()


def batch_workloads(small=False):
    """The 512x256x256 Mach-3 bubble and 8 128^3 bubbles whose Mach numbers
    are drawn (seed 4) uniformly in [1.5, 6]; (c1, c2, eta0, dt) of each from
    the von Neumann parameter rule (paper_1010_4135_gb300.stability) applied
    to the initial states and to the star states of the shock meeting the
    bubble.  small: the eight 128^3 bubbles alone."""
    import workloads
    from paper_1010_4135_gb300 import stability
    out = []
    big = [] if small else [((512, 256, 256), 3.0)]
    for n, mach in big + [((128, 128, 128), float(m)) for m in workloads.batch_machs(4, 8)]:
        r2, u2, p2, _ = workloads.rankine_hugoniot(mach)
        post, bubble = (r2, u2, 0.0, 0.0, p2 / r2), (0.1, 0.0, 0.0, 0.0, 10.0)
        states = [(1.0, 0.0, 0.0, 0.0, 1.0), post, bubble, *stability.interaction_states(post, bubble)]
        c1, c2, eta0, dt = stability.choose_parameters(states, 1.0 / n[1])
        w = workloads.shock_bubble(*n, mach=mach, c=(c1, c2, eta0), dt=dt)
        w.name = f"shock_bubble_{n[0]}x{n[1]}x{n[2]}_mach{mach:.2f}"
        out.append(w)
    return out


def run_batch(args):
    """One step = one batched launch advancing all grids of the batch; the
    timed steps replay a captured CUDA graph of `graph_steps` steps."""
    import torch
    from paper_1010_4135_gb300 import sim as S
    torch.cuda.set_device(0)
    ws = batch_workloads(small=args.workload == "batch_small")
    sims = []
    for w in ws:
        s = S.from_workload(w, precision="fp32")
        rho, u, T = w.initial_fields()
        s.init(rho, u, T)
        sims.append(s)
    cells = sum(w.ncell for w in ws)
    from paper_1010_4135_gb300 import autotune
    if args.zchunk == 0:
        tuned = autotune.tune_batch(sims)
    else:
        tuned = {"variant": args.variant if args.variant in ("tiled", "tiled64") else "tiled", "zchunk": args.zchunk,
                 "ztail": args.ztail}
    for s in sims:
        s.set_launch(tuned["variant"], tuned["zchunk"], tuned["ztail"])
    S.step_batch(sims, max(2, args.warmup))
    gsteps = 10 if args.steps % 10 == 0 else 2
    steps = max(gsteps, args.steps - args.steps % gsteps)
    g = S.Graph(sims, gsteps)
    g.launch(1)
    torch.cuda.synchronize()
    # the timed region lasts at least 1.2 s, so that the 200 ms clock samples
    # number at least five
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(sims[0].stream)
    g.launch(1)
    e1.record(sims[0].stream)
    e1.synchronize()
    per_step_est = e0.elapsed_time(e1) / gsteps
    steps = max(steps, gsteps * int(-(-1200.0 // (per_step_est * gsteps))))
    clocks = ClockSampler(gpu_smi_id(torch, 0))
    time.sleep(0.5)
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    t0 = time.time()
    ev0.record(sims[0].stream)
    g.launch(steps // gsteps)
    ev1.record(sims[0].stream)
    ev1.synchronize()
    t1 = time.time()
    ms = ev0.elapsed_time(ev1)
    clock = clocks.summary(t0, t1)
    clocks.stop()
    health = [s.health() for s in sims]
    accuracy = None
    if not args.no_accuracy:
        accuracy = []
        for w, s in zip(ws, sims):
            r32, _, _ = s.moments()
            accuracy.append(fp32_accuracy(w, r32, s.steps_done))
    peak, peak_kind = measured_peak()
    alg = 120.0 * cells
    per_step = ms * 1e-3 / steps
    line = {
        "metric": METRIC, "value": cells * steps / (ms * 1e-3), "unit": UNIT, "n_gpus": 1, "steps": steps,
        "warmup": args.warmup, "ms_per_step": ms / steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": "batch: " + ", ".join(w.name for w in ws), "cells": cells,
                   "c1_c2_eta0_dt": [[w.c1, w.c2, w.eta0, w.dt] for w in ws],
                   "launch": f"one persistent batched step kernel per step, CUDA graph of {gsteps} steps",
                   "variant": tuned["variant"], "zchunk": tuned["zchunk"], "ztail": tuned["ztail"],
                   "autotuned": args.zchunk == 0,
                   "tune_timings_ms": tuned.get("timings"),
                   "l2": "no flush: the f buffers (0.13-2.0 GB each) exceed the L2 together"},
        "roofline": {"bound": "hbm", "achieved": alg / per_step / 1e9, "peak": peak, "unit": "GB/s",
                     "frac": alg / per_step / 1e9 / peak, "peak_source": peak_kind,
                     "kernel": "step_pair_batch (all grids, one launch per step; time per step incl. graph gaps)",
                     "traffic": None},
        "accuracy": accuracy,
        "gpu_launches": steps, "clocks": clock, "health_flags": health,
    }
    print(json.dumps(line), flush=True)
    return 0


def fp32_accuracy(w, r32, steps):
    """L1 / Linf relative density error of an FP32 result after `steps`
    steps against the FP64 path run alone from the same initial fields (the
    FP64 path equals the oracle to 1e-12 on the parity cases and on one
    full-size step of the benchmarked grids)."""
    import numpy as np
    from paper_1010_4135_gb300 import sim as S
    s64 = S.from_workload(w, precision="fp64")
    rho, u, T = w.initial_fields()
    s64.init(rho, u, T)
    s64.step(steps)
    r64, _, _ = s64.moments()
    s64.close()
    r32 = np.asarray(r32, dtype=np.float64).reshape(r64.shape)
    return {"grid": w.name, "steps": int(steps), "vs": "fp64 path",
            "l1_rho": float(np.abs(r32 - r64).sum() / np.abs(r64).sum()),
            "linf_rho": float(np.abs(r32 - r64).max() / np.abs(r64).max())}


def describe(w, precision):
    return {
        "workload": w.name + (" (Mach %.0f shock, sphere rho=%g r=%g at %s)" % (
            w.meta["mach"], w.meta["sphere"][0], w.meta["radius"], tuple(w.meta["centre"]))),
        "grid": [w.nx, w.ny, w.nz],
        "cells": w.ncell,
        "precision": precision + " f" + (" storage and update; conservation sums in double-float per block, "
                                           "combined in fp64" if precision == "fp32" else ""),
        "scheme": "NND + extra dissipation, BGK, forward Euler",
        "c1_c2_eta0": [w.c1, w.c2, w.eta0],
        "dt": w.dt, "tau": w.tau, "dx": w.dx,
        "boundaries": "x: fixed post-shock inflow / extrapolated outflow; y, z: periodic",
        "l2": "no flush: the two f buffers exceed the 129 MB L2",
        "parallelism": "replicas",
    }


# ------------------------------------------------------------------ helpers

def measured_peak():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            return float(json.load(fh)["hbm_gbs"]), "of measured"
    except Exception:
        return FALLBACK_HBM_GBS, "of fallback"


# sources of each profiled kernel: its recorded DRAM traffic is used only while
# these files are unchanged
KERNEL_SOURCES = {
    "step_fp32": ("k_pair.cu", "pair_math.cuh", "tma_ring.cuh", "lbm_internal.cuh"),
    "step_fp64": ("k_plain.cu", "lbm_internal.cuh"),
}


def kernel_source_hash(key="step_fp32"):
    """Hash of the kernel's code: the token sequence of its source files
    without comments (a comment edit or a re-wrapped line does not change
    what ncu measured)."""
    import re
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_1010_4135_gb300", "csrc")
    for fn in KERNEL_SOURCES[key]:
        with open(os.path.join(csrc, fn)) as fh:
            text = re.sub(r"/\*.*?\*/", "", fh.read(), flags=re.S)
        code = "\n".join(ln.split("//", 1)[0] for ln in text.splitlines())
        h.update(fn.encode())
        h.update(" ".join(re.findall(r"\w+|[^\w\s]", code)).encode())
    return h.hexdigest()[:16]


def recorded_traffic(kernel_key, precision, cells):
    """DRAM bytes per launch from the committed ncu summary, if it was taken
    from the current kernel sources (else None)."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as fh:
            rec = json.load(fh)
    except Exception:
        return None
    key = f"{kernel_key}_{precision}"
    e = rec.get(key)
    if not e or key not in KERNEL_SOURCES or e.get("source_hash") != kernel_source_hash(key):
        return None
    return float(e["dram_bytes_per_cell"]) * cells


class ClockSampler:
    """nvidia-smi clock / throttle-reason samples every 200 ms."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id):
        self.samples = []
        self.proc = None
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(gpu_id), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.samples.append((time.time(), line.strip()))

    def stop(self):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self, t0, t1):
        rows = []
        for ts, line in self.samples:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            rows.append((ts, parts))
        inside = [r for r in rows if t0 <= r[0] <= t1]
        if not inside and rows:  # short timed region: the samples closest to it
            mid = 0.5 * (t0 + t1)
            inside = sorted(rows, key=lambda r: abs(r[0] - mid))[:2]
        if not inside:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no nvidia-smi samples"], "samples": 0}

        def num(x):
            try:
                return float(x)
            except ValueError:
                return None
        sm = [num(p[1]) for _, p in inside if num(p[1]) is not None]
        mx = [num(p[2]) for _, p in inside if num(p[2]) is not None]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for _, p in inside for k in range(4) if p[5 + k].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(inside),
                "power_w_max": max((num(p[3]) or 0.0) for _, p in inside)}


def gpu_smi_id(torch, dev):
    try:
        u = str(torch.cuda.get_device_properties(dev).uuid)
        return u if u.startswith("GPU-") else "GPU-" + u
    except Exception:
        return dev


# ---------------------------------------------------------------- CPU oracle

def cpu_oracle_rate(w, steps, nz_slab=None, nthreads=None):
    """cell-updates/s of the FP64 oracle on the same workload (optionally a z-slab
    of nz_slab planes with the workload's x/y extent and boundaries), on
    nthreads threads (default: all host cores)."""
    import numpy as np
    import oracle
    ww = w if nz_slab is None else w.with_grid(w.nx, w.ny, nz_slab, dx=w.dx)
    cfg = oracle.cfg_for(ww)
    rho, u, T = ww.initial_fields()
    f = oracle.init(cfg, rho, u, T)
    del rho, u, T
    nthreads = nthreads or os.cpu_count() or 1
    t0 = time.perf_counter()
    f = oracle.run(cfg, f, steps, nthreads)
    dt = time.perf_counter() - t0
    assert np.isfinite(f[0, 0, 0, 0])
    return ww.ncell * steps / dt, nthreads, ww, dt


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    w = workload(args.workload)
    # each step a z-slab sized so that warmup + steps stay within ~2 minutes
    probe_nz = 4
    rate, cores, _, _ = cpu_oracle_rate(w, 1, probe_nz)
    budget = 120.0
    per_plane = w.nx * w.ny / rate
    nz = int(max(2, min(w.nz, budget / max(1, args.steps + args.warmup) / per_plane)))
    if args.warmup:
        cpu_oracle_rate(w, args.warmup, nz)
    rate, cores, ww, dt = cpu_oracle_rate(w, args.steps, nz)
    sample = (f"{args.steps} oracle steps of a {ww.nx}x{ww.ny}x{nz} slab of the {w.name} workload "
              f"(same x/y extent, boundaries and constants), FP64, {cores} threads")
    line = {
        "impl": "reference", "metric": METRIC, "value": rate, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / max(1, args.steps),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": describe(w, "fp64"),
        "cpu_baseline": {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": rate, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# -------------------------------------------------------------------- GPU run

def run_ours(args):
    import numpy as np
    import torch

    from paper_1010_4135_gb300 import replicas
    rank, world, local = replicas.env_ranks()
    if world > 1:
        torch.cuda.set_device(local)
        replicas.init("nccl", device=torch.device("cuda", local))
    else:
        torch.cuda.set_device(0)
    dev = torch.cuda.current_device()

    from paper_1010_4135_gb300 import sim as S
    w = workload(args.workload)
    rho, u, T = w.initial_fields()
    s = S.from_workload(w, precision=args.precision)
    s.set_launch(args.variant, args.zchunk, args.ztail)
    s.init(rho, u, T)
    tuned = None
    if args.precision == "fp32" and args.variant in ("tiled", "tiled64") and args.zchunk == 0:
        from paper_1010_4135_gb300 import autotune
        tuned = autotune.tune(s)  # z chunk measured on a scratch copy of this state

    def barrier():
        torch.cuda.synchronize()
        replicas.barrier()
        torch.cuda.synchronize()

    s.step(args.warmup)
    s.sync()
    clocks = ClockSampler(gpu_smi_id(torch, dev)) if rank == 0 else None
    time.sleep(0.5 if clocks else 0.0)
    s.set_timing(True)
    s.timing(reset=True)
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    barrier()
    t0 = time.time()
    ev0.record(s.stream)
    s.step(args.steps)
    ev1.record(s.stream)
    ev1.synchronize()
    t1 = time.time()
    barrier()
    ms = ev0.elapsed_time(ev1)
    per_kernel = s.timing(reset=True)
    s.set_timing(False)
    health = s.health()
    ms_max, total_cells = replicas.aggregate(ms, w.ncell * args.steps, device=torch.device("cuda", dev))
    clock = clocks.summary(t0, t1) if clocks else None
    if clocks:
        clocks.stop()
    value = total_cells / (ms_max * 1e-3)

    # conservation sums of the final state (FP64, deterministic reduction)
    cons = s.conserved(check_health=False).tolist()

    # end to end through the C ABI with host buffers: init from pinned host
    # memory, the same number of steps, moments back to pinned host memory
    e2e = None
    if not args.no_e2e:
        hr = torch.from_numpy(rho).pin_memory()
        hu = torch.from_numpy(np.ascontiguousarray(u)).pin_memory()
        hT = torch.from_numpy(T).pin_memory()
        orho = torch.empty_like(hr).pin_memory()
        ou = torch.empty_like(hu).pin_memory()
        oT = torch.empty_like(hT).pin_memory()
        import ctypes
        from paper_1010_4135_gb300 import _abi as A

        def e2e_pass(nsteps):
            A.check(A.lbm_init(s.handle, ctypes.c_void_p(hr.data_ptr()), ctypes.c_void_p(hu.data_ptr()),
                               ctypes.c_void_p(hT.data_ptr()), 0), "lbm_init")
            A.check(A.lbm_step(s.handle, nsteps), "lbm_step")
            A.check(A.lbm_moments(s.handle, ctypes.c_void_p(orho.data_ptr()), ctypes.c_void_p(ou.data_ptr()),
                                  ctypes.c_void_p(oT.data_ptr()), 0), "lbm_moments")

        # one untimed pass (the warm-up step count): the first transfers from
        # freshly pinned buffers map their pages and ran at a fraction of the
        # link's rate
        e2e_pass(args.warmup)
        barrier()
        t0e = time.perf_counter()
        e2e_pass(args.steps)
        te = time.perf_counter() - t0e
        te, _ = replicas.aggregate(te, 0, device=torch.device("cuda", dev))
        io = (hr.numel() + hu.numel() + hT.numel()) * 8
        e2e = {"value": total_cells / te, "unit": UNIT,
               "h2d_bytes_per_step": io / args.steps, "d2h_bytes_per_step": io / args.steps,
               "note": "per run: lbm_init from pinned host (rho,u,T) + steps + lbm_moments to pinned host, "
                       "after one untimed pass of the same sequence with the warm-up step count"}

    # FP32 density error of a run of args.steps steps against the FP64 path
    accuracy = None
    if not args.no_accuracy and args.precision == "fp32" and rank == 0:
        if e2e is not None:
            r32 = orho.numpy()  # the end-to-end run: init, args.steps steps, moments
        else:
            s.init(rho, u, T)
            s.step(args.steps)
            r32, _, _ = s.moments()
        accuracy = fp32_accuracy(w, r32, args.steps)
        accuracy["metric"] = "L1 = sum|rho32 - rho64| / sum|rho64|; Linf = max|rho32 - rho64| / max|rho64|"

    if rank != 0:
        replicas.finish()
        return 0

    step_ms, step_n = per_kernel["step"]
    fill_ms, fill_n = per_kernel["fill"]
    esz = 4 if args.precision == "fp32" else 8
    alg_bytes = 2 * 15 * esz * w.ncell
    avg_step_s = step_ms * 1e-3 / max(1, step_n)
    peak, peak_kind = measured_peak()
    achieved = alg_bytes / avg_step_s / 1e9
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "peak_source": peak_kind, "kernel": f"step ({args.precision}, {s.launch[0] if args.precision == 'fp32' else 'plain'})",
                "algorithmic_bytes_per_launch": alg_bytes,
                "traffic": recorded_traffic("step", args.precision, w.ncell),
                "avg_launch_ms": avg_step_s * 1e3, "fill_avg_launch_ms": fill_ms / max(1, fill_n)}

    serving = None
    if args.serve_requests > 0 and world == 1 and args.precision == "fp32":
        s.close()
        torch.cuda.empty_cache()
        stats, srv, _, errors, sclock = serve_trace(args.serve_requests, args.serve_rate, "fifo", 0.1)
        serving = serving_summary(stats, errors, sclock, args.serve_requests, args.serve_rate, srv)

    cpu = None
    if not args.no_cpu and world == 1:
        rate, cores, ww, dt = cpu_oracle_rate(w, args.cpu_steps)
        rate1, _, ww1, dt1 = cpu_oracle_rate(w, 2, nz_slab=4, nthreads=1)
        cpu = {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": f"{args.cpu_steps} FP64 oracle steps of the full {w.nx}x{w.ny}x{w.nz} grid "
                         f"({dt:.1f} s)",
               "value_1thread": rate1,
               "sample_1thread": f"2 steps of a {ww1.nx}x{ww1.ny}x4 slab on 1 thread ({dt1:.1f} s)"}

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32" if args.precision == "fp32" else "f64", "data": "synthetic",
        "config": {**describe(w, args.precision),
                   "launch": {"variant": s.launch[0] if args.precision == "fp32" else "plain",
                              "zchunk": s.launch[1] if args.precision == "fp32" else None,
                              "ztail": s.launch[2] if args.precision == "fp32" else None,
                              "autotuned": tuned is not None,
                              "tune_timings_ms": tuned.get("timings") if tuned else None}},
        "roofline": roofline,
        "accuracy": accuracy,
        "serving": serving,
        "cpu_baseline": cpu,
        "e2e": e2e,
        "gpu_launches": int(step_n + fill_n) * world,
        "clocks": clock,
        "health_flags": health,
        "conserved_final": cons,
    }
    print(json.dumps(line), flush=True)
    replicas.finish()
    return 0


def serve_trace(requests, rate, policy="fifo", l1_frac=0.1, budget=None, seed=5):
    """The seeded Poisson request stream (`requests` arrivals at mean `rate`
    per second) through the continuous-batching server in real time, with
    nvidia-smi clocks sampled during it, and the L1 / Linf density error of a
    seeded fraction l1_frac of the finished requests against the FP64 path
    (parity-checked against the oracle).  Returns (summary, server, finished
    jobs, per-request errors, clocks)."""
    import numpy as np
    import torch
    import workloads
    from paper_1010_4135_gb300 import serve
    from paper_1010_4135_gb300 import sim as S
    trace = workloads.serving_trace(seed=seed, n=requests, rate=rate)
    srv = serve.Server(hbm_budget=budget, tick=50, keep_results=True, policy=policy)
    srv.tune_shapes(workloads.SERVING_GRIDS)  # before the trace starts: the server's grid menu
    clocks = ClockSampler(gpu_smi_id(torch, torch.cuda.current_device()))
    t0 = time.time()
    done = srv.run(trace)
    t1 = time.time()
    clock = clocks.summary(t0, t1)
    clocks.stop()
    stats = serve.summary(done, srv.wall)
    k = max(1, int(round(l1_frac * len(done))))
    pick = np.random.default_rng(11).choice(len(done), size=k, replace=False)
    errors = []
    for i in sorted(pick):
        j = done[i]
        w = workloads.request_workload(j.req, *j.params)
        s = S.from_workload(w, precision="fp64")
        rho, u, T = w.initial_fields()
        s.init(rho, u, T)
        s.step(j.req["steps"])
        r64, _, _ = s.moments()
        s.close()
        errors.append({"id": j.req["id"], "kind": j.req["kind"], "grid": list(j.req["grid"]), "steps": j.req["steps"],
                       "mach": j.req["mach"], "ratio": j.req["ratio"], "health": j.health,
                       "l1_rho": float(np.abs(j.rho - r64).sum() / np.abs(r64).sum()),
                       "linf_rho": float(np.abs(j.rho - r64).max() / np.abs(r64).max())})
    return stats, srv, done, errors, clock


def serving_summary(stats, errors, clock, requests, rate, srv):
    """The compact serving object of a bench line."""
    l1 = [e["l1_rho"] for e in errors]
    linf = [e["linf_rho"] for e in errors]
    return {"trace": f"{requests} requests, Poisson rate {rate}/s (seed 5), grids 64^3..256^3, Mach U[1.2,10], "
                     "density ratio log-U[0.1,10], 500-3000 steps, FP32",
            "admission": srv.policy, "p50_latency_s": stats["p50_latency_s"], "p99_latency_s": stats["p99_latency_s"],
            "solves_per_s": stats["solves_per_s"], "cell_updates_per_s": stats["cell_updates_per_s"],
            "unhealthy": stats["unhealthy"], "retried": stats["retried"],
            "l1_rho_vs_fp64": {"sample": f"seeded {len(errors)} of {stats['requests']} finished requests",
                               "median": float(statistics.median(l1)), "max": max(l1),
                               "linf_max": max(linf)},
            "parameter_rule": "on the device (lbm_vn_max_growth)" if srv.vn_device else "on the host",
            "preparation_s_per_request": {k: v / max(1, srv.prep_s.get("requests", 0))
                                          for k, v in srv.prep_s.items() if k != "requests"},
            "clocks": clock}


def run_serve(args):
    """The seeded Poisson request stream served in real time; reports latency
    percentiles, throughput, clocks and the L1 density error of a seeded
    sample of requests against the FP64 path (parity-checked against the
    oracle)."""
    import torch
    torch.cuda.set_device(0)
    budget = int(args.hbm_budget_gb * 2 ** 30) if args.hbm_budget_gb > 0 else None
    frac = args.l1_sample if args.l1_sample > 0 else 0.1
    stats, srv, done, l1, clock = serve_trace(args.requests, args.rate, args.policy, frac, budget)
    line = {
        "metric": METRIC, "value": stats["cell_updates_per_s"], "unit": UNIT, "n_gpus": 1,
        "steps": int(sum(j.req["steps"] for j in done)), "warmup": 0,
        "ms_per_step": None, "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": f"serving: {args.requests} requests, Poisson rate {args.rate}/s (seed 5), grids "
                               "64^3..256^3, Mach U[1.2,10], density ratio log-U[0.1,10], 500-3000 steps, FP32",
                   "admission": srv.policy, "hbm_budget_bytes": srv.budget, "peak_resident_bytes": srv.peak_bytes,
                   "peak_batch": srv.peak_batch, "host_seconds": dict(srv.host_s),
                   "preparation_seconds": dict(srv.prep_s),
                   "parameter_rule": "on the device (lbm_vn_max_growth)" if srv.vn_device else "on the host",
                   "l1_sample": f"seeded {frac:.0%} of the finished requests"},
        "serving": stats, "l1_vs_fp64_sample": l1, "gpu_launches": srv.launches, "clocks": clock,
        "unhealthy_requests": [{"id": j.req["id"], "kind": j.req["kind"], "grid": list(j.req["grid"]),
                                "mach": j.req["mach"], "ratio": j.req["ratio"], "c1_c2_eta0_dt": list(j.params),
                                "health": j.health} for j in done if j.health],
    }
    print(json.dumps(line), flush=True)
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload in ("batch", "batch_small"):
        return run_batch(args)
    if args.workload == "serve":
        return run_serve(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
