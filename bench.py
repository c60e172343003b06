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
    p.add_argument("--workload", default="droplet", choices=["droplet", "bubble"])
    p.add_argument("--cpu-steps", type=int, default=3, help="oracle steps of the CPU baseline sample")
    p.add_argument("--variant", default="tiled", choices=["tiled", "plain"], help="FP32 step kernel")
    p.add_argument("--zchunk", type=int, default=0, help="z planes per CTA of the tiled kernel (0 = auto)")
    p.add_argument("--no-cpu", action="store_true")
    p.add_argument("--no-e2e", action="store_true")
    return p.parse_args()


def workload(name):
    import workloads
    return workloads.shock_droplet(256) if name == "droplet" else workloads.shock_bubble()


def describe(w, precision):
    return {
        "workload": w.name + (" (Mach %.0f shock, sphere rho=%g r=%g at %s)" % (
            w.meta["mach"], w.meta["sphere"][0], w.meta["radius"], tuple(w.meta["centre"]))),
        "grid": [w.nx, w.ny, w.nz],
        "cells": w.ncell,
        "precision": precision + " f" + (", fp64 boundary fill / moments / conservation sums" if precision == "fp32" else ""),
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


def kernel_source_hash():
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_1010_4135_gb300", "csrc")
    for fn in sorted(os.listdir(csrc)):
        if fn.endswith((".cu", ".cuh")):
            with open(os.path.join(csrc, fn), "rb") as fh:
                h.update(fn.encode())
                h.update(fh.read())
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
    e = rec.get(f"{kernel_key}_{precision}")
    if not e or e.get("source_hash") != kernel_source_hash():
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

def cpu_oracle_rate(w, steps, nz_slab=None):
    """cell-updates/s of the FP64 oracle on the same workload (optionally a z-slab
    of nz_slab planes with the workload's x/y extent and boundaries)."""
    import numpy as np
    import oracle
    ww = w if nz_slab is None else w.with_grid(w.nx, w.ny, nz_slab, dx=w.dx)
    cfg = oracle.cfg_for(ww)
    rho, u, T = ww.initial_fields()
    f = oracle.init(cfg, rho, u, T)
    del rho, u, T
    nthreads = os.cpu_count() or 1
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

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        torch.cuda.set_device(0)
    dev = torch.cuda.current_device()

    from paper_1010_4135_gb300 import sim as S
    w = workload(args.workload)
    rho, u, T = w.initial_fields()
    s = S.from_workload(w, precision=args.precision)
    s.set_launch(args.variant, args.zchunk)
    s.init(rho, u, T)

    def barrier():
        torch.cuda.synchronize()
        if dist is not None:
            dist.barrier()
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
    ms_max = ms
    if dist is not None:
        t = torch.tensor([ms], device="cuda", dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms_max = float(t.item())
    clock = clocks.summary(t0, t1) if clocks else None
    if clocks:
        clocks.stop()
    total_cells = w.ncell * args.steps * world
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
        barrier()
        t0e = time.perf_counter()
        A.check(A.lbm_init(s.handle, ctypes.c_void_p(hr.data_ptr()), ctypes.c_void_p(hu.data_ptr()),
                           ctypes.c_void_p(hT.data_ptr()), 0), "lbm_init")
        A.check(A.lbm_step(s.handle, args.steps), "lbm_step")
        A.check(A.lbm_moments(s.handle, ctypes.c_void_p(orho.data_ptr()), ctypes.c_void_p(ou.data_ptr()),
                              ctypes.c_void_p(oT.data_ptr()), 0), "lbm_moments")
        te = time.perf_counter() - t0e
        if dist is not None:
            t = torch.tensor([te], device="cuda", dtype=torch.float64)
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            te = float(t.item())
        io = (hr.numel() + hu.numel() + hT.numel()) * 8
        e2e = {"value": total_cells / te, "unit": UNIT,
               "h2d_bytes_per_step": io / args.steps, "d2h_bytes_per_step": io / args.steps,
               "note": "per run: lbm_init from pinned host (rho,u,T) + steps + lbm_moments to pinned host"}

    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return 0

    step_ms, step_n = per_kernel["step"]
    fill_ms, fill_n = per_kernel["fill"]
    esz = 4 if args.precision == "fp32" else 8
    alg_bytes = 2 * 15 * esz * w.ncell
    avg_step_s = step_ms * 1e-3 / max(1, step_n)
    peak, peak_kind = measured_peak()
    achieved = alg_bytes / avg_step_s / 1e9
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "peak_source": peak_kind, "kernel": f"step ({args.precision}, {args.variant if args.precision == 'fp32' else 'plain'})",
                "algorithmic_bytes_per_launch": alg_bytes,
                "traffic": recorded_traffic("step", args.precision, w.ncell),
                "avg_launch_ms": avg_step_s * 1e3, "fill_avg_launch_ms": fill_ms / max(1, fill_n)}

    cpu = None
    if not args.no_cpu and world == 1:
        rate, cores, ww, dt = cpu_oracle_rate(w, args.cpu_steps)
        cpu = {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": f"{args.cpu_steps} FP64 oracle steps of the full {w.nx}x{w.ny}x{w.nz} grid "
                         f"({dt:.1f} s)"}

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32" if args.precision == "fp32" else "f64", "data": "synthetic",
        "config": describe(w, args.precision),
        "roofline": roofline,
        "cpu_baseline": cpu,
        "e2e": e2e,
        "gpu_launches": int(step_n + fill_n) * world,
        "clocks": clock,
        "health_flags": health,
        "conserved_final": cons,
    }
    print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
