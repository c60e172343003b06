"""Launch-configuration autotuner of the FP32 step.

The knobs are the tile shape of the pair kernel ("tiled": 32 x 8 tiles, two
CTAs of 4 warps per SM; "tiled64": 64 x 8 tiles, one CTA of 8 warps per SM),
its z chunk (planes one CTA marches) and the tail chunk: long chunks re-read
fewer boundary planes and pay fewer unit prologues, short chunks fill the SMs;
a tail of short chunks at the end of each column (launched last) lets the SMs
run out of work together (256^3 on GB300: 0.474 ms per step with 24-plane
chunks, 0.464 ms with 32-plane chunks ending in 8-plane ones).  The best
choice depends on the grid's shape and the SM count, so it is measured: each candidate runs a few steps of the sim's own
state on a scratch copy of the sim (its own workspace, so the user's state
and step count are untouched), timed with CUDA events on the scratch sim's
stream; the fastest is applied and cached per (device, grid, precision,
scheme, boundary kinds) in a JSON file (LBM_TUNE_CACHE, default
~/.cache/paper_1010_4135_gb300/launch.json), so each shape is tuned once.
FP64 sims always use the plain kernel and are not tuned.
"""
from __future__ import annotations

import json
import os
import threading

import torch

ZCHUNKS = (4, 8, 12, 16, 24, 32, 48)
ZTAILS = (0, 8, 16)  # 0: equal chunks; a tail length is tried only below the chunk length
VARIANTS = ("tiled", "tiled64")
_lock = threading.Lock()


def cache_path() -> str:
    return os.environ.get("LBM_TUNE_CACHE") or os.path.join(
        os.path.expanduser("~"), ".cache", "paper_1010_4135_gb300", "launch.json")


def _load(path):
    try:
        with open(path) as fh:
            return json.load(fh)
    except (OSError, ValueError):
        return {}


def _store(path, key, value):
    with _lock:
        data = _load(path)
        data[key] = value
        os.makedirs(os.path.dirname(path) or ".", exist_ok=True)
        tmp = f"{path}.tmp{os.getpid()}"
        with open(tmp, "w") as fh:
            json.dump(data, fh, indent=1, sort_keys=True)
        os.replace(tmp, path)


def key_of(sims, batched: bool, device_name: str | None = None, sms: int | None = None,
           variants=None) -> str:
    """Cache key: device, SM count, the candidate tile shapes and tail lengths,
    and per sim the grid, precision, scheme and boundary kinds."""
    if device_name is None or sms is None:
        props = torch.cuda.get_device_properties(sims[0].device)
        device_name, sms = props.name, props.multi_processor_count
    parts = [device_name.replace(" ", "_"), str(int(sms)), "batch" if batched else "single",
             ",".join(variants or VARIANTS), "tails" + ",".join(str(t) for t in ZTAILS)]
    for s in sims:
        c = s.config
        parts.append("x".join(str(int(v)) for v in (c["nx"], c["ny"], c["nz"])) + f":{c['precision']}:{c['scheme']}:"
                     + "".join(str(int(k)) for k in tuple(c["bc_lo"]) + tuple(c["bc_hi"])))
    return "|".join(parts)


def _time(run, steps: int, warmup: int) -> float:
    run(warmup)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    run(steps)
    e1.record()
    e1.synchronize()
    return e0.elapsed_time(e1) / steps


def candidates(zchunks=ZCHUNKS, variants=VARIANTS) -> list:
    """(variant, zchunk, ztail) launches to measure: every tile shape and z
    chunk with equal chunks, and with each tail length below the chunk."""
    return [(v, int(zc), int(zt)) for v in variants for zc in zchunks for zt in ZTAILS if not zt or zt < zc]


def measure(sims, zchunks=ZCHUNKS, steps: int = 10, warmup: int = 2, batched: bool = False,
            variants=VARIANTS) -> dict:
    """{(variant, zchunk, ztail): ms per step} of the given sims' current states on scratch copies."""
    from . import sim as S
    scratch = []
    try:
        with torch.cuda.stream(torch.cuda.Stream(device=sims[0].device)):
            for s in sims:
                f = torch.empty((15,) + s.shape, dtype=torch.float32, device=s.device)
                s.sync()
                s.get_f(out=f)
                s.sync()
                c = s.clone(stream=torch.cuda.current_stream(s.device))
                scratch.append((c, f))
            out = {}
            for v, zc, zt in candidates(zchunks, variants):
                for c, f in scratch:
                    c.set_launch(v, zc, zt)
                    c.set_f(f)
                if batched:
                    run = lambda n: S.step_batch([c for c, _ in scratch], n)
                else:
                    run = scratch[0][0].step
                out[(v, zc, zt)] = _time(run, steps, warmup)
            return out
    finally:
        for c, _ in scratch:
            c.close()


def tune(sim, zchunks=ZCHUNKS, steps: int = 10, use_cache: bool = True, path: str | None = None,
         variants=VARIANTS) -> dict:
    """Choose and apply the tile shape, z chunk and tail of one FP32 sim;
    returns {"variant", "zchunk", "ztail", "ms", "cached", "timings"}."""
    return _tune([sim], zchunks, steps, use_cache, path, batched=False, variants=variants)


def tune_batch(sims, zchunks=ZCHUNKS, steps: int = 10, use_cache: bool = True, path: str | None = None,
               variants=VARIANTS) -> dict:
    """Choose and apply one tile shape, z chunk and tail for sims stepped together (lbm_step_batch)."""
    return _tune(list(sims), zchunks, steps, use_cache, path, batched=True, variants=variants)


def _tune(sims, zchunks, steps, use_cache, path, batched, key=None, variants=VARIANTS):
    if any(s.config["precision"] not in ("fp32", 1) for s in sims):
        return {"variant": None, "zchunk": None, "ztail": None, "ms": None, "cached": False, "timings": {}}
    path = path or cache_path()
    key = key or key_of(sims, batched, variants=variants)
    hit = _load(path).get(key) if use_cache else None
    if hit is not None:
        for s in sims:
            s.set_launch(hit["variant"], int(hit["zchunk"]), int(hit.get("ztail", 0)))
        return {**hit, "cached": True}
    timings = measure(sims, zchunks, steps, batched=batched, variants=variants)
    best = min(timings, key=timings.get)
    for s in sims:
        s.set_launch(*best)
    rec = {"variant": best[0], "zchunk": best[1], "ztail": best[2], "ms": timings[best],
           "timings": {f"{v}:{z}:{t}": ms for (v, z, t), ms in timings.items()}}
    _store(path, key, rec)
    return {**rec, "cached": False}
