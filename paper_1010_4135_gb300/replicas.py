"""Replica bookkeeping for runs on several GPUs of one node.

The solver's grids are independent, so N GPUs run N replicas (one process
per GPU, launched by torch.distributed.run) with no collective on the data
path.  The only cross-rank traffic is the timing harness: a barrier around the
timed region, the maximum of the per-rank times, and the sum of the units
(cell updates) the ranks processed.
"""
from __future__ import annotations

import os

import torch
import torch.distributed as dist


def env_ranks():
    """(rank, world_size, local_rank) from the torch.distributed.run environment."""
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


def init(backend: str = "nccl", device=None):
    """Join the process group when running as one of several ranks."""
    rank, world, local = env_ranks()
    if world > 1 and not dist.is_initialized():
        if backend == "nccl":
            dist.init_process_group("nccl", device_id=device)
        else:
            dist.init_process_group(backend)
    return rank, world, local


def barrier():
    if dist.is_available() and dist.is_initialized():
        dist.barrier()


def aggregate(ms_local: float, units_local: float, device=None):
    """(max over ranks of ms_local, sum over ranks of units_local)."""
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(ms_local), float(units_local)
    dev = device if device is not None else torch.device("cpu")
    t = torch.tensor([float(ms_local)], dtype=torch.float64, device=dev)
    u = torch.tensor([float(units_local)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(t.item()), float(u.item())


def finish():
    if dist.is_available() and dist.is_initialized():
        dist.destroy_process_group()
