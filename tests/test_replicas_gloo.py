"""The multi-GPU harness logic (barrier, max-over-ranks time, summed units)
as two gloo ranks on the CPU."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    from paper_1010_4135_gb300 import replicas
    r, w, local = replicas.init(backend="gloo")
    replicas.barrier()
    ms, units = replicas.aggregate(10.0 + rank, 1000 * (rank + 1))
    q.put((r, w, local, ms, units))
    replicas.finish()


def test_two_ranks_aggregate_max_time_and_total_units():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [o[0] for o in out] == [0, 1]
    for r, w, local, ms, units in out:
        assert w == 2 and local == r
        assert ms == pytest.approx(11.0) and units == pytest.approx(3000.0)


def test_single_process_is_a_pass_through():
    from paper_1010_4135_gb300 import replicas
    assert replicas.aggregate(3.5, 7) == (3.5, 7.0)
