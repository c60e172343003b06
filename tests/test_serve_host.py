"""Admission policies of the solve server, on the host (no GPU)."""
import collections
import dataclasses

import pytest

from paper_1010_4135_gb300 import serve


class Done:
    def __init__(self, ok=True):
        self.ok = ok

    def done(self):
        return self.ok


@dataclasses.dataclass
class J:
    req: dict
    nbytes: int
    attempt: int = 0
    prep: object = dataclasses.field(default_factory=Done)
    bypassed: int = 0


def _job(i, grid, steps, nbytes, attempt=0, ready=True):
    return J(req={"id": i, "grid": grid, "steps": steps}, nbytes=nbytes, attempt=attempt, prep=Done(ready))


def test_fifo_takes_the_head_only():
    q = collections.deque([_job(0, (64, 64, 64), 1000, 50), _job(1, (16, 16, 16), 10, 5)])
    assert serve.next_admission(q, used=0, budget=100, policy="fifo").req["id"] == 0
    # the head does not fit: nothing is admitted, the smaller one waits behind it
    assert serve.next_admission(q, used=60, budget=100, policy="fifo") is None
    q[0].prep.ok = False
    assert serve.next_admission(q, used=0, budget=100, policy="fifo") is None


def test_sjf_takes_the_least_work_that_fits_and_resolves_first():
    q = collections.deque([_job(0, (64, 64, 64), 1000, 50), _job(1, (32, 32, 32), 500, 20),
                           _job(2, (16, 16, 16), 100, 5, ready=False), _job(3, (32, 32, 32), 400, 20)])
    assert serve.next_admission(q, used=0, budget=100, policy="sjf").req["id"] == 3
    assert serve.next_admission(q, used=85, budget=100, policy="sjf") is None
    q.append(_job(4, (64, 64, 64), 3000, 50, attempt=1))
    assert serve.next_admission(q, used=0, budget=100, policy="sjf").req["id"] == 4
    # equal work: arrival order
    q2 = collections.deque([_job(5, (8, 8, 8), 10, 1), _job(6, (8, 8, 8), 10, 1)])
    assert serve.next_admission(q2, used=0, budget=10, policy="sjf").req["id"] == 5


def test_work_and_policy_names():
    assert serve.work({"grid": (4, 5, 6), "steps": 7}) == 840
    assert serve.POLICIES == ("fifo", "sjf")


def test_unknown_policy_is_rejected_before_any_device_work():
    with pytest.raises(ValueError):
        serve.Server(hbm_budget=1, policy="lifo")


def test_sjf_admits_a_big_job_within_a_bounded_number_of_admissions():
    """Small jobs keep arriving (one per admission round, two batch slots'
    worth of memory free): under SJF the big job that arrived first is
    overtaken at most MAX_BYPASS times, then admitted before any younger
    job; FIFO admits it first."""
    for policy, limit in (("sjf", serve.MAX_BYPASS), ("fifo", 0)):
        big = _job(0, (256, 256, 256), 3000, 60)
        q = collections.deque([big])
        admitted, rounds = [], 0
        while big not in admitted:
            rounds += 1
            assert rounds <= 4 * serve.MAX_BYPASS + 4, policy
            q.append(_job(rounds, (64, 64, 64), 500, 10))
            j = serve.next_admission(q, used=0, budget=100, policy=policy)
            assert j is not None
            serve.note_admission(q, j)
            q.remove(j)
            admitted.append(j)
        assert admitted.index(big) == limit, (policy, admitted.index(big))


def test_a_starved_job_blocks_younger_ones_until_it_fits():
    big = _job(0, (256, 256, 256), 3000, 60)
    big.bypassed = serve.MAX_BYPASS
    q = collections.deque([big, _job(1, (16, 16, 16), 10, 5)])
    # the small job would fit, but the starved one goes first: nothing until memory frees up
    assert serve.next_admission(q, used=50, budget=100, policy="sjf") is None
    assert serve.next_admission(q, used=0, budget=100, policy="sjf") is big
