"""The autotuner on the GPU: it measures every candidate on a scratch copy,
leaves the tuned sim's state and step count alone, and the chosen launch
gives bitwise the same results (the z chunk only reorders work)."""
import numpy as np
import pytest

from parity_util import case_cfg, initial_f, sim_for

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def test_tune_measures_applies_and_caches(tmp_path):
    from paper_1010_4135_gb300 import autotune
    cfg = case_cfg("fixed_extrap_reflect_33x17x9")
    f0 = initial_f(cfg, seed=80).astype(np.float32)
    a = sim_for(cfg, "fp32")
    a.set_f(f0)
    a.step(3)
    before = a.get_f()
    path = str(tmp_path / "launch.json")
    r = autotune.tune(a, zchunks=(2, 4, 9), steps=4, path=path)
    # chunks 2, 4, 9 with equal chunks, and 9 with a tail of 8: four launches per tile shape
    assert not r["cached"] and r["zchunk"] in (2, 4, 9) and len(r["timings"]) == 8
    assert a.launch == (r["variant"], r["zchunk"], r["ztail"]) and a.steps_done == 3
    assert np.array_equal(a.get_f(), before)
    a.step(5)
    b = sim_for(cfg, "fp32")
    b.set_f(f0)
    b.step(8)
    assert np.array_equal(a.get_f(), b.get_f())
    r2 = autotune.tune(a, zchunks=(2, 4, 9), path=path)
    assert r2["cached"] and r2["zchunk"] == r["zchunk"]


def test_tune_batch_applies_one_chunk_to_all(tmp_path):
    from paper_1010_4135_gb300 import autotune, sim as S
    sims = []
    for k, name in enumerate(("periodic_37x19x11", "fixed_extrap_reflect_33x17x9")):
        cfg = case_cfg(name)
        s = sim_for(cfg, "fp32")
        s.set_f(initial_f(cfg, seed=81 + k).astype(np.float32))
        sims.append(s)
    r = autotune.tune_batch(sims, zchunks=(3, 8), steps=4, path=str(tmp_path / "b.json"))
    assert r["zchunk"] in (3, 8) and all(s.launch == (r["variant"], r["zchunk"], r["ztail"]) for s in sims)
    S.step_batch(sims, 2)
    assert all(s.health() == 0 for s in sims)
