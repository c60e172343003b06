"""Autotuner cache logic on the host (the timing itself needs the GPU)."""
import json

from paper_1010_4135_gb300 import autotune


class FakeSim:
    def __init__(self, prec="fp32"):
        self.config = dict(nx=64, ny=32, nz=16, precision=prec, scheme="nnd", bc_lo=(1, 0, 0), bc_hi=(2, 0, 0))
        self.launch = None

    def set_launch(self, variant, zchunk, ztail=0):
        self.launch = (variant, zchunk, ztail)


def test_key_names_device_grid_precision_scheme_and_boundaries():
    k = autotune.key_of([FakeSim(), FakeSim()], True, device_name="NVIDIA GB300", sms=152)
    assert k == ("NVIDIA_GB300|152|batch|tiled,tiled64|tails0,8,16|64x32x16:fp32:nnd:100200|"
                 "64x32x16:fp32:nnd:100200")
    assert autotune.key_of([FakeSim()], False, "d", 1, variants=("tiled",)) != autotune.key_of([FakeSim()], False, "d", 1)
    assert autotune.key_of([FakeSim()], False, "d", 1) != autotune.key_of([FakeSim()], True, "d", 1)


def test_cached_choice_is_applied_without_measuring(tmp_path, monkeypatch):
    path = str(tmp_path / "launch.json")
    autotune._store(path, "K", {"variant": "tiled64", "zchunk": 24, "ztail": 8, "ms": 0.5,
                                "timings": {"tiled64:24:8": 0.5}})
    autotune._store(path, "OLD", {"variant": "tiled", "zchunk": 16, "ms": 0.5, "timings": {"tiled:16": 0.5}})
    monkeypatch.setattr(autotune, "measure", lambda *a, **k: (_ for _ in ()).throw(AssertionError("measured")))
    s = FakeSim()
    r = autotune._tune([s], autotune.ZCHUNKS, 10, True, path, batched=False, key="K")
    assert r["cached"] and r["zchunk"] == 24 and s.launch == ("tiled64", 24, 8)
    autotune._tune([s], autotune.ZCHUNKS, 10, True, path, batched=False, key="OLD")
    assert s.launch == ("tiled", 16, 0)  # a record without a tail: equal chunks


def test_fastest_candidate_is_chosen_and_stored(tmp_path, monkeypatch):
    path = str(tmp_path / "launch.json")
    monkeypatch.setattr(autotune, "measure", lambda sims, zcs, steps, batched, variants:
                        {("tiled", 4, 0): 0.9, ("tiled", 16, 0): 0.55, ("tiled64", 16, 8): 0.5,
                         ("tiled64", 32, 0): 0.6})
    s = FakeSim()
    r = autotune._tune([s], (4, 16, 32), 10, True, path, batched=False, key="K2")
    assert not r["cached"] and (r["variant"], r["zchunk"], r["ztail"]) == ("tiled64", 16, 8)
    assert s.launch == ("tiled64", 16, 8)
    rec = json.load(open(path))["K2"]
    assert rec["zchunk"] == 16 and rec["ztail"] == 8 and rec["timings"]["tiled:4:0"] == 0.9


def test_fp64_sims_are_not_tuned(tmp_path):
    s = FakeSim("fp64")
    r = autotune._tune([s], autotune.ZCHUNKS, 10, True, str(tmp_path / "x.json"), batched=False, key="K")
    assert r["zchunk"] is None and s.launch is None


def test_candidates_try_tails_only_below_the_chunk_length():
    c = autotune.candidates((4, 8, 12, 24), ("tiled",))
    assert c == [("tiled", 4, 0), ("tiled", 8, 0), ("tiled", 12, 0), ("tiled", 12, 8),
                 ("tiled", 24, 0), ("tiled", 24, 8), ("tiled", 24, 16)]
    assert len(autotune.candidates()) == 2 * sum(1 + sum(1 for t in autotune.ZTAILS if t and t < z)
                                                 for z in autotune.ZCHUNKS)
