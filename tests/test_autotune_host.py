"""Autotuner cache logic on the host (the timing itself needs the GPU)."""
import json

from paper_1010_4135_gb300 import autotune


class FakeSim:
    def __init__(self, prec="fp32"):
        self.config = dict(nx=64, ny=32, nz=16, precision=prec, scheme="nnd", bc_lo=(1, 0, 0), bc_hi=(2, 0, 0))
        self.launch = None

    def set_launch(self, variant, zchunk):
        self.launch = (variant, zchunk)


def test_key_names_device_grid_precision_scheme_and_boundaries():
    k = autotune.key_of([FakeSim(), FakeSim()], True, device_name="NVIDIA GB300", sms=152)
    assert k == "NVIDIA_GB300|152|batch|tiled,tiled64|64x32x16:fp32:nnd:100200|64x32x16:fp32:nnd:100200"
    assert autotune.key_of([FakeSim()], False, "d", 1, variants=("tiled",)) != autotune.key_of([FakeSim()], False, "d", 1)
    assert autotune.key_of([FakeSim()], False, "d", 1) != autotune.key_of([FakeSim()], True, "d", 1)


def test_cached_choice_is_applied_without_measuring(tmp_path, monkeypatch):
    path = str(tmp_path / "launch.json")
    autotune._store(path, "K", {"variant": "tiled64", "zchunk": 24, "ms": 0.5, "timings": {"tiled64:24": 0.5}})
    monkeypatch.setattr(autotune, "measure", lambda *a, **k: (_ for _ in ()).throw(AssertionError("measured")))
    s = FakeSim()
    r = autotune._tune([s], autotune.ZCHUNKS, 10, True, path, batched=False, key="K")
    assert r["cached"] and r["zchunk"] == 24 and s.launch == ("tiled64", 24)


def test_fastest_candidate_is_chosen_and_stored(tmp_path, monkeypatch):
    path = str(tmp_path / "launch.json")
    monkeypatch.setattr(autotune, "measure", lambda sims, zcs, steps, batched, variants:
                        {("tiled", 4): 0.9, ("tiled", 16): 0.55, ("tiled64", 16): 0.5, ("tiled64", 32): 0.6})
    s = FakeSim()
    r = autotune._tune([s], (4, 16, 32), 10, True, path, batched=False, key="K2")
    assert not r["cached"] and (r["variant"], r["zchunk"]) == ("tiled64", 16) and s.launch == ("tiled64", 16)
    rec = json.load(open(path))["K2"]
    assert rec["zchunk"] == 16 and rec["variant"] == "tiled64" and rec["timings"]["tiled:4"] == 0.9


def test_fp64_sims_are_not_tuned(tmp_path):
    s = FakeSim("fp64")
    r = autotune._tune([s], autotune.ZCHUNKS, 10, True, str(tmp_path / "x.json"), batched=False, key="K")
    assert r["zchunk"] is None and s.launch is None
