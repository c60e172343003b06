"""Host logic of bench.py (no GPU): the kernel-source hash that keys the
recorded DRAM traffic, the traffic lookup, and the clock summary of
nvidia-smi samples that decides whether a timed region is acceptable."""
import json
import os
import shutil

import pytest

import bench


@pytest.fixture()
def tree(tmp_path, monkeypatch):
    """A copy of the kernel sources and profiles/traffic.json under tmp_path,
    with bench.ROOT pointed at it."""
    src = os.path.join(bench.ROOT, "paper_1010_4135_gb300", "csrc")
    dst = tmp_path / "paper_1010_4135_gb300" / "csrc"
    dst.mkdir(parents=True)
    for files in bench.KERNEL_SOURCES.values():
        for fn in files:
            shutil.copy(os.path.join(src, fn), dst / fn)
    (tmp_path / "profiles").mkdir()
    shutil.copy(os.path.join(bench.ROOT, "profiles", "traffic.json"), tmp_path / "profiles" / "traffic.json")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    return dst


def test_source_hash_ignores_comments_and_wrapping_but_not_code(tree):
    h0, h64 = bench.kernel_source_hash("step_fp32"), bench.kernel_source_hash("step_fp64")
    p = tree / "k_pair.cu"
    text = p.read_text()
    assert "const int tid = threadIdx.x;" in text
    p.write_text("// a new leading comment\n/* and a block\n   comment */\n" +
                 text.replace("const int tid = threadIdx.x;", "const int tid =\n      threadIdx.x;  // re-wrapped", 1))
    assert bench.kernel_source_hash("step_fp32") == h0
    p.write_text(text.replace("2 * tx", "2 * tx + 0", 1))
    assert bench.kernel_source_hash("step_fp32") != h0
    # the FP64 kernel's sources do not include k_pair.cu
    assert bench.kernel_source_hash("step_fp64") == h64


def test_recorded_traffic_only_for_the_sources_it_was_taken_from(tree):
    rec = json.loads((tree.parent.parent / "profiles" / "traffic.json").read_text())
    cells = 1000
    got = bench.recorded_traffic("step", "fp32", cells)
    if rec["step_fp32"]["source_hash"] == bench.kernel_source_hash("step_fp32"):
        assert got == pytest.approx(rec["step_fp32"]["dram_bytes_per_cell"] * cells)
    p = tree / "k_pair.cu"
    p.write_text(p.read_text().replace("2 * tx", "2 * tx + 0", 1))
    assert bench.recorded_traffic("step", "fp32", cells) is None
    assert bench.recorded_traffic("step", "bf16", cells) is None


def test_committed_traffic_matches_the_current_kernel_sources():
    """The DRAM bytes in profiles/traffic.json were taken from the kernels as
    they are: after a kernel change the counters are taken again (or the
    entry goes), so that the bench line never reports stale traffic."""
    with open(os.path.join(bench.ROOT, "profiles", "traffic.json")) as fh:
        rec = json.load(fh)
    for key in bench.KERNEL_SOURCES:
        assert rec[key]["source_hash"] == bench.kernel_source_hash(key), key


def _sampler(lines):
    s = object.__new__(bench.ClockSampler)
    s.samples = list(lines)
    s.proc = None
    return s


def _line(sm, mx=2070, power=900.0, hw="Not Active", thermal="Not Active", sw_thermal="Not Active",
          cap="Not Active"):
    return f"0, {sm}, {mx}, {power}, 0x0, {hw}, {thermal}, {sw_thermal}, {cap}"


def test_clock_summary_inside_the_timed_region():
    s = _sampler([(0.5, _line(1000)), (1.0, _line(2070)), (1.2, _line(2050, cap="Active")), (1.4, _line(2060)),
                  (3.0, _line(800, hw="Active"))])
    c = s.summary(0.9, 1.5)
    assert c["samples"] == 3 and c["sm_mhz"] == 2060 and c["sm_max_mhz"] == 2070
    assert c["reasons"] == ["sw_power_cap"]  # kept and noted, not a rejection reason
    assert bench.ClockSampler.summary(_sampler([(2.9, _line(800, hw="Active"))]), 2.8, 3.1)["reasons"] == \
        ["hw_slowdown"]


def test_clock_summary_of_a_short_region_takes_the_nearest_samples():
    s = _sampler([(0.0, _line(2070)), (1.0, _line(2060)), (5.0, _line(1200))])
    c = s.summary(1.05, 1.10)
    assert c["samples"] == 2 and c["sm_mhz"] == pytest.approx(2065)


def test_clock_summary_without_samples_says_so():
    c = _sampler([(0.0, "garbled"), (0.1, "[N/A]")]).summary(0.0, 1.0)
    assert c["samples"] == 0 and c["reasons"] == ["no nvidia-smi samples"]
