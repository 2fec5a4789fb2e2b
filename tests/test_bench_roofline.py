"""The roofline arithmetic and timing helpers of bench.py on CPU: algorithmic bytes and
evaluations per launch, the dominant kernel of a step, the measured peak, and
the DRAM traffic taken from the committed ncu record only while the kernel's
source fingerprint matches."""
import json
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import bench  # noqa: E402
from paper_2106_06161_gb300 import build as bsbuild  # noqa: E402

N = 2**28


def test_staged_step_reports_its_longer_pass_on_algorithmic_bytes():
    peak, _ = bench.measured_peaks()
    roof, lines = bench.roofline_for([1.80, 1.92], bsbuild, bench.STRATEGIES["auto"], step_ms=3.72)
    assert [ln["kernel"] for ln in lines] == ["staged_bucket_kernel<uint64, even k>",
                                              "staged_scatter_kernel<uint64>"]
    # algorithmic bytes are the metric's: one 8-byte read and one write per element
    algo = 2 * N * 8
    for ln, ms in zip(lines, (1.80, 1.92)):
        assert ln["algorithmic_bytes_per_launch"] == algo
        assert ln["achieved_gbps"] == pytest.approx(algo / (ms * 1e-3) / 1e9)
    # the staged intermediate (value + slot, 20 B per element) is reported beside it
    assert lines[0]["staged_bytes_per_launch"] == N * 20
    assert lines[1]["staged_gbps"] == pytest.approx(N * 20 / 1.92e-3 / 1e9)
    # pass 1 is bound by the inverse cipher: 2^28 evaluations per launch
    # against the FMA-heavy pipe's rate
    assert lines[0]["bound"] == "alu"
    assert lines[0]["alu"]["achieved"] == pytest.approx(N / 1.80e-3)
    assert lines[0]["alu"]["peak"] == pytest.approx(
        152 * 4 * 16 * 2.07e9 / bench.FMAHEAVY_INST_PER_INVERSE_EVAL)
    assert roof["kernel"] == "staged_scatter_kernel<uint64>"
    assert roof["achieved"] == pytest.approx(algo / 1.92e-3 / 1e9)
    assert roof["frac"] == pytest.approx(roof["achieved"] / peak)
    assert roof["step_frac"] == pytest.approx(algo / 3.72e-3 / 1e9 / peak)
    assert roof["peak"] == peak
    assert set(roof) >= {"bound", "achieved", "peak", "unit", "frac", "traffic"}


def test_single_pass_step_uses_logical_bytes():
    roof, lines = bench.roofline_for([5.0], bsbuild, bench.STRATEGIES["single_pass"])
    assert len(lines) == 1 and lines[0]["kernel"].startswith("elem_tile_kernel")
    assert roof["achieved"] == pytest.approx(2 * N * 8 / 5.0e-3 / 1e9)
    roof, lines = bench.roofline_for([5.0], bsbuild, bench.STRATEGIES["pipelined"])
    assert lines[0]["kernel"].startswith("pipe_tile_kernel")


def test_summary_is_the_last_key_and_reads_the_extras():
    line = {"value": 7.2e10, "ms_per_step": 3.7, "roofline": {"frac": 0.33, "step_frac": 0.17, "kernel": "k"},
            "e2e": {"value": 1e10},
            "extra": {"2p28_u64_pipelined": {"ms": 5.2}, "worst_case_2p28_plus_12345_u64_pipelined": {"ms": 5.8},
                      "batched_4096_uneven_int32": {"speedup": 4.6},
                      "sweep": {"rows": {"8B": {"2^28": {"elements_per_s_mean": 7.2e10}}}}},
            "cpu_baseline": {"value": 1e8, "cores": 16, "single_thread": {"value": 4e6},
                             "fisher_yates": {"value": 5e7}}}
    s = bench.summary(line)
    assert s["2p28_u64_ms"] == {"pipelined": 5.2}
    assert s["worst_case_2p28_plus_12345_u64_ms"] == {"pipelined": 5.8}
    assert s["sweep_gelem_per_s"] == {"8B": {"2^28": 72.0}}
    assert s["batched_speedup"] == 4.6 and s["cpu_elements_per_s"]["cores"] == 16


def test_reference_and_gpu_arms_share_the_config():
    assert bench.workload_config(1) == bench.workload_config(1)
    assert bench.workload_config(1)["n"] == N and bench.workload_config(1)["elem_bytes"] == 8


def test_traffic_needs_a_matching_fingerprint():
    with open(bench.TRAFFIC_FILE) as fh:
        record = json.load(fh)["kernels"]
    name = "staged_scatter_kernel<uint64>"
    entry = record[name]
    assert entry["dram_bytes_per_launch"] == entry["dram_bytes_read"] + entry["dram_bytes_write"]
    assert bench.traffic_for(name, entry["kernel_fingerprint"]) == entry["dram_bytes_per_launch"]
    assert bench.traffic_for(name, "0" * 16) is None
    assert bench.traffic_for("no_such_kernel", entry["kernel_fingerprint"]) is None


def test_kernel_fingerprint_covers_headers(tmp_path, monkeypatch):
    # the record of one kernel goes stale when its source or any csrc header
    # changes, and only then
    import shutil
    csrc = tmp_path / "csrc"
    shutil.copytree(bsbuild.CSRC, csrc)
    monkeypatch.setattr(bsbuild, "CSRC", str(csrc))
    fp = bsbuild.kernel_fingerprint("kernels_staged.cu")
    assert len(fp) == 16 and fp != bsbuild.kernel_fingerprint("kernels_pipe.cu")
    (csrc / "kernels_mc.cu").write_text((csrc / "kernels_mc.cu").read_text() + "\n// another kernel\n")
    assert bsbuild.kernel_fingerprint("kernels_staged.cu") == fp
    (csrc / "bshuffle_internal.h").write_text((csrc / "bshuffle_internal.h").read_text() + "\n// a header\n")
    assert bsbuild.kernel_fingerprint("kernels_staged.cu") != fp


class _FakeEvent:
    """Stands in for torch.cuda.Event: a clock that the fake launches advance."""
    clock = [0.0]

    def __init__(self, enable_timing=True):
        self.t = None

    def record(self, stream=None):
        self.t = _FakeEvent.clock[0]

    def elapsed_time(self, other):
        return other.t - self.t


class _FakeTorch:
    class cuda:  # noqa: N801 - mirrors torch.cuda
        Event = _FakeEvent

        @staticmethod
        def synchronize():
            pass


def test_timed_region_is_time_per_call_between_one_event_pair():
    _FakeEvent.clock[0] = 0.0
    calls = []

    def launch():
        calls.append(1)
        _FakeEvent.clock[0] += 0.046     # ms of device time per call

    ms = bench.timed_region(launch, 50, None, _FakeTorch)
    assert len(calls) == 50
    assert ms == pytest.approx(0.046)


def test_timed_launches_reports_each_call_and_the_region():
    _FakeEvent.clock[0] = 0.0

    def launch():
        _FakeEvent.clock[0] += 3.7

    per, region = bench.timed_launches(launch, 4, None, _FakeTorch)
    assert per == pytest.approx([3.7] * 4)
    assert region == pytest.approx(4 * 3.7)
