"""The roofline arithmetic of bench.py on CPU: algorithmic bytes and
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


def test_staged_step_reports_its_longer_pass():
    peak, _ = bench.measured_peaks()
    roof, lines = bench.roofline_for([1.80, 1.92], bsbuild, bench.STRATEGIES["auto"])
    assert [ln["kernel"] for ln in lines] == ["staged_bucket_kernel<uint64, even k>",
                                              "staged_scatter_kernel<uint64>"]
    # pass 1 is bound by the inverse cipher: 2^28 evaluations per launch
    assert lines[0]["bound"] == "alu"
    assert lines[0]["achieved"] == pytest.approx(N / 1.80e-3)
    assert lines[0]["peak"] == pytest.approx(152 * 128 * 2.07e9 / (24 * 7))
    # pass 2 moves 8 B value + 4 B slot in and 8 B out per element
    assert lines[1]["bound"] == "hbm"
    assert lines[1]["achieved"] == pytest.approx(N * 20 / 1.92e-3 / 1e9)
    assert roof["kernel"] == "staged_scatter_kernel<uint64>"
    assert roof["frac"] == pytest.approx(roof["achieved"] / peak)
    assert roof["peak"] == peak
    assert set(roof) >= {"bound", "achieved", "peak", "unit", "frac", "traffic"}


def test_single_pass_step_uses_logical_bytes():
    roof, lines = bench.roofline_for([5.0], bsbuild, bench.STRATEGIES["single_pass"])
    assert len(lines) == 1 and lines[0]["kernel"].startswith("elem_tile_kernel")
    assert roof["achieved"] == pytest.approx(2 * N * 8 / 5.0e-3 / 1e9)
    roof, lines = bench.roofline_for([5.0], bsbuild, bench.STRATEGIES["pipelined"])
    assert lines[0]["kernel"].startswith("pipe_tile_kernel")


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
