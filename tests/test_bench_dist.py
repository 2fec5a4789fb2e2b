"""The multi-rank path of bench.py on CPU (gloo, world size 2): rank setup,
the barrier, the max over ranks of the timed region, the whole-job value,
and the reference arm printing on rank 0 only."""
import io
import multiprocessing as mp
import os
import socket
import sys
from contextlib import redirect_stdout

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank),
                      MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import bench
    import torch.distributed as dist
    r, w, _ = bench.dist_setup(world)
    bench.barrier(w)
    slowest = bench.max_over_ranks(10.0 + 5.0 * r, w)
    value = bench.job_value(1000, w, 4, slowest)
    dist.destroy_process_group()
    q.put((r, w, slowest, value))


def test_two_ranks_take_the_slowest_region():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    got = sorted(q.get(timeout=10) for _ in range(2))
    for r, (rank, world, slowest, value) in enumerate(got):
        assert (rank, world) == (r, 2)
        assert slowest == 15.0
        # 2 ranks x 1000 elements x 4 steps over 15 ms
        assert value == pytest.approx(2 * 1000 * 4 / 15e-3)


def test_reference_arm_prints_on_rank_zero_only(monkeypatch):
    sys.path.insert(0, ROOT)
    import bench
    args = bench.argparse.Namespace(gpus=2, steps=1, warmup=0)
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    buf = io.StringIO()
    with redirect_stdout(buf):
        bench.run_reference(args)
    assert buf.getvalue() == ""


def test_reference_arm_line_on_rank_zero(monkeypatch):
    # the reference arm's JSON line on a tiny stand-in workload: the oracle
    # on host threads, the GPU arm's config, no host-device copies
    sys.path.insert(0, ROOT)
    import json

    import bench
    monkeypatch.setattr(bench, "N_MAIN", 2**16)
    monkeypatch.setattr(bench, "REF_DOMAIN_SAMPLE", 2**12)
    monkeypatch.setenv("RANK", "0")
    args = bench.argparse.Namespace(gpus=1, steps=3, warmup=1)
    buf = io.StringIO()
    with redirect_stdout(buf):
        bench.run_reference(args)
    line = json.loads(buf.getvalue().strip())
    assert line["impl"] == "reference" and line["steps"] == 3 and line["warmup"] == 1
    assert line["config"] == bench.workload_config(1)
    assert line["metric"] == bench.METRIC and line["unit"] == "elements/s" and line["value"] > 0
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] >= 1
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["d2h_bytes_per_step"] == 0
