"""Parity of the persistent batched launch with the oracle and with the plain
call, including the 4096-instance uneven batch (sizes log-uniform in
[100, 2,000,000], int32 payloads, instance seed = base seed + instance id)."""
import hashlib
import multiprocessing as mp
from concurrent.futures import ProcessPoolExecutor

import numpy as np
import pytest
import torch

import oracle
import workloads
from tests.gpu_helpers import assert_no_device_error, to_device, to_host

pytestmark = pytest.mark.gpu

bs = None


@pytest.fixture(scope="module", autouse=True)
def library():
    global bs
    from paper_2106_06161_gb300 import build
    build.build()
    import paper_2106_06161_gb300
    bs = paper_2106_06161_gb300
    bs.load()
    yield


def _oracle_digest(args):
    n, seed = args
    idx = oracle.indices(int(n), int(seed)).astype(np.uint32)
    return hashlib.sha256(idx.tobytes()).hexdigest()


@pytest.mark.parametrize("width", [1, 2, 4, 8, 16])
def test_batched_matches_oracle_edge_sizes(width):
    sizes = [0, 1, 2, 3, 16, 17, 2047, 2048, 2049, 4097, 100, 65537, 0, 300001, 5]
    rng = np.random.default_rng(width)
    dt = {1: np.uint8, 2: np.uint16, 4: np.uint32, 8: np.uint64}.get(width)
    xs = []
    for s in sizes:
        if dt is None:
            xs.append(rng.integers(0, 2**62, size=(s, 2), dtype=np.uint64))
        else:
            xs.append(rng.integers(0, np.iinfo(dt).max, size=s, dtype=dt, endpoint=True))
    seeds = [1000 + t for t in range(len(sizes))]
    outs = bs.batched([to_device(x) for x in xs], seeds)
    assert_no_device_error()
    for x, y, s in zip(xs, outs, seeds):
        assert np.array_equal(to_host(y, x), oracle.permute(x, s) if len(x) else x)


def test_batched_equals_plain_and_repeats():
    sizes = workloads.batched_sizes(count=64, hi=200_000, seed=5)
    data = torch.from_numpy(workloads.batched_payloads(sizes, seed=6)).cuda()
    seeds = [77 + t for t in range(len(sizes))]
    y1 = bs.batched_packed(data, sizes, seeds)
    y2 = bs.batched_packed(data, sizes, seeds)
    assert_no_device_error()
    assert torch.equal(y1, y2)
    off = 0
    for t, n in enumerate(sizes):
        plain = bs.permute(data[off:off + n], seeds[t])
        assert torch.equal(plain, y1[off:off + n])
        off += int(n)
    assert_no_device_error()


def test_uneven_batch_4096_instances_exact():
    sizes = workloads.batched_sizes()
    base_seed = 0
    seeds = [base_seed + t for t in range(len(sizes))]
    # oracle digests of every instance's index sequence, computed in parallel
    ctx = mp.get_context("spawn")
    with ProcessPoolExecutor(max_workers=min(16, mp.cpu_count()), mp_context=ctx) as ex:
        digests = list(ex.map(_oracle_digest, zip(sizes.tolist(), seeds), chunksize=16))
    # iota payload per instance: the output is each instance's index sequence
    iota = torch.cat([torch.arange(int(n), dtype=torch.int32) for n in sizes]).cuda()
    out = bs.batched_packed(iota, sizes, seeds)
    assert_no_device_error()
    host = out.cpu().numpy().view(np.uint32)
    off = 0
    for t, n in enumerate(sizes):
        got = hashlib.sha256(host[off:off + n].tobytes()).hexdigest()
        assert got == digests[t], f"instance {t} (n={n})"
        off += int(n)
    # random int32 payloads on a sample of instances, against oracle.permute
    payload = workloads.batched_payloads(sizes)
    dev = torch.from_numpy(payload).cuda()
    y = bs.batched_packed(dev, sizes, seeds).cpu().numpy()
    assert_no_device_error()
    offs = np.concatenate([[0], np.cumsum(sizes)])
    for t in np.random.default_rng(3).choice(len(sizes), 40, replace=False):
        a, b = offs[t], offs[t + 1]
        assert np.array_equal(y[a:b], oracle.permute(payload[a:b], seeds[t]))


def test_batched_graph_capture_replays():
    sizes = workloads.batched_sizes(count=200, hi=100_000, seed=9)
    data = torch.from_numpy(workloads.batched_payloads(sizes, seed=10)).cuda()
    seeds = list(range(500, 500 + len(sizes)))
    want = bs.batched_packed(data, sizes, seeds)
    out = torch.empty_like(data)
    descs = bs.packed_descs(data, out, sizes, seeds)
    torch.cuda.synchronize()
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        # first call on this stream creates its workspace, before capture
        bs.bshuffle_batched(descs.data_ptr(), len(sizes), 4, 24, s.cuda_stream)
        s.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=s):
            bs.bshuffle_batched(descs.data_ptr(), len(sizes), 4, 24, s.cuda_stream)
    torch.cuda.synchronize()
    for _ in range(3):
        out.zero_()
        g.replay()
        torch.cuda.synchronize()
        assert torch.equal(out, want)
