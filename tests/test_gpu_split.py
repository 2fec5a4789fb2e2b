"""One shuffle split by domain range, its parts run one after another on one
GPU: every part's count (bshuffle_count_range) must equal the oracle's count
of its range, and the parts' outputs (bshuffle_permute_range), placed at the
exclusive sums of the counts, must together equal the oracle's shuffle, bit
for bit.  The multi-rank exchange of the counts is tested on the CPU with
gloo ranks (test_split.py); runs on more than one GPU are not made here."""
import numpy as np
import pytest
import torch

import oracle
import workloads
from tests.gpu_helpers import assert_no_device_error, to_device, to_host

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def bs():
    from paper_2106_06161_gb300 import build
    build.build()
    import paper_2106_06161_gb300
    paper_2106_06161_gb300.load()
    return paper_2106_06161_gb300


def _payload(n, width, seed):
    if width in (4, 8, 16):
        return workloads.sweep_payload(n, width, seed)
    dt = {1: np.uint8, 2: np.uint16}[width]
    return np.random.default_rng(seed).integers(0, np.iinfo(dt).max, size=n, dtype=dt, endpoint=True)


@pytest.mark.parametrize("width", [1, 2, 4, 8, 16])
def test_parts_one_after_another_equal_the_shuffle(bs, width):
    from paper_2106_06161_gb300 import split
    stream = torch.cuda.current_stream().cuda_stream
    for n, seed in ((5, 1), (2049, 2), (100_003, 3), (2**20, 4), (1_000_003, 5)):
        x = _payload(n, width, seed)
        xd = to_device(x)
        want = oracle.permute(x, seed)
        for parts in (1, 2, 3, 4):
            plan = split.ranges(n, parts)
            counts = [split.count_range(n, seed, f, e) for f, e in plan]
            counts = [int(c.item()) for c in counts]
            assert counts == [oracle.count_range(n, seed, f, e) for f, e in plan], (n, parts)
            offs, total = split.offsets(counts)
            assert total == n
            out = torch.empty_like(xd)
            for (f, e), off, c in zip(plan, offs, counts):
                if c:
                    # the part writes straight into its slots of the whole output
                    ptr = out.data_ptr() + off * width
                    bs.bshuffle_permute_range(xd.data_ptr(), ptr, n, width, seed, 24, f, e, c, stream)
            assert_no_device_error()
            assert np.array_equal(to_host(out, x), want), (n, parts)


def test_shards_without_communication(bs):
    # each part recomputes the counts of the ranges before it (no exchange)
    from paper_2106_06161_gb300 import split
    n, seed = 2**22 + 7, 11
    x = workloads.uniform_u64(n, seed)
    xd = to_device(x)
    want = oracle.permute_mt(x, seed)
    for world in (2, 4):
        pieces = []
        for rank in range(world):
            part, offset = split.permute_shard(xd, seed, rank, world, exchange=False)
            pieces.append((offset, part))
        assert_no_device_error()
        assert [p[0] for p in pieces] == sorted(p[0] for p in pieces)
        got = torch.cat([p[1] for p in pieces])
        assert got.numel() == n
        assert np.array_equal(to_host(got, x), want)


def test_ranges_off_the_tile_grid_and_clipped(bs):
    # ranges that start inside a 2,048-index tile, empty ranges, and an end
    # past the domain (clipped to 2^k)
    stream = torch.cuda.current_stream().cuda_stream
    n, seed = 70_001, 6                    # domain 2^17
    x = workloads.uniform_u32(n, seed)
    xd = to_device(x)
    idx = oracle.indices(n, seed)
    bounds = [0, 1, 2047, 2049, 50_000, 50_000, 131_071, 2**40]
    c_dev = torch.empty(1, dtype=torch.int64, device="cuda")
    start = 0
    for f, e in zip(bounds[:-1], bounds[1:]):
        bs.bshuffle_count_range(n, seed, 24, f, e, c_dev.data_ptr(), stream)
        c = int(c_dev.item())
        assert c == oracle.count_range(n, seed, f, e), (f, e)
        out = torch.full((max(c, 1),), -1, dtype=torch.int32, device="cuda")
        if c:
            bs.bshuffle_permute_range(xd.data_ptr(), out.data_ptr(), n, 4, seed, 24, f, e, c, stream)
            assert_no_device_error()
            assert np.array_equal(out.cpu().numpy().view(np.uint32), x[idx[start:start + c].astype(np.int64)])
        start += c
    assert start == n


def test_range_argument_errors(bs):
    from paper_2106_06161_gb300 import _lib as L
    lib = L.load()
    x = torch.empty(64, dtype=torch.int64, device="cuda")
    y = torch.empty(64, dtype=torch.int64, device="cuda")
    s = torch.cuda.current_stream().cuda_stream
    assert lib.bshuffle_count_range(64, 0, 24, 10, 5, y.data_ptr(), s) == L.BSHUFFLE_ERR_INVALID
    assert lib.bshuffle_count_range(64, 0, 24, 0, 5, None, s) == L.BSHUFFLE_ERR_NULL
    assert lib.bshuffle_permute_range(x.data_ptr(), y.data_ptr(), 64, 8, 0, 24, 9, 3, 64, s) == L.BSHUFFLE_ERR_INVALID
    assert lib.bshuffle_permute_range(x.data_ptr(), y.data_ptr(), 64, 32, 0, 24, 0, 64, 64, s) == L.BSHUFFLE_ERR_ELEM
    assert lib.bshuffle_permute_range(x.data_ptr(), x.data_ptr() + 8, 64, 8, 0, 24, 0, 64, 64, s) == \
        L.BSHUFFLE_ERR_ALIAS
    # out right before in, holding exactly its capacity: no overlap
    buf = torch.empty(128, dtype=torch.int64, device="cuda")
    assert lib.bshuffle_permute_range(buf.data_ptr() + 64 * 8, buf.data_ptr(), 64, 8, 0, 24, 0, 64, 64, s) == 0
    torch.cuda.synchronize()


def test_capacity_bounds_the_writes(bs):
    # a capacity below the range's count: the slots past it are not written
    # and the call records BSHUFFLE_ERR_DEVICE_BOUNDS
    from paper_2106_06161_gb300 import _lib as L
    n, seed = 10_000, 2
    x = torch.arange(n, dtype=torch.int64, device="cuda")
    out = torch.full((n,), -1, dtype=torch.int64, device="cuda")
    s = torch.cuda.current_stream().cuda_stream
    bs.bshuffle_permute_range(x.data_ptr(), out.data_ptr(), n, 8, seed, 24, 0, 2**14, 100, s)
    torch.cuda.synchronize()
    assert bs.get_error() == L.BSHUFFLE_ERR_DEVICE_BOUNDS
    want = oracle.indices(n, seed)[:100].astype(np.int64)
    assert np.array_equal(out[:100].cpu().numpy(), want)
    assert bool((out[100:] == -1).all())


@pytest.mark.parametrize("width", [1, 2, 4, 8, 16])
def test_power_of_two_ranges_scan_free(bs, width):
    # n = 2^k: every domain index is kept, so a range's count is its length,
    # its t-th slot holds x[f(first + t)], and the scan-free gather serves it;
    # ranges off the 2,048-index grid, empty, and clipped past the domain
    stream = torch.cuda.current_stream().cuda_stream
    n, seed = 2**17, 9
    x = _payload(n, width, seed)
    xd = to_device(x)
    idx = oracle.indices(n, seed).astype(np.int64)
    c_dev = torch.empty(1, dtype=torch.int64, device="cuda")
    bounds = [0, 1, 2047, 2049, 50_001, 50_001, 131_071, 2**40]
    for f, e in zip(bounds[:-1], bounds[1:]):
        bs.bshuffle_count_range(n, seed, 24, f, e, c_dev.data_ptr(), stream)
        c = int(c_dev.item())
        assert c == min(e, n) - f == oracle.count_range(n, seed, f, e), (f, e)
        if not c:
            continue
        out = to_device(np.zeros_like(x[:c]))
        bs.bshuffle_permute_range(xd.data_ptr(), out.data_ptr(), n, width, seed, 24, f, e, c, stream)
        assert_no_device_error()
        assert np.array_equal(to_host(out, x[:c]), x[idx[f:f + c]]), (f, e)


def test_power_of_two_capacity_bounds_the_writes(bs):
    from paper_2106_06161_gb300 import _lib as L
    n, seed = 2**14, 4
    x = torch.arange(n, dtype=torch.int64, device="cuda")
    out = torch.full((n,), -1, dtype=torch.int64, device="cuda")
    s = torch.cuda.current_stream().cuda_stream
    bs.bshuffle_permute_range(x.data_ptr(), out.data_ptr(), n, 8, seed, 24, 100, n, 1000, s)
    torch.cuda.synchronize()
    assert bs.get_error() == L.BSHUFFLE_ERR_DEVICE_BOUNDS
    want = oracle.indices(n, seed)[100:1100].astype(np.int64)
    assert np.array_equal(out[:1000].cpu().numpy(), want)
    assert bool((out[1000:] == -1).all())
    # the next call on the stream is exact again
    bs.bshuffle_permute_range(x.data_ptr(), out.data_ptr(), n, 8, seed, 24, 0, n, n, s)
    assert_no_device_error()
    assert np.array_equal(out.cpu().numpy(), oracle.indices(n, seed).astype(np.int64))


def test_power_of_two_shards_need_no_exchange(bs):
    from paper_2106_06161_gb300 import split
    n, seed = 2**22, 12
    x = workloads.uniform_u64(n, seed)
    xd = to_device(x)
    want = oracle.permute_mt(x, seed)
    for world in (2, 3, 4):
        pieces = [split.permute_shard(xd, seed, r, world) for r in range(world)]
        assert_no_device_error()
        assert [p[1] for p in pieces] == [f for f, _ in split.ranges(n, world)]
        got = torch.cat([p[0] for p in pieces])
        assert np.array_equal(to_host(got, x), want)
