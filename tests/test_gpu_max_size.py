"""Maximum sizes: n = 2^32 - 1, the library's largest length (domain 2^32,
k = 32, 16-bit halves), and n = 2^31, the largest power-of-two length the
staged path takes.  At n = 2^32 - 1 exactly one domain index is dropped, d = f^-1(n),
so slot j holds X[f(j)] for j < d and X[f(j + 1)] for j >= d: sampled slots
are checked against the oracle's bijection and inverse, and sums and extrema
check that the output is a permutation of the input."""
import numpy as np
import pytest
import torch

import oracle
from tests.gpu_helpers import assert_no_device_error

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

N_MAX = 2**32 - 1


@pytest.fixture(scope="module")
def bs():
    from paper_2106_06161_gb300 import build
    build.build()
    import paper_2106_06161_gb300
    paper_2106_06161_gb300.load()
    yield paper_2106_06161_gb300
    paper_2106_06161_gb300.bshuffle_set_strategy(paper_2106_06161_gb300.BSHUFFLE_STRATEGY_AUTO)
    torch.cuda.empty_cache()


def _expected_sources(js: np.ndarray, seed: int) -> np.ndarray:
    keys = oracle.round_keys(seed, 24)
    d = int(oracle.varphilox_inverse(np.array([N_MAX], dtype=np.uint64), 32, keys)[0])
    i = js.astype(np.uint64) + (js.astype(np.uint64) >= np.uint64(d)).astype(np.uint64)
    return oracle.varphilox(i, 32, keys)


def _sample_slots(seed: int) -> np.ndarray:
    rng = np.random.default_rng(seed)
    return np.concatenate([np.arange(4096), rng.integers(0, N_MAX, 200_000), np.arange(N_MAX - 4096, N_MAX)])


def test_max_length_uint32_iota(bs):
    # 4-byte elements go through the staged path's ranked form (512 spans of
    # 2^23 domain indices, each ranked by a cluster of 8 CTAs; 32 GiB of
    # staging); x[i] = i, so the output is the index sequence itself
    # (16 GiB in, 16 GiB out)
    seed = 17
    x = torch.arange(N_MAX, dtype=torch.int64, device="cuda").to(torch.int32)
    y = bs.permute(x, seed)
    assert_no_device_error()
    js = _sample_slots(seed)
    got = y[torch.from_numpy(js).cuda()].cpu().numpy().view(np.uint32).astype(np.uint64)
    assert np.array_equal(got, _expected_sources(js, seed))
    # a permutation of 0 .. n - 1: same sum, same extrema
    yy = y.view(torch.int32)
    total = int(yy.to(torch.int64).remainder(2**32).sum())
    assert total == N_MAX * (N_MAX - 1) // 2
    del x, yy, y
    torch.cuda.empty_cache()


def test_max_length_bytes_and_indices(bs):
    # 1-byte elements (the plain kernel) and the 32-bit index output
    seed = 5
    # unsigned 32-bit indices through the C ABI (the tensor wrapper only
    # hands out signed int32 up to 2^31)
    idx = torch.empty(N_MAX, dtype=torch.int32, device="cuda")
    bs.bshuffle_indices(idx.data_ptr(), 4, N_MAX, seed, 24, torch.cuda.current_stream().cuda_stream)
    assert_no_device_error()
    js = _sample_slots(seed + 1)
    src = _expected_sources(js, seed)
    got = idx[torch.from_numpy(js).cuda()].cpu().numpy().view(np.uint32).astype(np.uint64)
    assert np.array_equal(got, src)
    del idx
    torch.cuda.empty_cache()
    g = torch.Generator(device="cuda").manual_seed(3)
    x = torch.randint(0, 256, (N_MAX,), dtype=torch.uint8, device="cuda", generator=g)
    y = bs.permute(x, seed)
    assert_no_device_error()
    assert torch.equal(y[torch.from_numpy(js).cuda()].cpu(), x[torch.from_numpy(src.astype(np.int64)).cuda()].cpu())
    assert torch.equal(torch.bincount(y, minlength=256), torch.bincount(x, minlength=256))
    del x, y
    torch.cuda.empty_cache()


def test_largest_staged_length(bs):
    # n = 2^31 uint32 through the staged path in both directions
    n, seed = 2**31, 9
    x = torch.arange(n, dtype=torch.int64, device="cuda").to(torch.int32)
    bs.bshuffle_set_strategy(bs.BSHUFFLE_STRATEGY_STAGED)
    try:
        y = bs.permute(x, seed)
        assert_no_device_error()
        rng = np.random.default_rng(8)
        js = np.concatenate([np.arange(2048), rng.integers(0, n, 200_000), np.arange(n - 2048, n)])
        src = oracle.varphilox(js.astype(np.uint64), 31, oracle.round_keys(seed, 24))
        got = y[torch.from_numpy(js).cuda()].cpu().numpy().view(np.uint32).astype(np.uint64)
        assert np.array_equal(got, src)
        z = bs.inverse(y, seed)
        assert_no_device_error()
        assert torch.equal(z, x)
    finally:
        bs.bshuffle_set_strategy(bs.BSHUFFLE_STRATEGY_AUTO)
    del x, y, z
    torch.cuda.empty_cache()


def test_max_length_ranges(bs):
    # the range entry points at the largest length: ranges at the start, the
    # middle and the top of the 2^32 domain (where a tile's 32-bit base
    # passes 2^32), 4-byte elements through the pipelined range kernel and
    # 1-byte elements through the plain one
    seed = 23
    keys = oracle.round_keys(seed, 24)
    s = torch.cuda.current_stream().cuda_stream
    c_dev = torch.empty(1, dtype=torch.int64, device="cuda")
    ranges = ((0, 2**20 + 3), (2**31 - 1000, 2**31 + 1000), (2**32 - 2**20 - 5, 2**32))
    expected = []
    for first, end in ranges:
        f = oracle.varphilox(np.arange(first, end, dtype=np.uint64), 32, keys)
        kept = f[f < N_MAX]
        assert kept.size == oracle.count_range(N_MAX, seed, first, end)
        bs.bshuffle_count_range(N_MAX, seed, 24, first, end, c_dev.data_ptr(), s)
        assert int(c_dev.item()) == kept.size, (first, end)
        expected.append(kept)
    x = torch.arange(N_MAX, dtype=torch.int64, device="cuda").to(torch.int32)  # x[b] = b
    for (first, end), kept in zip(ranges, expected):
        out = torch.full((kept.size,), -1, dtype=torch.int32, device="cuda")
        bs.bshuffle_permute_range(x.data_ptr(), out.data_ptr(), N_MAX, 4, seed, 24, first, end, kept.size, s)
        assert_no_device_error()
        assert np.array_equal(out.cpu().numpy().view(np.uint32).astype(np.uint64), kept), (first, end)
    del x
    torch.cuda.empty_cache()
    x8 = torch.arange(256, dtype=torch.uint8, device="cuda").repeat(N_MAX // 256 + 1)[:N_MAX].contiguous()
    for (first, end), kept in zip(ranges, expected):
        out = torch.empty(kept.size, dtype=torch.uint8, device="cuda")
        bs.bshuffle_permute_range(x8.data_ptr(), out.data_ptr(), N_MAX, 1, seed, 24, first, end, kept.size, s)
        assert_no_device_error()
        assert np.array_equal(out.cpu().numpy(), (kept & np.uint64(255)).astype(np.uint8)), (first, end)
    del x8
    torch.cuda.empty_cache()
