"""The pipelined single pass (BSHUFFLE_STRATEGY_PIPELINED) against the
oracle: the same output as Algorithm 1, bit for bit, for gathers and
scatters of 4-, 8- and 16-byte elements and for the index output, small
sizes with ragged last tiles up to the full worst-case length, plus its
bounded waits and the widths it hands to the plain kernel."""
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
    paper_2106_06161_gb300.bshuffle_set_strategy(paper_2106_06161_gb300.BSHUFFLE_STRATEGY_PIPELINED)
    yield paper_2106_06161_gb300
    paper_2106_06161_gb300.bshuffle_set_strategy(paper_2106_06161_gb300.BSHUFFLE_STRATEGY_AUTO)


def _payload(n, width, seed):
    rng = np.random.default_rng(seed * 31 + width)
    if width in (1, 2, 4, 8):
        dt = {1: np.uint8, 2: np.uint16, 4: np.uint32, 8: np.uint64}[width]
        return rng.integers(0, np.iinfo(dt).max, size=n, dtype=dt, endpoint=True)
    return rng.integers(0, 256, size=(n, width), dtype=np.uint8)


def _gpu(bs, x, seed, rounds=24):
    y = bs.permute(to_device(x), seed, rounds)
    assert_no_device_error()
    return to_host(y, x)


@pytest.mark.parametrize("width", [4, 8, 16])
def test_matches_oracle(bs, width):
    for n in (1, 2, 5, 17, 2047, 2048, 2049, 4097, 65537, 123457, 1_000_003):
        for seed in (0, 9):
            x = _payload(n, width, seed)
            assert np.array_equal(_gpu(bs, x, seed), oracle.permute(x, seed)), (n, seed)


@pytest.mark.parametrize("rounds", [0, 1, 24, 64])
def test_rounds(bs, rounds):
    for n in (33, 300_001):
        x = _payload(n, 8, rounds)
        assert np.array_equal(_gpu(bs, x, 5, rounds), oracle.permute(x, 5, rounds))


@pytest.mark.parametrize("idx_dtype", [torch.int32, torch.int64])
def test_indices_match_oracle(bs, idx_dtype):
    for n in (1, 3, 2047, 2049, 70_001, 1_000_003):
        for seed in (0, 4):
            got = bs.indices(n, seed, dtype=idx_dtype)
            assert_no_device_error()
            want = oracle.indices(n, seed)
            assert np.array_equal(got.cpu().numpy().astype(np.uint64), want), (n, seed)


@pytest.mark.parametrize("width", [1, 4, 8, 16])
def test_inverse_matches_oracle(bs, width):
    for n in (1, 5, 2049, 65537, 300_007):
        x = _payload(n, width, 3)
        y = bs.inverse(to_device(x), 8)
        assert_no_device_error()
        assert np.array_equal(to_host(y, x), oracle.inverse(x, 8)), n
        # inverse undoes permute
        z = bs.inverse(bs.permute(to_device(x), 8), 8)
        assert np.array_equal(to_host(z, x), x), n


def test_other_widths_use_the_plain_kernel(bs):
    for width in (1, 2, 32):
        x = _payload(10_007, width, 1)
        assert np.array_equal(_gpu(bs, x, 2), oracle.permute(x, 2))


def test_many_tiles_per_cta(bs):
    # 2^24 + 1: 8,192 tiles, several per persistent CTA, both buffers cycling
    for width in (4, 16):
        x = workloads.sweep_payload(2**24 + 1, width, 3)
        assert np.array_equal(_gpu(bs, x, 3), oracle.permute(x, 3))


def test_full_size_worst_case_sampled(bs):
    n, seed = 2**28 + 12345, 0
    want = oracle.indices(n, seed)
    idx = bs.indices(n, seed, dtype=torch.int64)
    assert_no_device_error()
    assert np.array_equal(idx.cpu().numpy().view(np.uint64), want)
    del idx
    x = workloads.uniform_u64(n, seed)
    y = bs.permute(to_device(x), seed)
    assert_no_device_error()
    rng = np.random.default_rng(4)
    js = np.concatenate([np.arange(4096), rng.integers(0, n, 400_000), np.arange(n - 4096, n)])
    got = y[torch.from_numpy(js).cuda()].cpu().numpy().view(np.uint64)
    assert np.array_equal(got, x[want[js].astype(np.int64)])
    # and slot for slot equal to the plain single pass
    bs.bshuffle_set_strategy(bs.BSHUFFLE_STRATEGY_SINGLE_PASS)
    try:
        y1 = bs.permute(to_device(x), seed)
        assert_no_device_error()
    finally:
        bs.bshuffle_set_strategy(bs.BSHUFFLE_STRATEGY_PIPELINED)
    assert torch.equal(y, y1)


def test_repeated_calls_and_streams(bs):
    x = _payload(500_009, 8, 2)
    want = oracle.permute(x, 11)
    for _ in range(4):
        assert np.array_equal(_gpu(bs, x, 11), want)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        y = bs.permute(to_device(x), 11)
        s.synchronize()
        assert bs.get_error() == 0
    assert np.array_equal(to_host(y, x), want)


def test_withheld_tile_times_out_and_recovers(bs):
    from paper_2106_06161_gb300 import _lib as L
    n = 40_000                      # domain 2^16: 32 tiles of 2,048 indices
    x = torch.arange(n, dtype=torch.int64, device="cuda")
    bs.bshuffle_set_lookback_timeout_ns(50_000_000)
    bs.bshuffle_debug_skip_publish(3)
    try:
        bs.permute(x, 3)
        torch.cuda.synchronize()
        code = bs.get_error()
    finally:
        bs.bshuffle_debug_skip_publish(-1)
        bs.bshuffle_set_lookback_timeout_ns(2_000_000_000)
    assert code == L.BSHUFFLE_ERR_LOOKBACK_TIMEOUT
    y = bs.permute(x, 3)
    assert bs.get_error() == 0
    assert np.array_equal(y.cpu().numpy(), oracle.permute(np.arange(n, dtype=np.int64), 3))


def test_graph_capture_replays(bs):
    # the pipelined kernel inside a captured CUDA graph: the workspace header
    # is reset by the last CTA of every launch, so replays stay exact
    n = 1_000_003
    x = torch.from_numpy(_payload(n, 8, 12).view(np.int64)).cuda()
    want = bs.permute(x, 21)
    want_idx = bs.indices(n, 21, dtype=torch.int32)
    y = torch.empty_like(x)
    idx = torch.empty(n, dtype=torch.int32, device="cuda")
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        # the first call on this stream creates its workspace, before capture
        bs.bshuffle_permute(x.data_ptr(), y.data_ptr(), n, 8, 21, 24, s.cuda_stream)
        s.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=s):
            bs.bshuffle_permute(x.data_ptr(), y.data_ptr(), n, 8, 21, 24, s.cuda_stream)
            bs.bshuffle_indices(idx.data_ptr(), 4, n, 21, 24, s.cuda_stream)
    torch.cuda.synchronize()
    for _ in range(3):
        y.zero_()
        idx.zero_()
        g.replay()
        torch.cuda.synchronize()
        assert torch.equal(y, want)
        assert torch.equal(idx, want_idx)
    assert bs.get_error() == 0


def test_concurrent_streams_share_the_gpu(bs):
    # Persistent kernels on three streams at once (pipelined single pass,
    # batched, staged): while they share the SMs not every CTA of a launch is
    # resident; tickets go only to running CTAs, so each still finishes, and
    # each stream's workspace keeps the results exact.
    n1 = 3_000_017
    x1 = torch.from_numpy(_payload(n1, 8, 31).view(np.int64)).cuda()
    sizes = workloads.batched_sizes(count=300, hi=200_000, seed=4)
    data = torch.from_numpy(workloads.batched_payloads(sizes, seed=5)).cuda()
    x3 = torch.from_numpy(workloads.uniform_u64(2**22, 6).view(np.int64)).cuda()
    want1 = oracle.permute(x1.cpu().numpy().view(np.uint64), 9)
    want3 = oracle.permute(x3.cpu().numpy().view(np.uint64), 10)
    seeds = list(range(40, 40 + len(sizes)))
    streams = [torch.cuda.Stream() for _ in range(3)]
    torch.cuda.synchronize()
    for _ in range(3):
        with torch.cuda.stream(streams[0]):
            y1 = bs.permute(x1, 9)
        with torch.cuda.stream(streams[1]):
            y2 = bs.batched_packed(data, sizes, seeds)
        with torch.cuda.stream(streams[2]):
            bs.bshuffle_set_strategy(bs.BSHUFFLE_STRATEGY_STAGED)
            try:
                y3 = bs.permute(x3, 10)
            finally:
                bs.bshuffle_set_strategy(bs.BSHUFFLE_STRATEGY_PIPELINED)
        torch.cuda.synchronize()
        for s in streams:
            with torch.cuda.stream(s):
                assert bs.get_error() == 0
        assert np.array_equal(y1.cpu().numpy().view(np.uint64), want1)
        assert np.array_equal(y3.cpu().numpy().view(np.uint64), want3)
        host = data.cpu().numpy()
        res = y2.cpu().numpy()
        off = 0
        for t in (0, 1, len(sizes) // 2, len(sizes) - 1):
            off = int(np.sum(sizes[:t]))
            m = int(sizes[t])
            assert np.array_equal(res[off:off + m], oracle.permute(host[off:off + m], seeds[t])), t
