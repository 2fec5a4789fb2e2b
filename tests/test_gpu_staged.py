"""The staged strategy of bshuffle_permute must produce exactly the single
pass's output.  For n = 2^k the inverse cipher turns the gather into a
scatter with a sequential source side, then an L2-resident window scatter;
for other n (the ranked form) pass 1 buckets each element by the span of
domain indices its preimage falls in, and pass 2 ranks the kept indices of a
span with a bitmap (spans larger than one CTA's bitmap are split over a
cluster of CTAs).  Checked against the oracle across widths and sizes,
against the single pass and the oracle at larger sizes, and through the
automatic choice at full size (test_gpu_full_size.py)."""
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
    yield paper_2106_06161_gb300
    paper_2106_06161_gb300.bshuffle_set_strategy(paper_2106_06161_gb300.BSHUFFLE_STRATEGY_AUTO)


def _run(bs, x: np.ndarray, seed: int, strategy: int, rounds: int = 24) -> np.ndarray:
    bs.bshuffle_set_strategy(strategy)
    try:
        y = bs.permute(to_device(x), seed, rounds)
        assert_no_device_error()
    finally:
        bs.bshuffle_set_strategy(bs.BSHUFFLE_STRATEGY_AUTO)
    return to_host(y, x)


@pytest.mark.parametrize("width", [4, 8, 16])
def test_staged_matches_oracle(bs, width):
    for n in (4096, 8192, 65536, 2**20, 2**22, 4097, 6000, 1_000_003):
        for seed in (0, 5):
            x = workloads.sweep_payload(n, width, seed)
            got = _run(bs, x, seed, bs.BSHUFFLE_STRATEGY_STAGED)
            assert np.array_equal(got, oracle.permute(x, seed)), (n, seed)


def _passes(bs, xd, seed, strategy, rounds=24):
    """Output and the number of passes the call ran (2 for the staged path)."""
    stream = torch.cuda.current_stream().cuda_stream
    bs.bshuffle_set_strategy(strategy)
    bs.bshuffle_set_pass_timing(True)
    try:
        y = bs.permute(xd, seed, rounds)
        passes = len(bs.bshuffle_last_pass_ms(stream))
        assert_no_device_error()
    finally:
        bs.bshuffle_set_pass_timing(False)
        bs.bshuffle_set_strategy(bs.BSHUFFLE_STRATEGY_AUTO)
    return y, passes


@pytest.mark.parametrize("width", [4, 8, 16])
def test_ranked_form_runs_for_other_lengths(bs, width):
    # lengths just above and below powers of two, ragged last chunks, one
    # element short of the domain, and rounds other than the default
    for n, seed, rounds in ((4097, 1, 24), (6000, 2, 24), (65535, 3, 24), (100_003, 4, 24), (2**20 + 1, 5, 24),
                            (3 * 2**20 - 7, 6, 24), (2**22 - 1, 7, 24), (1_000_003, 8, 0), (1_000_003, 9, 1),
                            (1_000_003, 10, 23)):
        x = workloads.sweep_payload(n, width, seed)
        y, passes = _passes(bs, to_device(x), seed, bs.BSHUFFLE_STRATEGY_STAGED, rounds)
        assert passes == 2, n
        assert np.array_equal(to_host(y, x), oracle.permute(x, seed, rounds)), (n, seed, rounds)


@pytest.mark.parametrize("n,width", [(2**29 + 3, 4), (2**30 + 5, 4), (2**28 + 12345, 16)])
def test_ranked_form_spans_over_several_ctas(bs, n, width):
    # on 2^30- and 2^31-index domains the 512 spans of 2^21 or 2^22 indices
    # are ranked by clusters of 2 or 4 CTAs; 16-byte elements at 2^28 + 12345
    # take 4,096-element pass-1 chunks
    seed = 11
    x = workloads.sweep_payload(n, width, seed) if width == 16 else None
    xd = to_device(x) if x is not None else torch.arange(n, dtype=torch.int32, device="cuda")
    y, passes = _passes(bs, xd, seed, bs.BSHUFFLE_STRATEGY_STAGED)
    assert passes == 2
    idx = torch.from_numpy(oracle.indices_mt(n, seed).view(np.int64)).cuda()
    assert torch.equal(y, xd[idx]), n
    del y, idx, xd


@pytest.mark.parametrize("rounds", [0, 1, 24])
def test_staged_rounds(bs, rounds):
    x = workloads.uniform_u64(2**18, rounds)
    assert np.array_equal(_run(bs, x, 3, bs.BSHUFFLE_STRATEGY_STAGED, rounds), oracle.permute(x, 3, rounds))


def test_staged_equals_single_pass_and_oracle_large(bs):
    for n, width in ((2**25, 8), (2**26, 4), (2**24, 16), (2**25 + 1, 8), (2**26 + 999, 4), (2**24 + 3, 16)):
        x = workloads.sweep_payload(n, width, 9)
        xd = to_device(x)
        outs = []
        for strategy in (bs.BSHUFFLE_STRATEGY_STAGED, bs.BSHUFFLE_STRATEGY_SINGLE_PASS):
            bs.bshuffle_set_strategy(strategy)
            outs.append(bs.permute(xd, 9))
            assert_no_device_error()
        bs.bshuffle_set_strategy(bs.BSHUFFLE_STRATEGY_AUTO)
        assert torch.equal(outs[0], outs[1]), (n, width)
        # every slot against the oracle (64 windows at 2^25 uint64 and 2^26
        # uint32; 256 spans of domain indices at the other lengths)
        idx = torch.from_numpy(oracle.indices_mt(n, 9).view(np.int64)).cuda()
        assert torch.equal(outs[0], xd[idx]), (n, width)


def test_staged_repeated_and_alternating(bs):
    x = workloads.uniform_u32(2**21, 4)
    want = oracle.permute(x, 12)
    for _ in range(3):
        assert np.array_equal(_run(bs, x, 12, bs.BSHUFFLE_STRATEGY_STAGED), want)
        assert np.array_equal(_run(bs, x, 12, bs.BSHUFFLE_STRATEGY_SINGLE_PASS), want)


def test_pass_timing_reports_each_kernel(bs):
    x = torch.arange(2**22, dtype=torch.int64, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    bs.bshuffle_set_pass_timing(True)
    try:
        for strategy, passes in ((bs.BSHUFFLE_STRATEGY_STAGED, 2), (bs.BSHUFFLE_STRATEGY_SINGLE_PASS, 1)):
            bs.bshuffle_set_strategy(strategy)
            bs.permute(x, 1)
            ms = bs.bshuffle_last_pass_ms(stream)
            assert len(ms) == passes and all(t > 0 for t in ms)
    finally:
        bs.bshuffle_set_pass_timing(False)
        bs.bshuffle_set_strategy(bs.BSHUFFLE_STRATEGY_AUTO)
    assert bs.bshuffle_get_strategy() == bs.BSHUFFLE_STRATEGY_AUTO


def _run_inverse(bs, x: np.ndarray, seed: int, strategy: int, rounds: int = 24) -> np.ndarray:
    bs.bshuffle_set_strategy(strategy)
    try:
        y = bs.inverse(to_device(x), seed, rounds)
        assert_no_device_error()
    finally:
        bs.bshuffle_set_strategy(bs.BSHUFFLE_STRATEGY_AUTO)
    return to_host(y, x)


@pytest.mark.parametrize("width", [4, 8, 16])
def test_staged_inverse_matches_oracle(bs, width):
    # out[f(j)] = in[j]: the same two passes with the forward cipher
    for n in (4096, 65536, 2**21, 5000):
        for seed in (1, 6):
            x = workloads.sweep_payload(n, width, seed)
            got = _run_inverse(bs, x, seed, bs.BSHUFFLE_STRATEGY_STAGED)
            assert np.array_equal(got, oracle.inverse(x, seed)), (n, seed)


@pytest.mark.parametrize("rounds", [0, 1, 24])
def test_staged_inverse_rounds(bs, rounds):
    x = workloads.uniform_u32(2**17, rounds)
    assert np.array_equal(_run_inverse(bs, x, 2, bs.BSHUFFLE_STRATEGY_STAGED, rounds), oracle.inverse(x, 2, rounds))


@pytest.mark.parametrize("n,width,rounds", [(2**29, 8, 24), (2**30, 4, 24), (2**29, 4, 20), (2**28, 16, 24)])
def test_staged_inputs_over_2gib(bs, n, width, rounds):
    # Inputs over 2 GiB of 4- and 8-byte elements bucket 4,096-element chunks
    # into up to 512 windows; 16-byte elements keep 2,048-element chunks with
    # windows over 8 MiB.  x[i] = i, so slot j must hold f(j) (n = 2^k).
    k, seed = n.bit_length() - 1, 21
    dtype = {4: torch.int32, 8: torch.int64, 16: torch.int64}[width]
    xd = torch.arange(n, dtype=dtype, device="cuda")
    if width == 16:
        xd = torch.stack([xd, ~xd], dim=1).contiguous()
    outs = []
    for strategy in (bs.BSHUFFLE_STRATEGY_STAGED, bs.BSHUFFLE_STRATEGY_PIPELINED):
        bs.bshuffle_set_strategy(strategy)
        try:
            outs.append(bs.permute(xd, seed, rounds))
            assert_no_device_error()
        finally:
            bs.bshuffle_set_strategy(bs.BSHUFFLE_STRATEGY_AUTO)
    assert torch.equal(outs[0], outs[1])
    js = np.concatenate([np.arange(4096), np.random.default_rng(k).integers(0, n, 100_000),
                         np.arange(n - 4096, n)]).astype(np.uint64)
    want = oracle.varphilox(js, k, oracle.round_keys(seed, rounds)).astype(np.int64)
    got = outs[0][torch.from_numpy(js.astype(np.int64)).cuda()].cpu().numpy()
    if width == 16:
        assert np.array_equal(got[:, 0], want) and np.array_equal(got[:, 1], ~want)
    else:
        assert np.array_equal(got.astype(np.int64), want)
    del outs
    if width != 16:
        # the inverse shuffle over the same chunking undoes the shuffle
        bs.bshuffle_set_strategy(bs.BSHUFFLE_STRATEGY_STAGED)
        try:
            y = bs.permute(xd, seed, rounds)
            z = bs.inverse(y, seed, rounds)
            assert_no_device_error()
        finally:
            bs.bshuffle_set_strategy(bs.BSHUFFLE_STRATEGY_AUTO)
        assert torch.equal(z, xd)
