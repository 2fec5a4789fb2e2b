"""Power-of-two lengths through the scan-free kernels.

When n = 2^k nothing is dropped and the exclusive scan of Algorithm 1 is the
identity, so by default (the automatic strategy) the library writes
out[i] = in[f(i)], out[f(i)] = in[i] or out[i] = f(i) directly.  The output
must equal the oracle's bit for bit, and the fused kernels' (requested
explicitly), for every mode, element width and row width."""
import numpy as np
import pytest
import torch

import oracle
from tests.gpu_helpers import assert_no_device_error, to_device, to_host

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def bs():
    from paper_2106_06161_gb300 import build
    build.build()
    import paper_2106_06161_gb300
    paper_2106_06161_gb300.load()
    paper_2106_06161_gb300.bshuffle_set_strategy(paper_2106_06161_gb300.BSHUFFLE_STRATEGY_AUTO)
    yield paper_2106_06161_gb300
    paper_2106_06161_gb300.bshuffle_set_strategy(paper_2106_06161_gb300.BSHUFFLE_STRATEGY_AUTO)


def _payload(n: int, width: int, seed: int) -> np.ndarray:
    rng = np.random.default_rng(seed * 7919 + width)
    if width in (1, 2, 4, 8):
        dt = {1: np.uint8, 2: np.uint16, 4: np.uint32, 8: np.uint64}[width]
        return rng.integers(0, np.iinfo(dt).max, size=n, dtype=dt, endpoint=True)
    return rng.integers(0, 256, size=(n, width), dtype=np.uint8)


@pytest.mark.parametrize("width", [1, 2, 4, 8, 16, 32, 48, 4096])
def test_permute_and_inverse_match_oracle(bs, width):
    for n in (16, 32, 2048, 65536, 2**20):
        if width >= 48 and n > 65536:
            continue
        for seed in (0, 5):
            x = _payload(n, width, seed)
            xd = to_device(x)
            y = bs.permute(xd, seed)
            assert_no_device_error()
            assert np.array_equal(to_host(y, x), oracle.permute(x, seed)), (n, seed)
            z = bs.inverse(xd, seed)
            assert_no_device_error()
            assert np.array_equal(to_host(z, x), oracle.inverse(x, seed)), (n, seed)
            assert torch.equal(bs.inverse(y, seed), xd)


@pytest.mark.parametrize("idx_dtype", [torch.int32, torch.int64])
def test_indices_match_oracle(bs, idx_dtype):
    for n in (16, 1024, 2**17, 2**22):
        idx = bs.indices(n, 9, dtype=idx_dtype)
        assert_no_device_error()
        assert np.array_equal(idx.cpu().numpy().astype(np.uint64), oracle.indices(n, 9)), n


@pytest.mark.parametrize("rounds", [0, 1, 2, 24, 64])
def test_rounds(bs, rounds):
    # odd (2^13) and even (2^14) domain exponents
    for n in (2**13, 2**14):
        x = _payload(n, 8, rounds)
        y = bs.permute(to_device(x), 4, rounds)
        assert_no_device_error()
        assert np.array_equal(to_host(y, x), oracle.permute(x, 4, rounds)), n


def test_equals_the_fused_kernels(bs):
    n, seed = 2**21, 3
    x = torch.from_numpy(_payload(n, 8, 1).view(np.int64)).cuda()
    rows = torch.randn(2**12, 256, device="cuda")
    outs = {}
    for name, strategy in (("auto", bs.BSHUFFLE_STRATEGY_AUTO), ("single", bs.BSHUFFLE_STRATEGY_SINGLE_PASS),
                           ("pipe", bs.BSHUFFLE_STRATEGY_PIPELINED)):
        bs.bshuffle_set_strategy(strategy)
        try:
            outs[name] = (bs.permute(x, seed), bs.inverse(x, seed), bs.indices(n, seed),
                          bs.permute(rows, seed), bs.inverse(rows, seed))
            assert_no_device_error()
        finally:
            bs.bshuffle_set_strategy(bs.BSHUFFLE_STRATEGY_AUTO)
    for name in ("single", "pipe"):
        for got, want in zip(outs["auto"], outs[name]):
            assert torch.equal(got, want), name
