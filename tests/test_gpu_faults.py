"""Failure detection without a GPU fault: the look-back wait is bounded.

A test hook makes one tile withhold its tile status, so the waits of the
tiles after it run out (after a short, explicit limit).  The kernels must
report BSHUFFLE_ERR_LOOKBACK_TIMEOUT through bshuffle_get_error, finish, and
leave the stream and its workspace usable: the next call is exact again."""
import numpy as np
import pytest
import torch

import oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def bs():
    from paper_2106_06161_gb300 import build
    build.build()
    import paper_2106_06161_gb300
    paper_2106_06161_gb300.load()
    return paper_2106_06161_gb300


def _with_withheld_tile(bs, tile, fn):
    bs.bshuffle_set_lookback_timeout_ns(50_000_000)   # 50 ms per wait
    bs.bshuffle_debug_skip_publish(tile)
    try:
        fn()
        torch.cuda.synchronize()
        return bs.get_error()
    finally:
        bs.bshuffle_debug_skip_publish(-1)
        bs.bshuffle_set_lookback_timeout_ns(2_000_000_000)


def test_permute_wait_runs_out_and_recovers(bs):
    from paper_2106_06161_gb300 import _lib as L
    n = 10_000                      # domain 2^14: 8 tiles of 2,048 indices
    x = torch.arange(n, dtype=torch.int64, device="cuda")
    code = _with_withheld_tile(bs, 1, lambda: bs.permute(x, 3))
    assert code == L.BSHUFFLE_ERR_LOOKBACK_TIMEOUT
    assert bs.get_error() == 0                       # the error word was cleared
    y = bs.permute(x, 3)
    assert bs.get_error() == 0
    assert np.array_equal(y.cpu().numpy(), oracle.permute(np.arange(n, dtype=np.int64), 3))


def test_batched_wait_runs_out_and_recovers(bs):
    from paper_2106_06161_gb300 import _lib as L
    sizes = [9_000, 5_000]          # 4 + 2 tiles; global tile 1 belongs to instance 0
    data = torch.arange(sum(sizes), dtype=torch.int32, device="cuda")
    code = _with_withheld_tile(bs, 1, lambda: bs.batched_packed(data, sizes, [1, 2]))
    assert code == L.BSHUFFLE_ERR_LOOKBACK_TIMEOUT
    out = bs.batched_packed(data, sizes, [1, 2])
    assert bs.get_error() == 0
    host = data.cpu().numpy()
    res = out.cpu().numpy()
    assert np.array_equal(res[:9000], oracle.permute(host[:9000], 1))
    assert np.array_equal(res[9000:], oracle.permute(host[9000:], 2))
