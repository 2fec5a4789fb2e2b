"""Full-size parity of the default strategy with the oracle, slot by slot.

The sweep's two largest lengths through the C ABI, exactly as bench.py calls
them (library default strategy, 24 rounds):

* n = 2^28: nothing is dropped, so the default runs the staged two-pass path
  for 4-, 8- and 16-byte elements (256 output windows for uint64);
* n = 2^28 + 12345: domain 2^29 with about half of the images dropped (the
  paper's worst-case padding), run by the staged path's ranked form for 4-
  and 8-byte elements and by the pipelined single pass for 16-byte ones.

For every seed 0..4 of the sweep, every one of the n output slots of the
uint64 shuffle and of the 64-bit index output is compared with one full pass
of the oracle (Algorithm 1 run by host threads over domain ranges: count,
exclusive scan, write; pinned to brute force on the CPU).  Seed 0 also
checks every slot of the 4- and 16-byte shuffles.  The expected payload
x[idx] is formed on the device from the oracle's indices, so the comparison
covers every element without a host-side gather of gigabytes."""
import numpy as np
import pytest
import torch

import oracle
import workloads
from tests.gpu_helpers import assert_no_device_error, to_device

pytestmark = pytest.mark.gpu

FULL_SIZES = (2**28, 2**28 + 12345)


@pytest.fixture(scope="module")
def bs():
    from paper_2106_06161_gb300 import build
    build.build()
    import paper_2106_06161_gb300
    paper_2106_06161_gb300.load()
    assert paper_2106_06161_gb300.bshuffle_get_strategy() == paper_2106_06161_gb300.BSHUFFLE_STRATEGY_AUTO
    return paper_2106_06161_gb300


def _oracle_idx_on_device(n: int, seed: int) -> torch.Tensor:
    idx = oracle.indices_mt(n, seed)
    assert idx.size == n
    return torch.from_numpy(idx.view(np.int64)).cuda()


def _check_payload(bs, n: int, width: int, seed: int, idx_d: torch.Tensor):
    x = workloads.sweep_payload(n, width, seed)
    xd = to_device(x)
    y = bs.permute(xd, seed)
    assert_no_device_error()
    assert y.shape == xd.shape
    want = xd[idx_d]                       # slot j holds x[f(i_j)]
    assert torch.equal(y, want), (n, width, seed)
    del x, xd, y, want
    torch.cuda.empty_cache()


@pytest.mark.parametrize("seed", workloads.SWEEP_SEEDS)
@pytest.mark.parametrize("n", FULL_SIZES)
def test_full_size_u64_every_slot(bs, n, seed):
    idx_d = _oracle_idx_on_device(n, seed)
    got = bs.indices(n, seed, dtype=torch.int64)
    assert_no_device_error()
    assert torch.equal(got, idx_d), (n, seed)
    del got
    _check_payload(bs, n, 8, seed, idx_d)
    if seed == 0:
        for width in (4, 16):
            _check_payload(bs, n, width, seed, idx_d)


def test_full_size_staged_inverse_every_slot(bs):
    # the inverse shuffle at n = 2^28 uint64 (staged with the forward
    # cipher): slot f(j) receives x[j] for every j, and permute undoes it
    n, seed = 2**28, 3
    idx_d = _oracle_idx_on_device(n, seed)
    x = workloads.uniform_u64(n, seed)
    xd = to_device(x)
    y = bs.inverse(xd, seed)
    assert_no_device_error()
    assert torch.equal(y[idx_d], xd)
    z = bs.permute(y, seed)
    assert_no_device_error()
    assert torch.equal(z, xd)
