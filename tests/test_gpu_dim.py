"""The tensor API along a dimension other than 0: permute(x, seed, dim=d)
shuffles the slices x.select(d, i) as Algorithm 1 orders them, so it equals
indexing dimension d with the oracle's index sequence, and inverse undoes it."""
import numpy as np
import pytest
import torch

import oracle
from tests.gpu_helpers import assert_no_device_error

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def bs():
    from paper_2106_06161_gb300 import build
    build.build()
    import paper_2106_06161_gb300
    paper_2106_06161_gb300.load()
    return paper_2106_06161_gb300


def test_permute_and_inverse_along_a_dimension(bs):
    seed = 13
    g = torch.Generator(device="cpu").manual_seed(4)
    # rows after moving the dimension to the front: 64 B (dim 1), 16,016 B
    # (dims 0 and -1); the library takes rows of 1, 2, 4, 8 or 16 k bytes
    x = torch.randn(4, 1001, 4, generator=g).cuda()
    idx = torch.from_numpy(oracle.indices(1001, seed).astype(np.int64)).cuda()
    y = bs.permute(x, seed, dim=1)
    assert_no_device_error()
    assert y.is_contiguous() and torch.equal(y, x[:, idx, :])
    assert torch.equal(bs.inverse(y, seed, dim=1), x)
    # the last dimension, by its negative index (n = 4: the smallest domain, 2^4)
    idx4 = torch.from_numpy(oracle.indices(4, seed).astype(np.int64)).cuda()
    assert torch.equal(bs.permute(x, seed, dim=-1), x[..., idx4])
    # dim 0 and an explicit output
    assert torch.equal(bs.permute(x, seed, dim=0), x[idx4])
    out = torch.empty_like(x)
    assert bs.permute(x, seed, out=out, dim=1) is out
    assert torch.equal(out, x[:, idx, :])
    assert_no_device_error()
