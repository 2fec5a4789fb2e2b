"""Row shuffle and its autograd: [65536 x 1024] FP32 and BF16, permuting dim 0
with seed 7.  Forward must equal the oracle byte for byte; backward (a
scatter through the regenerated pairs, no stored index) must equal
index_select's autograd exactly; FP64 gradcheck on [64 x 8]."""
import numpy as np
import pytest
import torch

import oracle
import workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def bs():
    from paper_2106_06161_gb300 import build
    build.build()
    import paper_2106_06161_gb300
    paper_2106_06161_gb300.load()
    return paper_2106_06161_gb300


@pytest.mark.parametrize("extra_row", [0, 1])
@pytest.mark.parametrize("dtype", [torch.float32, torch.bfloat16])
def test_row_shuffle_forward_backward(bs, dtype, extra_row):
    # 65536 rows: the scan-free launch; 65537 rows (domain 2^17, about half
    # of the images dropped): the count kernel and the copy kernel
    rows, cols = workloads.ROWS_SHAPE
    rows += extra_row
    seed = workloads.ROWS_SEED
    host = torch.from_numpy(workloads.normal_rows(rows, cols)).to(dtype)
    x = host.cuda().requires_grad_(True)
    y = bs.shuffle_rows(x, seed)
    # forward: byte-exact against the oracle
    raw = host.view(torch.int16 if dtype == torch.bfloat16 else torch.int32).numpy()
    want = oracle.permute(raw, seed)
    got = y.detach().cpu().view(torch.int16 if dtype == torch.bfloat16 else torch.int32).numpy()
    assert np.array_equal(got, want)
    # backward: exact against index_select's autograd
    g = torch.from_numpy(workloads.normal_rows(rows, cols, seed=8)).to(dtype).cuda()
    y.backward(g)
    idx = bs.indices(rows, seed)
    x_ref = host.cuda().requires_grad_(True)
    y_ref = x_ref.index_select(0, idx)
    assert torch.equal(y_ref.detach(), y.detach())
    y_ref.backward(g)
    assert torch.equal(x.grad, x_ref.grad)
    assert bs.get_error() == 0


def test_gradcheck_fp64(bs):
    x = torch.randn(64, 8, dtype=torch.float64, device="cuda", requires_grad=True)
    assert torch.autograd.gradcheck(lambda t: bs.shuffle_rows(t, 7), (x,), eps=1e-6, atol=1e-9)
    # the Jacobian is a permutation matrix: each output row picks one input row
    y = bs.shuffle_rows(x, 7)
    jac = torch.autograd.functional.jacobian(lambda t: bs.shuffle_rows(t, 7), x).reshape(512, 512)
    assert torch.equal(jac.sum(0), torch.ones(512, dtype=torch.float64, device="cuda"))
    assert torch.equal(jac.sum(1), torch.ones(512, dtype=torch.float64, device="cuda"))
    assert torch.equal(y, x[bs.indices(64, 7)])


def test_row_widths_and_inverse(bs):
    # rows of 16 B to 4,112 B; 2,080 and 4,112 B rows are longer than 2 KiB
    # and not a whole number of 4 KiB blocks
    for cols, dt in ((2, torch.float64), (12, torch.float32), (1024, torch.float32), (6, torch.int64),
                     (4, torch.int16), (520, torch.float32), (1028, torch.float32)):
        for n in (1, 17, 300, 5000):
            x = torch.randn(n, cols, dtype=torch.float64).to(dt).cuda() if dt.is_floating_point else \
                torch.randint(-9, 9, (n, cols), dtype=dt).cuda()
            y = bs.permute(x, 3)
            assert torch.equal(y, x[bs.indices(n, 3)])
            assert torch.equal(bs.inverse(y, 3), x)
    with pytest.raises(bs.BShuffleError):
        bs.permute(torch.zeros(10, 3, dtype=torch.float64, device="cuda"), 1)   # 24-byte rows
