"""The GPU statistical harness (Sec. 5) against the oracle: Kendall counts are
integers and must match exactly; sampled ranks must equal the oracle's
permutations; the MMD^2 estimate must agree to FP64 rounding; and the
round-count result of Sec. 5 must hold at n = 100 and 1000."""
import numpy as np
import pytest
import torch

import oracle
from oracle import stats as ostats

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def st():
    from paper_2106_06161_gb300 import build
    build.build()
    import paper_2106_06161_gb300
    paper_2106_06161_gb300.load()
    from paper_2106_06161_gb300 import stats
    return stats


def test_kendall_counts_exact(st):
    rng = np.random.default_rng(0)
    for n in (1, 2, 7, 100, 1001, 4096):
        perms = np.stack([rng.permutation(n) for _ in range(40)]).astype(np.uint32)
        got = st.kendall_pairs(torch.from_numpy(perms.view(np.int32)).cuda()).cpu().numpy()
        assert np.array_equal(got.astype(np.uint64), oracle.kendall_pairs(perms)), n


def test_sampled_ranks_equal_oracle(st):
    for n in (5, 100, 1000):
        ranks = st.sample_ranks(n, 64, seed0=17).cpu().numpy()
        want = ostats.ranks_from_indices(oracle.sample_permutations(n, 64, seed0=17))
        assert np.array_equal(ranks.astype(np.int64), want.astype(np.int64)), n


def test_mmd_estimate_matches_oracle(st):
    n, count = 100, 20_000
    gpu = st.mmd2_estimate(st.sample_ranks(n, count, 0))
    ref = ostats.mmd2_estimate(ostats.ranks_from_indices(oracle.sample_permutations(n, count, 0)))
    assert abs(gpu - ref) <= 1e-12 + 1e-9 * abs(ref)
    assert st.mallows_expectation(n) == pytest.approx(ostats.mallows_expectation(n), rel=1e-13)
    assert st.clt_threshold(n, count) == pytest.approx(ostats.clt_threshold(n, count), rel=1e-13)


@pytest.mark.parametrize("n", [100, 1000])
def test_round_count_result_on_gpu(st, n):
    # Sec. 5: 24 rounds pass the MMD tests with |Pi| = 100,000; too few rounds fail.
    ok = st.mmd_test(n, 100_000, rounds=24)
    assert ok["passes_clt"] and ok["passes_hoeffding"], ok
    bad = st.mmd_test(n, 100_000, rounds=2)
    assert not bad["passes_clt"], bad
