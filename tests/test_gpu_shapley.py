"""Shapley values of weighted voting games by fused permutation sampling
against the oracle: pivot counts are integers, so the GPU counts must equal
the oracle's exactly for the same seeds."""
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


def _gpu(bs, w, q, seed0, samples, rounds=24):
    t = torch.from_numpy(np.ascontiguousarray(w, dtype=np.uint32).view(np.int32)).cuda()
    return bs.shapley_voting(t, q, seed0, samples, rounds).cpu().numpy().astype(np.uint64)


@pytest.mark.parametrize("n", [1, 3, 5, 16, 17, 1000, 2048, 2049, 4097, 70_001])
def test_counts_match_oracle(bs, n):
    rng = np.random.default_rng(n)
    w = rng.integers(0, 20, size=n).astype(np.uint32)
    w[0] = max(w[0], 1)
    total = int(w.sum())
    samples = 3000 if n <= 5000 else 150
    for q in sorted({1, total // 3 + 1, total // 2 + 1, total}):
        got = _gpu(bs, w, q, seed0=7 * n, samples=samples)
        want = oracle.shapley_voting(w, q, seed0=7 * n, samples=samples)
        np.testing.assert_array_equal(got, want)
        assert int(got.sum()) == samples


def test_textbook_game(bs):
    got = _gpu(bs, [4, 2, 1], 5, seed0=0, samples=60_000)
    np.testing.assert_array_equal(got, oracle.shapley_voting(np.array([4, 2, 1], np.uint32), 5, 0, 60_000))
    assert abs(got[0] / 60_000 - 2 / 3) < 0.01


def test_no_pivot_cases_and_rounds(bs):
    w = np.arange(1, 40, dtype=np.uint32)
    total = int(w.sum())
    assert not _gpu(bs, w, 0, 3, 100).any()
    assert not _gpu(bs, w, total + 1, 3, 100).any()
    for rounds in (0, 1, 7, 24, 64):
        np.testing.assert_array_equal(_gpu(bs, w, total // 2, 3, 500, rounds),
                                      oracle.shapley_voting(w, total // 2, 3, 500, rounds))
    assert bs.shapley_voting(torch.zeros(0, dtype=torch.int32, device="cuda"), 5, 0, 10).numel() == 0


def test_full_size_game(bs):
    # 10,000 players, lognormal weights, simple majority, 100,000 sampled orders
    w = workloads.voting_weights()
    q = workloads.majority_quota(w)
    got = _gpu(bs, w, q, seed0=0, samples=workloads.VOTING_SAMPLES)
    assert int(got.sum()) == workloads.VOTING_SAMPLES
    # the first 120 orders, counted one launch at a time and all together
    want = oracle.shapley_voting(w, q, seed0=0, samples=120)
    np.testing.assert_array_equal(_gpu(bs, w, q, seed0=0, samples=120), want)
    for s in (0, 57, 119):
        np.testing.assert_array_equal(_gpu(bs, w, q, seed0=s, samples=1),
                                      oracle.shapley_voting(w, q, seed0=s, samples=1))
    # heavier players are pivotal more often: compare the top and bottom deciles
    order = np.argsort(w, kind="stable")
    light = got[order[: w.size // 10]].sum()
    heavy = got[order[-(w.size // 10):]].sum()
    assert heavy > 5 * light
