"""The statistical tests of Sec. 5 applied to the oracle, and pins of the test
harness itself: the Mallows-kernel closed forms against brute-force
enumeration of the symmetric group, the Kendall count against its definition,
and a generator outside this repository (numpy) as a uniform control."""
import itertools
import math

import numpy as np
import pytest

import oracle
from oracle import stats
from tests import golden


def _ndis_brute(s, t):
    n = len(s)
    c = 0
    for i in range(n):
        for j in range(i + 1, n):
            if (s[i] < s[j]) != (t[i] < t[j]):
                c += 1
    return c


def test_kendall_count_matches_definition():
    rng = np.random.default_rng(0)
    for n in (1, 2, 3, 7, 30, 101):
        for _ in range(20):
            s, t = rng.permutation(n), rng.permutation(n)
            assert oracle.kendall_discordant(s, t) == _ndis_brute(s, t)
    s = np.arange(50)
    assert oracle.kendall_discordant(s, s[::-1].copy()) == 50 * 49 // 2


@pytest.mark.parametrize("n", [2, 3, 4, 5, 6, 7])
def test_mallows_moments_match_enumeration(n):
    lam = stats.LAMBDA
    c = n * (n - 1) / 2
    ident = list(range(n))
    ks = [math.exp(-lam * _ndis_brute(ident, p) / c) for p in itertools.permutations(range(n))]
    mean = math.fsum(ks) / len(ks)
    var = math.fsum(k * k for k in ks) / len(ks) - mean * mean
    assert stats.mallows_expectation(n) == pytest.approx(mean, rel=1e-12)
    assert stats.mallows_variance(n) == pytest.approx(var, rel=1e-10)


def test_chi2_harness_controls():
    rng = np.random.default_rng(5)
    uniform = np.stack([rng.permutation(5) for _ in range(100_000)])
    chi2, dof, crit = stats.chi2_uniform(uniform)
    assert dof == 119 and crit == pytest.approx(145.46, abs=0.01)
    assert chi2 < crit
    ident = np.tile(np.arange(5), (1000, 1))
    assert stats.chi2_uniform(ident)[0] > crit


def test_chi2_n5_paper_round_count():
    # Sec. 5 (tests/golden): at n = 5 with 100,000 permutations, fewer than
    # 20 rounds are unlikely to be uniform, while 24 rounds pass.
    g = golden.load("sec5_chi2_n5.txt")
    n, perms = int(g["n"]), int(g["permutations"])
    idx24 = oracle.sample_permutations(n, perms, seed0=0, rounds=int(g["passing_rounds"]))
    chi24, dof, crit = stats.chi2_uniform(stats.ranks_from_indices(idx24))
    assert dof == int(g["dof"])
    assert chi24 < crit, chi24
    idx16 = oracle.sample_permutations(n, perms, seed0=0, rounds=int(g["failing_rounds"]))
    chi16, _, _ = stats.chi2_uniform(stats.ranks_from_indices(idx16))
    assert chi16 > crit, chi16


@pytest.mark.parametrize("n", [3, 4, 6])
def test_chi2_other_small_lengths_pass_at_24_rounds(n):
    idx = oracle.sample_permutations(n, 60_000, seed0=10_000, rounds=24)
    chi, _, crit = stats.chi2_uniform(stats.ranks_from_indices(idx))
    assert chi < crit, chi


def test_mmd_thresholds():
    assert stats.hoeffding_threshold(100_000) == pytest.approx(math.sqrt(math.log(40) / 1e5))
    # the asymptotic bound is tighter than Hoeffding's at |Pi| = 100,000 (Sec. 5)
    for n in (5, 100, 1000):
        assert stats.clt_threshold(n, 100_000) < stats.hoeffding_threshold(100_000)


def test_mmd_control_uniform_and_identity():
    rng = np.random.default_rng(1)
    sample = np.stack([rng.permutation(100) for _ in range(20_000)])
    assert abs(stats.mmd2_estimate(sample)) < stats.clt_threshold(100, 20_000)
    ident = np.tile(np.arange(100), (2000, 1))
    assert abs(stats.mmd2_estimate(ident)) > stats.hoeffding_threshold(2000)


@pytest.mark.parametrize("n", [5, 100, 1000])
def test_mmd_24_rounds_pass(n):
    # Sec. 5: 24 rounds pass the MMD tests at n = 5, 100 and 1000 (|Pi| = 100,000).
    idx = oracle.sample_permutations(n, 100_000, seed0=0, rounds=24)
    mmd = stats.mmd2_estimate(stats.ranks_from_indices(idx))
    assert abs(mmd) < stats.clt_threshold(n, 100_000), mmd
    assert abs(mmd) < stats.hoeffding_threshold(100_000)


def test_mmd_detects_too_few_rounds():
    idx = oracle.sample_permutations(100, 20_000, seed0=0, rounds=2)
    mmd = stats.mmd2_estimate(stats.ranks_from_indices(idx))
    assert abs(mmd) > stats.clt_threshold(100, 20_000), mmd


def test_chi2_lcg_fails_in_the_paper_region():
    # Sec. 5 (tests/golden): the LCG bijective function scores about 500,000
    # at n = 5 (100,000 permutations).
    g = golden.load("sec5_chi2_n5.txt")
    lo, hi = (int(v) for v in g["lcg_chi2_range"].split())
    perms = oracle.sample_permutations_lcg(int(g["n"]), int(g["permutations"]), 0)
    chi, _, crit = stats.chi2_uniform(stats.ranks_from_indices(perms))
    assert lo < chi < hi, chi
    assert chi > 1000 * crit
