"""Shapley values of weighted voting games by permutation sampling (an
application named in Sec. 1): the exact values against enumeration of every
player order and against published results, then the oracle's sampling
estimate against the exact values."""
import itertools
import math
from fractions import Fraction

import numpy as np
import pytest

import oracle
from oracle.shapley import shapley_shubik
from tests import golden


def _by_enumeration(weights, quota):
    n = len(weights)
    piv = [0] * n
    for order in itertools.permutations(range(n)):
        before = 0
        for p in order:
            if before < quota <= before + weights[p]:
                piv[p] += 1
                break
            before += weights[p]
    return [Fraction(c, math.factorial(n)) for c in piv]


def test_exact_values_match_enumeration_of_orders():
    rng = np.random.default_rng(3)
    for n in range(1, 8):
        for _ in range(6):
            w = [int(x) for x in rng.integers(0, 7, size=n)]
            total = sum(w)
            for q in sorted({1, max(total // 2, 1), total, total + 1, 0}):
                assert shapley_shubik(w, q) == _by_enumeration(w, q), (w, q)


def test_small_textbook_game():
    # [5; 4, 2, 1]: of the 6 orders, the heaviest player is pivotal in the 4
    # where it does not come first; each of the others in one of the two
    # orders that start with the heaviest player.
    assert shapley_shubik([4, 2, 1], 5) == [Fraction(2, 3), Fraction(1, 6), Fraction(1, 6)]


def test_security_council_game():
    # The UN Security Council as analysed by Shapley and Shubik (1954), values
    # stored in tests/golden.
    g = golden.load("shapley_shubik_security_council.txt")
    weights = [int(v) for v in g["weights"].split()]
    want = [Fraction(v) for v in g["values"].split()]
    phi = shapley_shubik(weights, int(g["quota"]))
    assert phi == want
    assert phi[:5] == [Fraction(421, 2145)] * 5 and phi[5:] == [Fraction(4, 2145)] * 10


def test_exact_value_axioms():
    rng = np.random.default_rng(8)
    for _ in range(10):
        w = [int(x) for x in rng.integers(1, 12, size=14)] + [0, 0]
        q = int(rng.integers(1, sum(w) + 1))
        phi = shapley_shubik(w, q)
        assert sum(phi) == 1                      # efficiency
        assert phi[-1] == 0 and phi[-2] == 0      # null players
        for a in range(len(w)):                   # symmetry
            for b in range(len(w)):
                if w[a] == w[b]:
                    assert phi[a] == phi[b]
    assert shapley_shubik([3] * 9, 14) == [Fraction(1, 9)] * 9


def test_sampling_counts_invariants():
    w = np.array([5, 0, 3, 9, 1, 0, 2, 7, 4, 6, 8], dtype=np.uint32)
    total = int(w.sum())
    for q in (1, total // 3, total // 2 + 1, total):
        counts = oracle.shapley_voting(w, q, seed0=11, samples=3000)
        assert int(counts.sum()) == 3000
        assert counts[1] == 0 and counts[5] == 0
    for q in (0, total + 1):
        assert not oracle.shapley_voting(w, q, seed0=11, samples=500).any()
    assert oracle.shapley_voting(np.zeros(0, dtype=np.uint32), 3, 0, 10).size == 0


def test_sample_order_is_the_algorithm_1_shuffle():
    # sample s orders the players as the shuffle with seed seed0 + s: slot j
    # holds player idx[j]
    w = np.array([4, 1, 6, 2, 2, 9, 3, 5, 1, 7, 3, 8, 2, 6, 4, 1, 5, 3, 2], dtype=np.uint32)
    q = int(w.sum()) // 2 + 1
    for s in range(40):
        idx = oracle.indices(w.size, seed=100 + s)
        run = np.cumsum(w[idx].astype(np.int64))
        pivot = idx[int(np.argmax(run >= q))]
        counts = oracle.shapley_voting(w, q, seed0=100 + s, samples=1)
        assert int(np.argmax(counts)) == pivot and int(counts.sum()) == 1


def test_sampling_estimate_converges_to_exact():
    rng = np.random.default_rng(21)
    w = rng.integers(1, 10, size=12).astype(np.uint32)
    q = int(0.6 * int(w.sum()))
    samples = 40_000
    est = oracle.shapley_voting(w, q, seed0=0, samples=samples) / samples
    exact = np.array([float(x) for x in shapley_shubik(w.tolist(), q)])
    sd = np.sqrt(exact * (1 - exact) / samples)
    assert np.all(np.abs(est - exact) <= 4.5 * sd + 1e-12), (est, exact)


def test_unanimity_makes_the_last_player_pivotal():
    # quota = total weight with all weights positive: the last player of the
    # order is pivotal, so counts are uniform over players
    w = np.arange(1, 9, dtype=np.uint32)
    counts = oracle.shapley_voting(w, int(w.sum()), seed0=5, samples=16_000)
    expected = 16_000 / 8
    chi2 = float((((counts - expected) ** 2) / expected).sum())
    assert chi2 < 24.3  # 7 dof, alpha = 0.001
