"""Pins of the oracle's arbitrary-length shuffle (Sec. 4, Algorithm 1): brute
force on small inputs, the Sec. 2 worked example of the permutation
convention, and invariants that hold at any size."""
import math

import numpy as np
import pytest

import oracle
import workloads
from oracle import stats
from tests import golden


def _brute_force_indices(n, seed, rounds, k):
    """Algorithm 1 by its definition: keep f(i) < n in increasing i."""
    keys = oracle.round_keys(seed, rounds)
    dom = np.arange(2**k, dtype=np.uint64)
    img = oracle.varphilox(dom, k, keys)
    return img[img < n]


@pytest.mark.parametrize("n", [1, 2, 3, 5, 7, 16, 17, 31, 100, 1000, 4097])
def test_indices_follow_algorithm_1(n):
    for seed in (0, 3):
        idx = oracle.indices(n, seed)
        k = oracle.domain_bits(n)
        assert np.array_equal(idx, _brute_force_indices(n, seed, 24, k))
        assert np.array_equal(np.sort(idx), np.arange(n, dtype=np.uint64))


def test_kept_order_is_increasing_domain_index():
    n, seed = 1000, 5
    k = oracle.domain_bits(n)
    keys = oracle.round_keys(seed, 24)
    idx = oracle.indices(n, seed)
    pre = oracle.varphilox_inverse(idx, k, keys)     # i_j = f^-1(idx[j])
    assert np.all(np.diff(pre.astype(np.int64)) > 0)
    dropped = np.setdiff1d(np.arange(2**k, dtype=np.uint64), pre)
    assert np.all(oracle.varphilox(dropped, k, keys) >= n)


def test_power_of_two_length_drops_nothing():
    for k in (4, 10, 16):
        n = 2**k
        keys = oracle.round_keys(77, 24)
        assert np.array_equal(oracle.indices(n, 77),
                              oracle.varphilox(np.arange(n, dtype=np.uint64), k, keys))


def test_permute_of_iota_is_indices():
    for n in (5, 1000, 65537):
        x = workloads.iota(n, np.uint64)
        assert np.array_equal(oracle.permute(x, 9), oracle.indices(n, 9))


@pytest.mark.parametrize("width", [1, 2, 4, 8, 16, 48, 4096])
def test_permute_moves_whole_elements(width):
    n = 300
    rng = np.random.default_rng(width)
    x = rng.integers(0, 256, size=(n, width), dtype=np.uint8)
    y = oracle.permute(x, 1234)
    idx = oracle.indices(n, 1234).astype(np.int64)
    assert np.array_equal(y, x[idx])


def test_permute_first_is_a_prefix():
    for n in (17, 1000, 70001):
        x = workloads.uniform_u64(n, 3)
        full = oracle.permute(x, 8)
        for slots in (1, 5, n // 2, n):
            assert np.array_equal(oracle.permute_first(x, 8, slots), full[:slots])


def test_inverse_undoes_permute():
    for n in (1, 2, 17, 1000, 4099):
        x = workloads.uniform_u64(n, n)
        y = oracle.permute(x, 21)
        assert np.array_equal(oracle.inverse(y, 21), x)
        assert np.array_equal(oracle.permute(oracle.inverse(x, 21), 21), x)


def test_literal_domain_override():
    # The explicit-k entry point reproduces Algorithm 1 on a wider domain too.
    n = 100
    for k in (7, 9):
        assert np.array_equal(oracle.indices(n, 4, k=k), _brute_force_indices(n, 4, 24, k))


def test_sec2_worked_example_of_the_convention():
    # Sec. 2's example of one-line notation (tests/golden): slot j of a
    # shuffle output holds element idx[j], so sigma = idx^-1.
    g = golden.load("sec2_one_line_notation.txt")
    sigma = np.array([[int(v) for v in g["sigma"].split()]])
    items = np.array(g["items"].split())
    idx = np.argsort(sigma, axis=1)
    assert idx.tolist() == [[0, 2, 3, 1]]
    assert items[idx[0]].tolist() == g["reordered"].split()
    assert stats.ranks_from_indices(idx).tolist() == sigma.tolist()


def test_fisher_yates_is_a_permutation():
    x = workloads.uniform_u64(10_000, 1)
    y = oracle.fisher_yates(x, 3)
    assert np.array_equal(np.sort(x), np.sort(y))
    assert not np.array_equal(x, y)


def test_mc_statistic_closed_forms():
    x = workloads.mc_samples(group=500, seed=3)
    n1 = 500
    # zero rounds: the identity permutation, so T is the plain group-mean gap
    t0 = oracle.mc_statistics(x, n1, 0, 3, rounds=0)
    want = math.fsum(x[:n1].astype(np.float64)) / n1 - math.fsum(x[n1:].astype(np.float64)) / (x.size - n1)
    assert np.allclose(t0, want, rtol=1e-13, atol=1e-15)
    # any seed: T_b is the gap of the oracle's own permuted sample
    T = oracle.mc_statistics(x, n1, 100, 4)
    for b in range(4):
        y = oracle.permute(x, 100 + b).astype(np.float64)
        gap = math.fsum(y[:n1]) / n1 - math.fsum(y[n1:]) / (x.size - n1)
        assert abs(T[b] - gap) <= 1e-12 * max(1.0, abs(gap))


@pytest.mark.parametrize("threads", [1, 2, 3, 8, 0])
def test_threaded_algorithm_1_matches_brute_force(threads):
    # count per domain range, exclusive scan of the counts, write per range:
    # the same output as Algorithm 1 by its definition, for any split
    for n in (1, 2, 3, 5, 17, 1000, 4097, 65537):
        for seed in (0, 4):
            want = _brute_force_indices(n, seed, 24, oracle.domain_bits(n))
            assert np.array_equal(oracle.indices_mt(n, seed, threads=threads), want), (n, seed)
    x = workloads.uniform_u64(100_003, 1)
    want = x[_brute_force_indices(100_003, 6, 24, oracle.domain_bits(100_003)).astype(np.int64)]
    assert np.array_equal(oracle.permute_mt(x, 6, threads=threads), want)
    rows = np.random.default_rng(2).integers(0, 256, size=(5000, 48), dtype=np.uint8)
    want = rows[_brute_force_indices(5000, 7, 24, oracle.domain_bits(5000)).astype(np.int64)]
    assert np.array_equal(oracle.permute_mt(rows, 7, threads=threads), want)


def test_count_range_gives_the_scan_at_range_boundaries():
    # splitting the domain into consecutive ranges: each range's kept count,
    # scanned in range order, is the first output slot of the range, and the
    # slots of the range hold exactly the range's kept images in order
    n, seed = 3001, 12
    k = oracle.domain_bits(n)
    keys = oracle.round_keys(seed, 24)
    img = oracle.varphilox(np.arange(2**k, dtype=np.uint64), k, keys)
    idx = oracle.indices(n, seed)
    bounds = [0, 1, 700, 2048, 2049, 4000, 2**k]
    start = 0
    for i0, i1 in zip(bounds[:-1], bounds[1:]):
        c = oracle.count_range(n, seed, i0, i1)
        kept = img[i0:i1][img[i0:i1] < n]
        assert c == kept.size
        assert np.array_equal(idx[start:start + c], kept)
        start += c
    assert start == n
    assert oracle.count_range(n, seed, 0, 2**40) == n  # clipped to the domain
    assert oracle.count_range(n, seed, 5, 5) == 0


def test_threaded_range_gives_the_range_slots():
    # the kept elements of a domain range are the output slots that follow the
    # earlier ranges' counts
    n, seed = 50_001, 3
    x = workloads.uniform_u64(n, 8)
    full = oracle.permute(x, seed)
    start = 0
    for f, e in ((0, 1), (1, 4096), (4096, 40_000), (40_000, 2**16), (2**16, 2**40)):
        part = oracle.permute_range_mt(x, seed, f, e, threads=3)
        assert part.shape[0] == oracle.count_range(n, seed, f, e)
        assert np.array_equal(part, full[start:start + part.shape[0]]), (f, e)
        start += part.shape[0]
    assert start == n
