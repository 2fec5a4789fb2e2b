"""Pins of the oracle's VariablePhilox bijection (Sec. 3.2) against facts that do
not come from the oracle itself: the exhaustive bijection property, the
inversion equations of Sec. 3.2, the text's F/B/G description of one round,
published SplitMix64 outputs, and closed-form degenerate cases."""
import numpy as np
import pytest

import oracle
from tests import golden

M0 = 0xD2B74407B1CE6E93  # the Philox constant printed in Listing 1
MASK64 = (1 << 64) - 1


def test_domain_bits_is_nearest_power_of_two_with_floor_4():
    # Sec. 4: the smallest power of two >= n, floored at 2^4 (reading R2).
    assert oracle.domain_bits(0) == 0
    for n in range(1, 17):
        assert oracle.domain_bits(n) == 4
    assert oracle.domain_bits(17) == 5
    assert oracle.domain_bits(2**20) == 20
    assert oracle.domain_bits(2**20 + 1) == 21
    assert oracle.domain_bits(1_000_003) == 20
    assert oracle.domain_bits(2**28) == 28
    assert oracle.domain_bits(2**28 + 12345) == 29
    for n in [33, 1000, 65535, 65536, 65537, 123457]:
        k = oracle.domain_bits(n)
        assert 2**k >= n and 2 ** (k - 1) < n


def test_round_keys_are_splitmix64_outputs():
    # The first three outputs of the published SplitMix64 generator from
    # state 0 (tests/golden); the round keys are their low 32 bits.
    g = golden.load("splitmix64_state0.txt")
    outputs = [int(v, 16) for v in g["outputs"].split()]
    keys = oracle.round_keys(int(g["seed"]), len(outputs))
    assert [int(k) for k in keys] == [v & 0xFFFFFFFF for v in outputs]
    assert [int(k) for k in keys] == [0x7B1DCDAF, 0xA1B965F4, 0x8009454F]
    # keys depend on the seed only, not on n, and a prefix is stable
    assert np.array_equal(oracle.round_keys(7, 24)[:10], oracle.round_keys(7, 10))
    assert not np.array_equal(oracle.round_keys(7, 24), oracle.round_keys(8, 24))


def test_m0_inverse_modulo_2_64():
    inv = oracle.m0_inverse()
    assert (M0 * inv) & MASK64 == 1


@pytest.mark.parametrize("rounds", [0, 1, 2, 24])
@pytest.mark.parametrize("seed", [0, 1, 12345])
def test_exhaustive_bijectivity_small_domains(rounds, seed):
    # Sec. 3.2: VariablePhilox is a bijection on [0, 2^k) for every k.
    keys = oracle.round_keys(seed, rounds)
    for k in range(1, 17):
        x = np.arange(2**k, dtype=np.uint64)
        y = oracle.varphilox(x, k, keys)
        assert y.max() < 2**k
        assert np.array_equal(np.sort(y), x), f"k={k} not a permutation"


def test_bijectivity_k20_and_k21():
    keys = oracle.round_keys(99, 24)
    for k in (20, 21):
        x = np.arange(2**k, dtype=np.uint64)
        y = oracle.varphilox(x, k, keys)
        assert np.array_equal(np.sort(y), x)


def test_zero_rounds_is_identity():
    for k in range(1, 33):
        x = np.random.default_rng(k).integers(0, 2**k, size=200, dtype=np.uint64)
        assert np.array_equal(oracle.varphilox(x, k, np.zeros(0, np.uint32)), x)


@pytest.mark.parametrize("k", list(range(1, 17)) + [20, 21, 29, 32])
def test_inverse_cipher_round_trip(k):
    # Inversion equations of Sec. 3.2: f^-1(f(x)) = x and f(f^-1(y)) = y.
    keys = oracle.round_keys(1000 + k, 24)
    if k <= 16:
        x = np.arange(2**k, dtype=np.uint64)
    else:
        x = np.random.default_rng(k).integers(0, 2**k, size=50_000, dtype=np.uint64)
    y = oracle.varphilox(x, k, keys)
    assert np.array_equal(oracle.varphilox_inverse(y, k, keys), x)
    assert np.array_equal(oracle.varphilox(oracle.varphilox_inverse(x, k, keys), k, keys), x)


def _text_round(state: int, k: int, key: int) -> int:
    """One round written from the prose of Sec. 3.2, not from Listing 1.

    The state is (L, R, b): L has floor(k/2) bits, R has floor(k/2) bits and b
    is the odd bit (present when k is odd), stored above R.  Multiplying L by
    the odd constant M0 gives upper bits forming F and lower bits forming the
    bijection B (Philox); L' = F_k(L) xor R; G inserts b below B_k(L) and the
    bit pushed out at the top becomes b'.
    """
    half = k // 2
    odd = k - 2 * half
    right_bits = half + odd
    left = state >> right_bits
    right_full = state & ((1 << right_bits) - 1)
    r = right_full & ((1 << half) - 1)
    b = right_full >> half
    product = (M0 * left) & MASK64
    f = ((product >> 32) ^ key) & ((1 << half) - 1)
    bij = product & ((1 << half) - 1)
    new_left = f ^ r
    if odd:
        g = (bij << 1) | b          # b' is bit `half` of g, R' its low bits
        new_right = g
    else:
        new_right = bij
    return (new_left << right_bits) | new_right


@pytest.mark.parametrize("k", [2, 3, 4, 5, 8, 9, 12, 13, 20, 29])
def test_rounds_match_text_description(k):
    rng = np.random.default_rng(k)
    keys = rng.integers(0, 2**32, size=24, dtype=np.uint32)
    xs = rng.integers(0, 2**k, size=300, dtype=np.uint64)
    for rounds in (1, 2, 24):
        got = oracle.varphilox(xs, k, keys[:rounds])
        for x, g in zip(xs.tolist(), got.tolist()):
            s = x
            for r in range(rounds):
                s = _text_round(s, k, int(keys[r]))
            assert g == s


def test_feistel_structure_of_one_round():
    # L' = F_k(L) xor R: flipping bits of R flips the same bits of L' and
    # leaves the new right half (a function of L and b only) unchanged.
    k, half = 16, 8
    keys = np.array([0xDEADBEEF], dtype=np.uint32)
    base = np.arange(0, 2**k, 257, dtype=np.uint64)
    for delta in (1, 0x10, 0x80, 0xFF):
        y0 = oracle.varphilox(base, k, keys)
        y1 = oracle.varphilox(base ^ np.uint64(delta), k, keys)
        assert np.array_equal((y0 ^ y1) >> np.uint64(half), np.full_like(y0, delta))
        assert np.array_equal(y0 & np.uint64(0xFF), y1 & np.uint64(0xFF))


def test_literal_one_bit_domain_is_identity():
    # With k = 1 the left half is empty: F = 0, B is the empty map and G just
    # moves b back in place, so every key gives the identity.
    for seed in range(50):
        keys = oracle.round_keys(seed, 24)
        assert oracle.varphilox(np.arange(2, dtype=np.uint64), 1, keys).tolist() == [0, 1]


def test_literal_tiny_domains_are_affine():
    # With k <= 3 the left half has one bit, so M0 * L is linear over GF(2)
    # and each round is x -> A x + c(key): at most 2^k distinct permutations.
    # This is why the domain floor of 2^4 is taken (reading R2).
    for k in (2, 3):
        seen = set()
        for seed in range(300):
            keys = oracle.round_keys(seed, 24)
            seen.add(tuple(oracle.varphilox(np.arange(2**k, dtype=np.uint64), k, keys).tolist()))
        assert len(seen) <= 2**k
    seen4 = set()
    for seed in range(300):
        keys = oracle.round_keys(seed, 24)
        seen4.add(tuple(oracle.varphilox(np.arange(16, dtype=np.uint64), 4, keys).tolist()))
    assert len(seen4) > 250   # 4 bits: no longer affine, almost all distinct


def test_lcg_is_a_bijection_with_constant_stride():
    # Sec. 3.1: y = a x + c mod 2^k is a bijection when a is coprime to 2^k
    # (odd); consecutive inputs map a constant stride a apart.
    for k in range(4, 17):
        for seed in (0, 9):
            a, c = oracle.lcg_params(seed, k)
            assert a % 2 == 1 and a < 2**k and c < 2**k
            ys = [oracle.lcg(x, k, a, c) for x in range(2**k)] if k <= 10 else None
            if ys is not None:
                assert sorted(ys) == list(range(2**k))
                assert all((ys[x + 1] - ys[x]) % 2**k == a for x in range(2**k - 1))
    idx = oracle.indices_lcg(1000, 3)
    assert np.array_equal(np.sort(idx), np.arange(1000, dtype=np.uint64))
