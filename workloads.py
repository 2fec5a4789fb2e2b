"""Seeded synthetic inputs shared by the tests, the smoke check and the benchmark.

This module draws data only: it holds none of the shuffle's arithmetic, so both
the CUDA library and the CPU oracle can be fed from it without sharing code.
Every generator is a pure function of its arguments (numpy PCG64 streams).

The shapes follow the paper's throughput experiments (Sec. 6: arrays of
64-bit keys, worst case 2^w + 1 elements) and the five workloads this library
is measured on:

* single shuffle of n = 1,000,003 uint32 iota values, seed 42, domain 2^20;
* bandwidth sweep: n in {2^10, 2^16, 2^20, 2^24, 2^28, 2^28 + 12345} for
  4-byte iota/uniform values, 8-byte uniform random keys and 16-byte
  {key, value} pairs, seeds 0..4;
* batched: 4096 independent shuffles, sizes log-uniform in [100, 2,000,000],
  int32 payloads, instance seed = base seed + instance id;
* row shuffle for autograd: [65536 x 1024] N(0, 1) in FP32 and BF16;
* permutation Monte Carlo: 50,000 + 50,000 float32 samples from N(0, 1) and
  N(0.05, 1), 10,000 shuffles.
"""
from __future__ import annotations

import numpy as np

SWEEP_SIZES = (2**10, 2**16, 2**20, 2**24, 2**28, 2**28 + 12345)
SWEEP_SEEDS = (0, 1, 2, 3, 4)
SINGLE_N = 1_000_003
SINGLE_SEED = 42
BATCH_COUNT = 4096
BATCH_MIN, BATCH_MAX = 100, 2_000_000
MC_GROUP = 50_000
MC_SHIFT = 0.05
MC_SHUFFLES = 10_000
ROWS_SHAPE = (65536, 1024)
ROWS_SEED = 7
VOTING_PLAYERS = 10_000
VOTING_SAMPLES = 100_000


def _rng(seed: int) -> np.random.Generator:
    return np.random.default_rng(np.random.PCG64(seed))


def iota(n: int, dtype=np.uint32) -> np.ndarray:
    """in[i] = i."""
    return np.arange(n, dtype=dtype)


def uniform_u32(n: int, seed: int) -> np.ndarray:
    return _rng(seed).integers(0, 2**32, size=n, dtype=np.uint32)


def uniform_u64(n: int, seed: int) -> np.ndarray:
    """Uniform random 64-bit keys (the paper's Sec. 6 payload)."""
    return _rng(seed).integers(0, 2**64 - 1, size=n, dtype=np.uint64, endpoint=True)


def key_value_pairs(n: int, seed: int) -> np.ndarray:
    """n records of {uint64 key, uint64 value}: a (n, 2) uint64 array, 16 B per row."""
    rng = _rng(seed)
    out = np.empty((n, 2), dtype=np.uint64)
    out[:, 0] = rng.integers(0, 2**64 - 1, size=n, dtype=np.uint64, endpoint=True)
    out[:, 1] = np.arange(n, dtype=np.uint64)
    return out


def sweep_payload(n: int, elem_bytes: int, seed: int) -> np.ndarray:
    """The sweep's payload for one width: 4 B uniform, 8 B keys, 16 B key/value."""
    if elem_bytes == 4:
        return uniform_u32(n, seed)
    if elem_bytes == 8:
        return uniform_u64(n, seed)
    if elem_bytes == 16:
        return key_value_pairs(n, seed)
    raise ValueError(f"no sweep payload of {elem_bytes} bytes")


def batched_sizes(count: int = BATCH_COUNT, lo: int = BATCH_MIN, hi: int = BATCH_MAX,
                  seed: int = 2024) -> np.ndarray:
    """floor(exp(U(ln lo, ln hi))) per instance, as int64."""
    u = _rng(seed).uniform(np.log(lo), np.log(hi), size=count)
    return np.floor(np.exp(u)).astype(np.int64)


def batched_payloads(sizes: np.ndarray, seed: int = 99) -> np.ndarray:
    """One int32 array holding every instance back to back."""
    total = int(np.asarray(sizes).sum())
    return _rng(seed).integers(-2**31, 2**31 - 1, size=total, dtype=np.int32, endpoint=True)


def mc_samples(group: int = MC_GROUP, shift: float = MC_SHIFT, seed: int = 11) -> np.ndarray:
    """Two groups of N(0,1) and N(shift,1), concatenated, float32."""
    rng = _rng(seed)
    a = rng.standard_normal(group)
    b = rng.standard_normal(group) + shift
    return np.concatenate([a, b]).astype(np.float32)


def normal_rows(rows: int, cols: int, seed: int = ROWS_SEED) -> np.ndarray:
    """A [rows x cols] float32 N(0,1) matrix (cast to BF16 by the caller if needed)."""
    return _rng(seed).standard_normal((rows, cols), dtype=np.float32)


def voting_weights(n: int = VOTING_PLAYERS, seed: int = 31) -> np.ndarray:
    """Player weights of a weighted voting game: 1 + floor(LogNormal(2, 1)),
    uint32 (a few heavy players among many light ones)."""
    return (1 + np.floor(_rng(seed).lognormal(2.0, 1.0, size=n))).astype(np.uint32)


def majority_quota(weights: np.ndarray) -> int:
    """Simple majority of the total weight."""
    return int(np.asarray(weights, dtype=np.int64).sum()) // 2 + 1
