"""CPU oracle for the bijective shuffle (arXiv 2106.06161).

TEST INFRASTRUCTURE ONLY.  Only the test-suite, ``__graft_entry__.smoke()`` and
the CPU-baseline leg of ``bench.py`` may import this package.  It shares no code
with the CUDA library in ``paper_2106_06161_gb300`` and never calls it; the
product path must not import it.

The arithmetic lives in ``bshuffle_oracle.c`` (plain sequential C, built with
gcc on first use; the ``*_mt`` functions run Algorithm 1 on several host
threads over consecutive domain ranges: count, exclusive scan, write).  This
module only marshals numpy arrays in and out.  The
statistical tests of Sec. 5 are in :mod:`oracle.stats`.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "bshuffle_oracle.c")
_BUILD_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD_DIR, "liboracle.so")
_lock = threading.Lock()
_lib = None

# Reading R2 of the oracle source: smallest domain exponent.
K_MIN = 4
DEFAULT_ROUNDS = 24  # Sec. 5: 24 rounds pass every test and are used throughout


def build(force: bool = False) -> str:
    """Compile the C oracle with gcc into oracle/_build/liboracle.so."""
    os.makedirs(_BUILD_DIR, exist_ok=True)
    stale = (not os.path.exists(_LIB_PATH)
             or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC))
    if force or stale:
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c99", "-Wall", "-pthread", "-shared", "-fPIC",
                               "-o", tmp, _SRC])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        # BSHUFFLE_ORACLE_LIB names another build of this source to load
        # instead: the test that plants mistakes in the oracle (each in a
        # temporary copy of bshuffle_oracle.c) runs the pins against it.
        lib = ctypes.CDLL(os.environ.get("BSHUFFLE_ORACLE_LIB") or build())
        u32, u64, p = ctypes.c_uint32, ctypes.c_uint64, ctypes.c_void_p
        sig = {
            "oracle_domain_bits": (u32, [u64]),
            "oracle_round_keys": (None, [u64, u32, p]),
            "oracle_varphilox": (u64, [u64, u32, p, u32]),
            "oracle_varphilox_inverse": (u64, [u64, u32, p, u32]),
            "oracle_m0_inverse": (u64, []),
            "oracle_varphilox_array": (None, [p, p, u64, u32, p, u32]),
            "oracle_varphilox_inverse_array": (None, [p, p, u64, u32, p, u32]),
            "oracle_indices_k": (u64, [p, u64, u32, u64, u32]),
            "oracle_indices": (u64, [p, u64, u64, u32]),
            "oracle_permute_k": (u64, [p, p, u64, u32, u32, u64, u32]),
            "oracle_permute": (u64, [p, p, u64, u32, u64, u32]),
            "oracle_permute_first": (u64, [p, p, u64, u32, u64, u32, u64]),
            "oracle_inverse": (u64, [p, p, u64, u32, u64, u32]),
            "oracle_count_range": (u64, [u64, u64, u32, u64, u64]),
            "oracle_default_threads": (u32, []),
            "oracle_indices_mt": (u64, [p, u64, u64, u32, u32]),
            "oracle_permute_mt": (u64, [p, p, u64, u32, u64, u32, u32]),
            "oracle_permute_range_mt": (u64, [p, p, u64, u32, u64, u32, u64, u64, u32]),
            "oracle_sample_permutations": (None, [p, u32, u64, u64, u32]),
            "oracle_fisher_yates": (None, [p, u64, u32, u64]),
            "oracle_mc_statistics": (None, [p, u64, u64, u64, u64, u32, p]),
            "oracle_kendall_discordant": (u64, [p, p, u32]),
            "oracle_kendall_pairs": (None, [p, u32, u64, p]),
            "oracle_lcg_params": (None, [u64, u32, p, p]),
            "oracle_lcg": (u64, [u64, u32, u64, u64]),
            "oracle_indices_lcg": (u64, [p, u64, u64]),
            "oracle_sample_permutations_lcg": (None, [p, u32, u64, u64]),
            "oracle_shapley_voting": (None, [p, u64, u64, u64, u64, u32, p]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
        return lib


def _ptr(a: np.ndarray) -> int:
    return a.ctypes.data


# ---------------------------------------------------------------- bijection

def domain_bits(n: int) -> int:
    """k = max(ceil(log2 n), 4); 0 for n = 0 (Sec. 4, reading R2)."""
    return int(_load().oracle_domain_bits(n))


def round_keys(seed: int, rounds: int = DEFAULT_ROUNDS) -> np.ndarray:
    """Per-round 32-bit keys from the seed (SplitMix64, reading R3)."""
    keys = np.zeros(max(rounds, 1), dtype=np.uint32)
    _load().oracle_round_keys(seed & (2**64 - 1), rounds, _ptr(keys))
    return keys[:rounds]


def _keys_arg(keys: np.ndarray) -> np.ndarray:
    keys = np.ascontiguousarray(keys, dtype=np.uint32)
    return keys if keys.size else np.zeros(1, dtype=np.uint32)


def varphilox(x, k: int, keys: np.ndarray) -> np.ndarray:
    """VariablePhilox image of each x in [0, 2^k) (Sec. 3.2, Listing 1)."""
    x = np.ascontiguousarray(np.asarray(x, dtype=np.uint64).reshape(-1))
    y = np.empty_like(x)
    kk = _keys_arg(keys)
    _load().oracle_varphilox_array(_ptr(x), _ptr(y), x.size, k, _ptr(kk), len(keys))
    return y


def varphilox_inverse(y, k: int, keys: np.ndarray) -> np.ndarray:
    """Inverse cipher following the inversion steps of Sec. 3.2."""
    y = np.ascontiguousarray(np.asarray(y, dtype=np.uint64).reshape(-1))
    x = np.empty_like(y)
    kk = _keys_arg(keys)
    _load().oracle_varphilox_inverse_array(_ptr(y), _ptr(x), y.size, k, _ptr(kk), len(keys))
    return x


def m0_inverse() -> int:
    return int(_load().oracle_m0_inverse())


# ---------------------------------------------------------------- Algorithm 1

def indices(n: int, seed: int, rounds: int = DEFAULT_ROUNDS, k: int | None = None) -> np.ndarray:
    """idx[j] = f(i_j): the source index of output slot j (Algorithm 1)."""
    idx = np.zeros(max(n, 1), dtype=np.uint64)
    if n == 0:
        return idx[:0]
    kk = domain_bits(n) if k is None else k
    got = _load().oracle_indices_k(_ptr(idx), n, kk, seed & (2**64 - 1), rounds)
    if got != n:
        raise ValueError(f"domain 2^{kk} kept {got} of {n} indices")
    return idx


def permute(x: np.ndarray, seed: int, rounds: int = DEFAULT_ROUNDS, k: int | None = None) -> np.ndarray:
    """Y[j] = X[f(i_j)] along axis 0; rows of any byte width are moved whole."""
    x = np.ascontiguousarray(x)
    n = x.shape[0]
    out = np.empty_like(x)
    if n == 0:
        return out
    elem_bytes = x.nbytes // n
    kk = domain_bits(n) if k is None else k
    got = _load().oracle_permute_k(_ptr(x), _ptr(out), n, elem_bytes, kk, seed & (2**64 - 1), rounds)
    if got != n:
        raise ValueError(f"domain 2^{kk} kept {got} of {n} elements")
    return out


def permute_first(x: np.ndarray, seed: int, slots: int, rounds: int = DEFAULT_ROUNDS) -> np.ndarray:
    """The first `slots` rows of permute(x, seed, rounds), computed alone."""
    x = np.ascontiguousarray(x)
    n = x.shape[0]
    slots = min(slots, n)
    out = np.empty((max(slots, 1),) + x.shape[1:], dtype=x.dtype)
    if n == 0 or slots == 0:
        return out[:0]
    got = _load().oracle_permute_first(_ptr(x), _ptr(out), n, x.nbytes // n, seed & (2**64 - 1), rounds, slots)
    if got != slots:
        raise ValueError("permute_first wrote a wrong count")
    return out


def inverse(y: np.ndarray, seed: int, rounds: int = DEFAULT_ROUNDS) -> np.ndarray:
    """X[f(i_j)] = Y[j]: undoes :func:`permute` for the same seed and rounds."""
    y = np.ascontiguousarray(y)
    n = y.shape[0]
    out = np.empty_like(y)
    if n == 0:
        return out
    elem_bytes = y.nbytes // n
    got = _load().oracle_inverse(_ptr(y), _ptr(out), n, elem_bytes, seed & (2**64 - 1), rounds)
    if got != n:
        raise ValueError("inverse kept a wrong count")
    return out


def count_range(n: int, seed: int, i0: int, i1: int, rounds: int = DEFAULT_ROUNDS) -> int:
    """Kept domain indices in [i0, i1) of the shuffle of length n: the range's
    share of Algorithm 1's exclusive scan."""
    return int(_load().oracle_count_range(n, seed & (2**64 - 1), rounds, i0, i1))


def default_threads() -> int:
    """Host threads the threaded functions use when given threads=0."""
    return int(_load().oracle_default_threads())


def indices_mt(n: int, seed: int, rounds: int = DEFAULT_ROUNDS, threads: int = 0) -> np.ndarray:
    """:func:`indices` computed by `threads` host threads over consecutive
    domain ranges (count, exclusive scan of the counts, write); same output."""
    idx = np.zeros(max(n, 1), dtype=np.uint64)
    if n == 0:
        return idx[:0]
    got = _load().oracle_indices_mt(_ptr(idx), n, seed & (2**64 - 1), rounds, threads)
    if got != n:
        raise ValueError(f"threaded indices kept {got} of {n}")
    return idx


def permute_mt(x: np.ndarray, seed: int, rounds: int = DEFAULT_ROUNDS, threads: int = 0) -> np.ndarray:
    """:func:`permute` computed by `threads` host threads (count, scan, gather)."""
    x = np.ascontiguousarray(x)
    n = x.shape[0]
    out = np.empty_like(x)
    if n == 0:
        return out
    got = _load().oracle_permute_mt(_ptr(x), _ptr(out), n, x.nbytes // n, seed & (2**64 - 1), rounds, threads)
    if got != n:
        raise ValueError(f"threaded permute kept {got} of {n}")
    return out


def permute_range_mt(x: np.ndarray, seed: int, first: int, end: int, rounds: int = DEFAULT_ROUNDS,
                     threads: int = 0) -> np.ndarray:
    """The kept elements of domain indices [first, end), in order: the output
    slots of that range of the shuffle, computed on host threads."""
    x = np.ascontiguousarray(x)
    n = x.shape[0]
    out = np.empty((max(min(n, max(end - first, 0)), 1),) + x.shape[1:], dtype=x.dtype)
    if n == 0 or end <= first:
        return out[:0]
    got = _load().oracle_permute_range_mt(_ptr(x), _ptr(out), n, x.nbytes // n, seed & (2**64 - 1), rounds,
                                          first, end, threads)
    return out[:got]


def sample_permutations(n: int, count: int, seed0: int = 0, rounds: int = DEFAULT_ROUNDS) -> np.ndarray:
    """count index arrays of length n from seeds seed0, seed0+1, ... (uint32)."""
    perms = np.zeros((count, n), dtype=np.uint32)
    _load().oracle_sample_permutations(_ptr(perms), n, seed0, count, rounds)
    return perms


def fisher_yates(x: np.ndarray, seed: int) -> np.ndarray:
    """Sequential Fisher-Yates (Durstenfeld) shuffle of a copy of x along axis 0."""
    y = np.ascontiguousarray(x).copy()
    n = y.shape[0]
    if n:
        _load().oracle_fisher_yates(_ptr(y), n, y.nbytes // n, seed & (2**64 - 1))
    return y


def mc_statistics(x: np.ndarray, n1: int, base_seed: int, count: int,
                  rounds: int = DEFAULT_ROUNDS) -> np.ndarray:
    """T_b = mean(y[:n1]) - mean(y[n1:]) of the shuffle with seed base_seed + b, FP64."""
    x = np.ascontiguousarray(x, dtype=np.float32)
    T = np.zeros(count, dtype=np.float64)
    _load().oracle_mc_statistics(_ptr(x), x.size, n1, base_seed, count, rounds, _ptr(T))
    return T


def kendall_discordant(s: np.ndarray, t: np.ndarray) -> int:
    s = np.ascontiguousarray(s, dtype=np.uint32)
    t = np.ascontiguousarray(t, dtype=np.uint32)
    return int(_load().oracle_kendall_discordant(_ptr(s), _ptr(t), s.size))


def kendall_pairs(perms: np.ndarray) -> np.ndarray:
    """n_dis of the consecutive pairs (0,1), (2,3), ... of a (count, n) array."""
    perms = np.ascontiguousarray(perms, dtype=np.uint32)
    count, n = perms.shape
    out = np.zeros(count // 2, dtype=np.uint64)
    _load().oracle_kendall_pairs(_ptr(perms), n, count // 2, _ptr(out))
    return out


def shapley_voting(weights: np.ndarray, quota: int, seed0: int, samples: int,
                   rounds: int = DEFAULT_ROUNDS) -> np.ndarray:
    """Pivot counts of the weighted voting game [quota; weights] over `samples`
    player orders, order s being the shuffle with seed seed0 + s."""
    w = np.ascontiguousarray(weights, dtype=np.uint32)
    counts = np.zeros(max(w.size, 1), dtype=np.uint64)
    _load().oracle_shapley_voting(_ptr(w), w.size, quota, seed0 & (2**64 - 1), samples, rounds, _ptr(counts))
    return counts[:w.size]


# ---------------------------------------------------------------- LCG (Sec. 3.1)

def lcg_params(seed: int, k: int) -> tuple[int, int]:
    """(a, c) of the LCG bijection for a seed on a 2^k domain (reading R6)."""
    a = ctypes.c_uint64(0)
    c = ctypes.c_uint64(0)
    _load().oracle_lcg_params(seed & (2**64 - 1), k, ctypes.addressof(a), ctypes.addressof(c))
    return a.value, c.value


def lcg(x: int, k: int, a: int, c: int) -> int:
    return int(_load().oracle_lcg(x, k, a, c))


def indices_lcg(n: int, seed: int) -> np.ndarray:
    """Algorithm 1 with the LCG of Sec. 3.1 as the bijection."""
    idx = np.zeros(max(n, 1), dtype=np.uint64)
    if n == 0:
        return idx[:0]
    got = _load().oracle_indices_lcg(_ptr(idx), n, seed & (2**64 - 1))
    if got != n:
        raise ValueError("LCG kept a wrong count")
    return idx


def permute_lcg(x: np.ndarray, seed: int) -> np.ndarray:
    x = np.ascontiguousarray(x)
    return x[indices_lcg(x.shape[0], seed).astype(np.int64)]


def sample_permutations_lcg(n: int, count: int, seed0: int = 0) -> np.ndarray:
    perms = np.zeros((count, n), dtype=np.uint32)
    _load().oracle_sample_permutations_lcg(_ptr(perms), n, seed0, count)
    return perms
