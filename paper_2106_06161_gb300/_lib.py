"""ctypes binding of libbshuffle.so with the C names of include/bshuffle.h.

Argument marshalling only: every function forwards to the C ABI of the
in-tree library and raises :class:`BShuffleError` on a negative return code.
There is no fallback: if the library has not been built, loading fails with
an error that says how to build it.
"""
from __future__ import annotations

import ctypes
import os
import threading

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libbshuffle.so")

BSHUFFLE_OK = 0
BSHUFFLE_ERR_NULL = -1
BSHUFFLE_ERR_ELEM = -2
BSHUFFLE_ERR_ROUNDS = -3
BSHUFFLE_ERR_TOO_LARGE = -4
BSHUFFLE_ERR_ALIAS = -5
BSHUFFLE_ERR_ALIGN = -6
BSHUFFLE_ERR_CUDA = -7
BSHUFFLE_ERR_LOOKBACK_TIMEOUT = -8
BSHUFFLE_ERR_DEVICE_BOUNDS = -9
BSHUFFLE_ERR_INVALID = -10
BSHUFFLE_STRATEGY_AUTO = 0
BSHUFFLE_STRATEGY_SINGLE_PASS = 1
BSHUFFLE_STRATEGY_STAGED = 2
BSHUFFLE_STRATEGY_PIPELINED = 3
BSHUFFLE_KERNEL_SINGLE_PASS = 0
BSHUFFLE_KERNEL_PIPELINED = 1
BSHUFFLE_KERNEL_BATCHED = 2
DEFAULT_ROUNDS = 24
MAX_ROUNDS = 64
MAX_N = 2**32 - 1

# Every function the header declares, with (restype, argtypes).
_u32, _u64, _i64, _p = ctypes.c_uint32, ctypes.c_uint64, ctypes.c_int64, ctypes.c_void_p
_int, _str = ctypes.c_int, ctypes.c_char_p
SIGNATURES = {
    "bshuffle_permute": (_int, [_p, _p, _u64, _u32, _u64, _u32, _p]),
    "bshuffle_indices": (_int, [_p, _u32, _u64, _u64, _u32, _p]),
    "bshuffle_inverse": (_int, [_p, _p, _u64, _u32, _u64, _u32, _p]),
    "bshuffle_batched": (_int, [_p, _u32, _u32, _u32, _p]),
    "bshuffle_get_error": (_int, [_p]),
    "bshuffle_last_cuda_error": (_int, []),
    "bshuffle_cuda_error_name": (_str, [_int]),
    "bshuffle_error_string": (_str, [_int]),
    "bshuffle_domain_bits": (_int, [_u64, ctypes.POINTER(_u32)]),
    "bshuffle_round_keys": (_int, [_u64, _u32, _p]),
    "bshuffle_release_workspaces": (_int, []),
    "bshuffle_set_lookback_timeout_ns": (_int, [_u64]),
    "bshuffle_debug_skip_publish": (_int, [_i64]),
    "bshuffle_debug_lookback_cycles": (_int, [_p, ctypes.POINTER(_u64), ctypes.POINTER(_u64)]),
    "bshuffle_version": (_int, []),
    "bshuffle_permute_static": (_int, [_p, _p, _u64, _u32, _u64, _u32, _p]),
    "bshuffle_mc_group_diff": (_int, [_p, _u64, _u64, _u64, _u32, _u32, _p, _p]),
    "bshuffle_shapley_voting": (_int, [_p, _u64, _u64, _u64, _u64, _u32, _p, _p]),
    "bshuffle_window_scatter": (_int, [_p, _p, _u64, _u32, _u32, _p]),
    "bshuffle_random_gather": (_int, [_p, _p, _u64, _u32, _p]),
    "bshuffle_set_strategy": (_int, [_int]),
    "bshuffle_get_strategy": (_int, []),
    "bshuffle_set_pass_timing": (_int, [_int]),
    "bshuffle_last_pass_ms": (_int, [_p, _p, _int]),
    "bshuffle_tuning_configs": (_int, []),
    "bshuffle_tuning_describe": (_int, [_int, ctypes.POINTER(_int), ctypes.POINTER(_int), ctypes.POINTER(_int)]),
    "bshuffle_tuning_select": (_int, [_u32, _int]),
    "bshuffle_tuning_selected": (_int, [_u32]),
    "bshuffle_kernel_configs": (_int, [_int]),
    "bshuffle_kernel_describe": (_int, [_int, _int, ctypes.POINTER(_int), ctypes.POINTER(_int),
                                        ctypes.POINTER(_int), ctypes.POINTER(_int)]),
    "bshuffle_kernel_select": (_int, [_int, _u32, _int]),
    "bshuffle_kernel_selected": (_int, [_int, _u32]),
    "bshuffle_permute_lcg": (_int, [_p, _p, _u64, _u32, _u64, _p]),
    "bshuffle_count_range": (_int, [_u64, _u64, _u32, _u64, _u64, _p, _p]),
    "bshuffle_permute_range": (_int, [_p, _p, _u64, _u32, _u64, _u32, _u64, _u64, _u64, _p]),
    "bshuffle_lcg_params": (_int, [_u64, _u64, ctypes.POINTER(_u64), ctypes.POINTER(_u64)]),
    "bshuffle_permute_ablation": (_int, [_p, _p, _u64, _u32, _u64, _u32, _int, _p]),
    "bshuffle_kendall_pairs": (_int, [_p, _u32, _u64, _p, _p]),
    "bshuffle_invert_rows": (_int, [_p, _u32, _u64, _p, _p]),
}

_lock = threading.Lock()
_lib = None


class BShuffleError(RuntimeError):
    """A negative return code of libbshuffle."""

    def __init__(self, code: int, where: str = ""):
        self.code = code
        self.cuda_error = 0
        msg = error_string(code) if _lib is not None else f"error {code}"
        if code == BSHUFFLE_ERR_CUDA and _lib is not None:
            self.cuda_error = _lib.bshuffle_last_cuda_error()
            msg += f" [{_lib.bshuffle_cuda_error_name(self.cuda_error).decode()}]"
        super().__init__(f"{where}: {msg} (code {code})" if where else f"{msg} (code {code})")


def load() -> ctypes.CDLL:
    """Load the in-tree libbshuffle.so (built by paper_2106_06161_gb300.build)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(
                    f"{LIB_PATH} is missing: build it with `python -m paper_2106_06161_gb300.build` "
                    "(or __graft_entry__.build()); there is no CPU fallback")
            lib = ctypes.CDLL(LIB_PATH)
            for name, (res, args) in SIGNATURES.items():
                fn = getattr(lib, name)
                fn.restype = res
                fn.argtypes = args
            _lib = lib
        return _lib


def _check(rc: int, where: str) -> int:
    if rc < 0:
        raise BShuffleError(rc, where)
    return rc


def error_string(code: int) -> str:
    return load().bshuffle_error_string(code).decode()


def bshuffle_permute(in_ptr: int, out_ptr: int, n: int, elem_bytes: int, seed: int,
                     rounds: int = DEFAULT_ROUNDS, stream: int = 0) -> None:
    _check(load().bshuffle_permute(in_ptr, out_ptr, n, elem_bytes, seed & (2**64 - 1), rounds, stream),
           "bshuffle_permute")


def bshuffle_indices(out_ptr: int, idx_bytes: int, n: int, seed: int, rounds: int = DEFAULT_ROUNDS,
                     stream: int = 0) -> None:
    _check(load().bshuffle_indices(out_ptr, idx_bytes, n, seed & (2**64 - 1), rounds, stream),
           "bshuffle_indices")


def bshuffle_inverse(in_ptr: int, out_ptr: int, n: int, elem_bytes: int, seed: int,
                     rounds: int = DEFAULT_ROUNDS, stream: int = 0) -> None:
    _check(load().bshuffle_inverse(in_ptr, out_ptr, n, elem_bytes, seed & (2**64 - 1), rounds, stream),
           "bshuffle_inverse")


def bshuffle_batched(descs_ptr: int, count: int, elem_bytes: int, rounds: int = DEFAULT_ROUNDS,
                     stream: int = 0) -> None:
    _check(load().bshuffle_batched(descs_ptr, count, elem_bytes, rounds, stream), "bshuffle_batched")


def bshuffle_mc_group_diff(x_ptr: int, n: int, n1: int, base_seed: int, count: int, rounds: int,
                           t_ptr: int, stream: int = 0) -> None:
    _check(load().bshuffle_mc_group_diff(x_ptr, n, n1, base_seed & (2**64 - 1), count, rounds, t_ptr, stream),
           "bshuffle_mc_group_diff")


def bshuffle_shapley_voting(w_ptr: int, n: int, quota: int, seed0: int, samples: int, rounds: int,
                            counts_ptr: int, stream: int = 0) -> None:
    _check(load().bshuffle_shapley_voting(w_ptr, n, quota, seed0 & (2**64 - 1), samples, rounds, counts_ptr, stream),
           "bshuffle_shapley_voting")


def bshuffle_window_scatter(in_ptr: int, out_ptr: int, n: int, elem_bytes: int, window_log2: int,
                            stream: int = 0) -> None:
    _check(load().bshuffle_window_scatter(in_ptr, out_ptr, n, elem_bytes, window_log2, stream),
           "bshuffle_window_scatter")


def bshuffle_random_gather(in_ptr: int, out_ptr: int, n: int, elem_bytes: int, stream: int = 0) -> None:
    _check(load().bshuffle_random_gather(in_ptr, out_ptr, n, elem_bytes, stream), "bshuffle_random_gather")


def bshuffle_get_error(stream: int = 0) -> int:
    """Device-side error recorded on the stream since the last call (0 = none)."""
    return load().bshuffle_get_error(stream)


def bshuffle_last_cuda_error() -> int:
    """cudaError_t behind the latest BSHUFFLE_ERR_CUDA on this thread (0 = none)."""
    return load().bshuffle_last_cuda_error()


def bshuffle_cuda_error_name(error: int) -> str:
    return load().bshuffle_cuda_error_name(error).decode()


def bshuffle_domain_bits(n: int) -> int:
    k = _u32(0)
    _check(load().bshuffle_domain_bits(n, ctypes.byref(k)), "bshuffle_domain_bits")
    return k.value


def bshuffle_round_keys(seed: int, rounds: int = DEFAULT_ROUNDS) -> list[int]:
    buf = (_u32 * max(rounds, 1))()
    _check(load().bshuffle_round_keys(seed & (2**64 - 1), rounds, ctypes.addressof(buf)),
           "bshuffle_round_keys")
    return [int(buf[i]) for i in range(rounds)]


def bshuffle_release_workspaces() -> None:
    _check(load().bshuffle_release_workspaces(), "bshuffle_release_workspaces")


def bshuffle_set_lookback_timeout_ns(ns: int) -> None:
    _check(load().bshuffle_set_lookback_timeout_ns(ns), "bshuffle_set_lookback_timeout_ns")


def bshuffle_debug_skip_publish(tile: int) -> None:
    _check(load().bshuffle_debug_skip_publish(tile), "bshuffle_debug_skip_publish")


def bshuffle_set_strategy(strategy: int) -> None:
    _check(load().bshuffle_set_strategy(strategy), "bshuffle_set_strategy")


def bshuffle_get_strategy() -> int:
    return load().bshuffle_get_strategy()


def bshuffle_set_pass_timing(on: bool) -> None:
    _check(load().bshuffle_set_pass_timing(1 if on else 0), "bshuffle_set_pass_timing")


def bshuffle_last_pass_ms(stream: int = 0) -> list[float]:
    buf = (ctypes.c_float * 8)()
    count = _check(load().bshuffle_last_pass_ms(stream, ctypes.addressof(buf), 8), "bshuffle_last_pass_ms")
    return [float(buf[i]) for i in range(count)]


def bshuffle_tuning_configs() -> list[dict]:
    """Every configuration of the tunable single-pass kernel."""
    out = []
    for c in range(load().bshuffle_tuning_configs()):
        b, i, r = _int(0), _int(0), _int(0)
        _check(load().bshuffle_tuning_describe(c, ctypes.byref(b), ctypes.byref(i), ctypes.byref(r)),
               "bshuffle_tuning_describe")
        out.append({"config": c, "block": b.value, "items": i.value, "rounds_unrolled": r.value})
    return out


def bshuffle_kernel_configs(kernel: int) -> list[dict]:
    """Every configuration of a tunable kernel (BSHUFFLE_KERNEL_*)."""
    count = _check(load().bshuffle_kernel_configs(kernel), "bshuffle_kernel_configs")
    out = []
    for c in range(count):
        t, i, m, r = _int(0), _int(0), _int(0), _int(0)
        _check(load().bshuffle_kernel_describe(kernel, c, ctypes.byref(t), ctypes.byref(i), ctypes.byref(m),
                                               ctypes.byref(r)), "bshuffle_kernel_describe")
        out.append({"config": c, "threads": t.value, "items": i.value, "ctas_per_sm": m.value,
                    "rounds_unrolled": r.value})
    return out


def bshuffle_kernel_select(kernel: int, elem_bytes: int, config: int) -> None:
    _check(load().bshuffle_kernel_select(kernel, elem_bytes, config), "bshuffle_kernel_select")


def bshuffle_kernel_selected(kernel: int, elem_bytes: int) -> int:
    return _check(load().bshuffle_kernel_selected(kernel, elem_bytes), "bshuffle_kernel_selected")


def bshuffle_tuning_select(elem_bytes: int, config: int) -> None:
    _check(load().bshuffle_tuning_select(elem_bytes, config), "bshuffle_tuning_select")


def bshuffle_tuning_selected(elem_bytes: int) -> int:
    return load().bshuffle_tuning_selected(elem_bytes)


def bshuffle_permute_lcg(in_ptr: int, out_ptr: int, n: int, elem_bytes: int, seed: int, stream: int = 0) -> None:
    _check(load().bshuffle_permute_lcg(in_ptr, out_ptr, n, elem_bytes, seed & (2**64 - 1), stream),
           "bshuffle_permute_lcg")


def bshuffle_count_range(n: int, seed: int, rounds: int, first: int, end: int, count_ptr: int,
                         stream: int = 0) -> None:
    _check(load().bshuffle_count_range(n, seed & (2**64 - 1), rounds, first, end, count_ptr, stream),
           "bshuffle_count_range")


def bshuffle_permute_range(in_ptr: int, out_ptr: int, n: int, elem_bytes: int, seed: int, rounds: int,
                           first: int, end: int, out_capacity: int, stream: int = 0) -> None:
    _check(load().bshuffle_permute_range(in_ptr, out_ptr, n, elem_bytes, seed & (2**64 - 1), rounds, first, end,
                                         out_capacity, stream), "bshuffle_permute_range")


def bshuffle_lcg_params(seed: int, n: int) -> tuple[int, int]:
    a, c = _u64(0), _u64(0)
    _check(load().bshuffle_lcg_params(seed & (2**64 - 1), n, ctypes.byref(a), ctypes.byref(c)),
           "bshuffle_lcg_params")
    return a.value, c.value


def bshuffle_permute_ablation(in_ptr: int, out_ptr: int, n: int, elem_bytes: int, seed: int, rounds: int,
                              variant: int, stream: int = 0) -> None:
    _check(load().bshuffle_permute_ablation(in_ptr, out_ptr, n, elem_bytes, seed & (2**64 - 1), rounds, variant,
                                            stream), "bshuffle_permute_ablation")


def bshuffle_kendall_pairs(perms_ptr: int, n: int, num_pairs: int, out_ptr: int, stream: int = 0) -> None:
    _check(load().bshuffle_kendall_pairs(perms_ptr, n, num_pairs, out_ptr, stream), "bshuffle_kendall_pairs")


def bshuffle_invert_rows(idx_ptr: int, n: int, rows: int, sigma_ptr: int, stream: int = 0) -> None:
    _check(load().bshuffle_invert_rows(idx_ptr, n, rows, sigma_ptr, stream), "bshuffle_invert_rows")


def bshuffle_version() -> int:
    return load().bshuffle_version()
