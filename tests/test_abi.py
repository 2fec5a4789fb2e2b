"""The C-ABI library on the CPU: it loads, exports every function that
include/bshuffle.h declares, its host-side arithmetic (domain exponent, key
schedule) agrees with the oracle, and argument errors are reported before any
CUDA call.  No compute call is made here."""
import ctypes
import os
import re

import numpy as np
import pytest

import oracle

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "bshuffle.h")


@pytest.fixture(scope="module")
def lib():
    from paper_2106_06161_gb300 import _lib, build
    build.build()
    return _lib.load()


def _declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(bshuffle_[a-z0-9_]+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = _declared_functions()
    for required in ("bshuffle_permute", "bshuffle_indices", "bshuffle_inverse", "bshuffle_batched",
                     "bshuffle_get_error", "bshuffle_error_string"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    from paper_2106_06161_gb300 import _lib
    for name in _declared_functions():
        assert hasattr(lib, name), name
        assert name in _lib.SIGNATURES, f"binding lacks {name}"


def test_exports_are_c_symbols():
    from paper_2106_06161_gb300 import _lib, build
    path = build.build()
    syms = ctypes.CDLL(path)
    for name in _declared_functions():
        ctypes.cast(getattr(syms, name), ctypes.c_void_p)  # resolvable without C++ mangling
    assert os.path.dirname(path).startswith(os.path.join(ROOT, "paper_2106_06161_gb300"))
    assert _lib.LIB_PATH == path


def test_domain_bits_agree_with_oracle(lib):
    from paper_2106_06161_gb300 import bshuffle_domain_bits
    for n in [1, 2, 5, 16, 17, 1000, 65536, 65537, 1_000_003, 2**28, 2**28 + 12345, 2**32 - 1]:
        assert bshuffle_domain_bits(n) == oracle.domain_bits(n), n


def test_round_keys_agree_with_oracle(lib):
    from paper_2106_06161_gb300 import bshuffle_round_keys
    for seed in [0, 1, 42, 2**63 + 5, 2**64 - 1]:
        for rounds in [0, 1, 24, 64]:
            assert bshuffle_round_keys(seed, rounds) == oracle.round_keys(seed, rounds).tolist()


def test_error_strings(lib):
    from paper_2106_06161_gb300 import error_string
    for code in range(0, -11, -1):
        s = error_string(code)
        assert s and "unknown" not in s
    assert "unknown" in error_string(-1234)


def test_argument_errors_precede_cuda(lib):
    from paper_2106_06161_gb300 import _lib as L
    buf = (ctypes.c_uint64 * 64)()
    a = ctypes.addressof(buf)
    p = lib.bshuffle_permute
    assert p(a, a + 256, 4, 8, 0, 65, None) == L.BSHUFFLE_ERR_ROUNDS
    assert p(a, a + 256, 4, 3, 0, 24, None) == L.BSHUFFLE_ERR_ELEM
    assert p(a, a + 256, 4, 24, 0, 24, None) == L.BSHUFFLE_ERR_ELEM
    assert p(None, a + 256, 4, 8, 0, 24, None) == L.BSHUFFLE_ERR_NULL
    assert p(a, a + 16, 4, 8, 0, 24, None) == L.BSHUFFLE_ERR_ALIAS
    assert p(a + 4, a + 256, 4, 8, 0, 24, None) == L.BSHUFFLE_ERR_ALIGN
    assert p(a, a + 256, 2**32, 1, 0, 24, None) == L.BSHUFFLE_ERR_TOO_LARGE
    assert p(a, a + 256, 0, 8, 0, 24, None) == L.BSHUFFLE_OK       # empty: no-op
    assert lib.bshuffle_inverse(a, a + 8, 4, 8, 0, 24, None) == L.BSHUFFLE_ERR_ALIAS
    assert lib.bshuffle_indices(a, 2, 4, 0, 24, None) == L.BSHUFFLE_ERR_ELEM
    assert lib.bshuffle_indices(None, 4, 4, 0, 24, None) == L.BSHUFFLE_ERR_NULL
    assert lib.bshuffle_indices(a + 2, 4, 4, 0, 24, None) == L.BSHUFFLE_ERR_ALIGN
    assert lib.bshuffle_batched(None, 0, 8, 24, None) == L.BSHUFFLE_OK
    assert lib.bshuffle_batched(None, 3, 8, 24, None) == L.BSHUFFLE_ERR_NULL
    assert lib.bshuffle_batched(a, 3, 8, 99, None) == L.BSHUFFLE_ERR_ROUNDS


def test_no_device_means_cuda_error(lib):
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_2106_06161_gb300 import _lib as L
    buf = (ctypes.c_uint64 * 64)()
    a = ctypes.addressof(buf)
    assert lib.bshuffle_permute(a, a + 256, 4, 8, 0, 24, None) == L.BSHUFFLE_ERR_CUDA
    # the cause is kept: the CUDA runtime's error of the failed call
    cause = lib.bshuffle_last_cuda_error()
    assert cause != 0
    name = lib.bshuffle_cuda_error_name(cause).decode()
    assert name.startswith("cuda") and name != "cudaSuccess"
    with pytest.raises(L.BShuffleError) as err:
        L.bshuffle_permute(a, a + 256, 4, 8, 0)
    assert err.value.cuda_error == cause and name in str(err.value)


def test_binding_has_no_cpu_fallback():
    # The product package must not reach the oracle or any CPU shuffle.
    pkg = os.path.join(ROOT, "paper_2106_06161_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                text = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in text and "from oracle" not in text, f
                assert "bshuffle_oracle" not in text, f


def test_lcg_params_agree_with_oracle(lib):
    from paper_2106_06161_gb300 import bshuffle_lcg_params
    for seed in (0, 1, 77, 2**64 - 1):
        for n in (5, 1000, 2**20 + 1, 2**28 + 12345):
            assert bshuffle_lcg_params(seed, n) == oracle.lcg_params(seed, oracle.domain_bits(n))


def test_shapley_argument_errors(lib):
    from paper_2106_06161_gb300 import _lib as L
    buf = (ctypes.c_uint64 * 64)()
    a = ctypes.addressof(buf)
    f = lib.bshuffle_shapley_voting
    assert f(a, 8, 5, 0, 10, 65, a + 256, None) == L.BSHUFFLE_ERR_ROUNDS
    assert f(None, 8, 5, 0, 10, 24, a + 256, None) == L.BSHUFFLE_ERR_NULL
    assert f(a, 8, 5, 0, 10, 24, None, None) == L.BSHUFFLE_ERR_NULL
    assert f(a + 2, 8, 5, 0, 10, 24, a + 256, None) == L.BSHUFFLE_ERR_ALIGN
    assert f(a, 8, 5, 0, 10, 24, a + 260, None) == L.BSHUFFLE_ERR_ALIGN
    assert f(a, 2**32, 5, 0, 10, 24, a + 256, None) == L.BSHUFFLE_ERR_TOO_LARGE
    assert f(None, 0, 5, 0, 10, 24, None, None) == L.BSHUFFLE_OK


def test_every_launch_path_fails_loudly_without_a_device(lib):
    # Lengths that take the scan-free launch (n = 2^k), the fused single pass
    # (other n) and the allocation-free entry point: without a device each
    # returns BSHUFFLE_ERR_CUDA, never a host-side result.
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_2106_06161_gb300 import _lib as L
    buf = (ctypes.c_uint64 * 64)()
    a = ctypes.addressof(buf)
    for n, elem in ((16, 8), (5, 8), (32, 4), (4, 32)):
        assert lib.bshuffle_permute(a, a + 256, n, elem, 0, 24, None) == L.BSHUFFLE_ERR_CUDA, (n, elem)
        assert lib.bshuffle_inverse(a, a + 256, n, elem, 0, 24, None) == L.BSHUFFLE_ERR_CUDA, (n, elem)
    for n in (16, 17):
        assert lib.bshuffle_indices(a, 8, n, 0, 24, None) == L.BSHUFFLE_ERR_CUDA
    assert lib.bshuffle_permute_static(a, a + 256, 16, 8, 0, 24, None) == L.BSHUFFLE_ERR_CUDA
    assert buf[:] == [0] * 64  # nothing was written on the host


def test_allocation_free_entry_point_argument_errors(lib):
    # size and width limits of the fixed scratch array are checked before
    # any CUDA call
    from paper_2106_06161_gb300 import _lib as L
    buf = (ctypes.c_uint64 * 64)()
    a = ctypes.addressof(buf)
    f = lib.bshuffle_permute_static
    assert f(a, a + 256, 2**27 + 1, 1, 0, 24, None) == L.BSHUFFLE_ERR_TOO_LARGE
    assert f(a, a + 256, 4, 32, 0, 24, None) == L.BSHUFFLE_ERR_ELEM
    assert f(a, a + 256, 4, 3, 0, 24, None) == L.BSHUFFLE_ERR_ELEM
    assert f(a, a + 256, 4, 8, 0, 65, None) == L.BSHUFFLE_ERR_ROUNDS
    assert f(a, a + 16, 4, 8, 0, 24, None) == L.BSHUFFLE_ERR_ALIAS
    assert f(a + 4, a + 256, 4, 8, 0, 24, None) == L.BSHUFFLE_ERR_ALIGN
    assert f(a, a + 256, 0, 8, 0, 24, None) == L.BSHUFFLE_OK


def test_kernel_shape_tables_on_the_host(lib):
    # describe / select / selected need no device
    from paper_2106_06161_gb300 import _lib as L
    for kernel in (L.BSHUFFLE_KERNEL_SINGLE_PASS, L.BSHUFFLE_KERNEL_PIPELINED, L.BSHUFFLE_KERNEL_BATCHED):
        configs = L.bshuffle_kernel_configs(kernel)
        assert len(configs) >= 2 and configs[0]["config"] == 0
        for c in configs:
            assert c["threads"] % 32 == 0 and c["items"] in (4, 8, 16) and c["rounds_unrolled"] in (0, 24)
        for w in (4, 8, 16):
            L.bshuffle_kernel_select(kernel, w, len(configs) - 1)
            assert L.bshuffle_kernel_selected(kernel, w) == len(configs) - 1
            L.bshuffle_kernel_select(kernel, w, 0)
            assert L.bshuffle_kernel_selected(kernel, w) == 0
    # the single-pass table is the one of bshuffle_tuning_*
    assert len(L.bshuffle_kernel_configs(L.BSHUFFLE_KERNEL_SINGLE_PASS)) == len(L.bshuffle_tuning_configs())
    assert lib.bshuffle_kernel_configs(9) == L.BSHUFFLE_ERR_INVALID
    assert lib.bshuffle_kernel_select(L.BSHUFFLE_KERNEL_PIPELINED, 2, 0) == L.BSHUFFLE_ERR_INVALID
    assert lib.bshuffle_kernel_select(L.BSHUFFLE_KERNEL_BATCHED, 8, 99) == L.BSHUFFLE_ERR_INVALID


def test_lookback_cycles_need_a_measurement_build(lib):
    # the default build has no cycle accounting: the reader says so
    from paper_2106_06161_gb300 import _lib as L
    a, b = ctypes.c_uint64(7), ctypes.c_uint64(7)
    assert lib.bshuffle_debug_lookback_cycles(None, ctypes.byref(a), ctypes.byref(b)) == L.BSHUFFLE_ERR_INVALID
    assert a.value == 0 and b.value == 0
    assert lib.bshuffle_debug_lookback_cycles(None, None, ctypes.byref(b)) == L.BSHUFFLE_ERR_NULL


def test_range_entry_points_check_arguments_first(lib):
    from paper_2106_06161_gb300 import _lib as L
    buf = (ctypes.c_uint64 * 64)()
    a = ctypes.addressof(buf)
    assert lib.bshuffle_count_range(100, 0, 24, 5, 4, a, None) == L.BSHUFFLE_ERR_INVALID
    assert lib.bshuffle_count_range(100, 0, 99, 0, 4, a, None) == L.BSHUFFLE_ERR_ROUNDS
    assert lib.bshuffle_count_range(100, 0, 24, 0, 4, a + 4, None) == L.BSHUFFLE_ERR_ALIGN
    assert lib.bshuffle_permute_range(a, a + 256, 16, 3, 0, 24, 0, 16, 16, None) == L.BSHUFFLE_ERR_ELEM
    assert lib.bshuffle_permute_range(a, a + 256, 16, 8, 0, 24, 9, 2, 16, None) == L.BSHUFFLE_ERR_INVALID
    assert lib.bshuffle_permute_range(a, a + 8, 16, 8, 0, 24, 0, 16, 16, None) == L.BSHUFFLE_ERR_ALIAS
    assert lib.bshuffle_permute_range(a, a + 256, 16, 8, 0, 24, 0, 16, 0, None) == L.BSHUFFLE_OK  # nothing to write
