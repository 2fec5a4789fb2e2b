"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Everything the library computes is integer index arithmetic and byte moves,
so the bar is bit-exact equality for every width, compared element by
element.  The sweep's full sizes (2^28 and 2^28 + 12345, seeds 0..4) are
compared slot by slot in test_gpu_full_size.py."""
import numpy as np
import pytest
import torch

import oracle
import workloads
from tests.gpu_helpers import assert_no_device_error, to_device, to_host

pytestmark = pytest.mark.gpu

bs = None


@pytest.fixture(scope="module", autouse=True)
def library():
    global bs
    from paper_2106_06161_gb300 import build
    build.build()
    import paper_2106_06161_gb300
    bs = paper_2106_06161_gb300
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    bs.load()
    yield


def gpu_permute(x: np.ndarray, seed: int, rounds: int = 24) -> np.ndarray:
    y = bs.permute(to_device(x), seed, rounds)
    assert_no_device_error()
    return to_host(y, x)


def gpu_inverse(x: np.ndarray, seed: int, rounds: int = 24) -> np.ndarray:
    y = bs.inverse(to_device(x), seed, rounds)
    assert_no_device_error()
    return to_host(y, x)


SMALL_N = [1, 2, 3, 5, 15, 16, 17, 31, 100, 1000, 2047, 2048, 2049, 4095, 4097, 65535, 65537, 123457]


def _payload(n: int, width: int, seed: int) -> np.ndarray:
    rng = np.random.default_rng(seed * 1000 + width)
    if width in (1, 2, 4, 8):
        dt = {1: np.uint8, 2: np.uint16, 4: np.uint32, 8: np.uint64}[width]
        return rng.integers(0, np.iinfo(dt).max, size=n, dtype=dt, endpoint=True)
    return rng.integers(0, 256, size=(n, width), dtype=np.uint8)


def test_single_shuffle_config():
    # n = 1,000,003 uint32 iota, seed 42, domain 2^20, 24 rounds
    n = workloads.SINGLE_N
    assert bs.domain_bits(n) == 20
    x = workloads.iota(n, np.uint32)
    y = gpu_permute(x, workloads.SINGLE_SEED)
    want = oracle.permute(x, workloads.SINGLE_SEED)
    assert np.array_equal(y, want)
    assert np.array_equal(np.sort(y), x)  # a permutation


@pytest.mark.parametrize("width", [1, 2, 4, 8, 16, 32, 48, 4096])
def test_permute_matches_oracle_all_widths(width):
    for n in SMALL_N:
        if width >= 48 and n > 20000:
            continue
        for seed in (0, 7):
            x = _payload(n, width, seed)
            assert np.array_equal(gpu_permute(x, seed), oracle.permute(x, seed)), (n, seed)


@pytest.mark.parametrize("rounds", [0, 1, 2, 23, 24, 64])
def test_permute_rounds(rounds):
    for n in (17, 4097, 100003):
        x = _payload(n, 8, rounds)
        assert np.array_equal(gpu_permute(x, 11, rounds), oracle.permute(x, 11, rounds))


@pytest.mark.parametrize("idx_dtype", [torch.int32, torch.int64])
def test_indices_match_oracle(idx_dtype):
    for n in SMALL_N + [2**20 + 1]:
        idx = bs.indices(n, 5, dtype=idx_dtype)
        assert_no_device_error()
        assert np.array_equal(idx.cpu().numpy().astype(np.uint64), oracle.indices(n, 5)), n


@pytest.mark.parametrize("width", [1, 4, 8, 16, 64])
def test_inverse_matches_oracle(width):
    for n in (1, 3, 17, 2049, 65537):
        x = _payload(n, width, 3)
        y = gpu_inverse(x, 9)
        assert np.array_equal(y, oracle.inverse(x, 9)), n
        assert np.array_equal(gpu_inverse(gpu_permute(x, 9), 9), x)


def test_unaligned_heads_and_views():
    # output/input starting inside a 16-byte line, and a strided source
    for width, dt in ((4, torch.int32), (8, torch.int64)):
        n = 70001
        base = torch.arange(n + 3, dtype=dt, device="cuda")
        x = base[1:n + 1]
        out = torch.empty(n + 3, dtype=dt, device="cuda")[3:]
        bs.permute(x, 123, out=out)
        assert_no_device_error()
        want = oracle.permute(np.arange(1, n + 1, dtype=np.int64).astype(np.uint64 if width == 8 else np.uint32), 123)
        assert np.array_equal(out.cpu().numpy().astype(np.uint64), want.astype(np.uint64))
    m = torch.arange(4000, dtype=torch.int64, device="cuda").reshape(1000, 4)[:, 1]  # non-contiguous
    y = bs.permute(m, 2)
    assert np.array_equal(y.cpu().numpy(), oracle.permute(m.cpu().numpy(), 2))


def test_empty_input_is_a_noop():
    x = torch.empty(0, dtype=torch.int64, device="cuda")
    assert bs.permute(x, 1).numel() == 0
    assert bs.indices(0, 1).numel() == 0
    assert_no_device_error()


@pytest.mark.parametrize("width", [4, 8, 16])
def test_sweep_sizes_up_to_2_24(width):
    for n in (2**10, 2**16, 2**20, 2**24):
        for seed in workloads.SWEEP_SEEDS:
            if n == 2**24 and seed > 1:
                continue
            x = workloads.sweep_payload(n, width, seed)
            assert np.array_equal(gpu_permute(x, seed), oracle.permute(x, seed)), (n, seed)


def test_repeated_calls_reuse_workspace():
    # The per-stream header is reset by the last CTA of every launch.
    x = _payload(300001, 4, 1)
    want = oracle.permute(x, 77)
    for _ in range(5):
        assert np.array_equal(gpu_permute(x, 77), want)
    # a bigger call grows the workspace, a smaller one reuses it
    big = _payload(2**22 + 5, 4, 2)
    assert np.array_equal(gpu_permute(big, 1), oracle.permute(big, 1))
    assert np.array_equal(gpu_permute(x, 77), want)


def test_other_stream():
    x = _payload(100000, 8, 5)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        y = bs.permute(to_device(x), 4)
        s.synchronize()
        assert bs.get_error() == 0
    assert np.array_equal(to_host(y, x), oracle.permute(x, 4))


def _scramble(i: np.ndarray, k: int) -> np.ndarray:
    """The measurement kernel's index map, restated: three rounds of
    multiply-by-odd-constant mod 2^k then xor with the value shifted by k/2."""
    mask = np.uint64((1 << k) - 1)
    half = np.uint64(k // 2)
    x = i.astype(np.uint64)
    for c in (0x9E3779B1, 0x85EBCA77, 0xC2B2AE3D):
        x = (x * np.uint64(c)) & mask
        x ^= x >> half
    return x


@pytest.mark.parametrize("width", [4, 8, 16])
def test_random_gather_measurement_kernel(width):
    for k in (4, 10, 20):
        n = 2**k
        x = _payload(n, width, k)
        xd = to_device(x)
        out = torch.empty_like(xd)
        bs.bshuffle_random_gather(xd.data_ptr(), out.data_ptr(), n, width, torch.cuda.current_stream().cuda_stream)
        torch.cuda.synchronize()
        assert np.array_equal(to_host(out, x), x[_scramble(np.arange(n), k).astype(np.int64)])


@pytest.mark.parametrize("width", [4, 8, 16])
def test_window_scatter_measurement_kernel(width):
    # out[w 2^m + h_m(i mod 2^m)] = in[i]: a permutation inside every window
    for k, m in ((4, 4), (12, 8), (20, 16), (20, 20)):
        n = 2**k
        x = _payload(n, width, k + m)
        xd = to_device(x)
        out = torch.empty_like(xd)
        bs.bshuffle_window_scatter(xd.data_ptr(), out.data_ptr(), n, width, m, torch.cuda.current_stream().cuda_stream)
        torch.cuda.synchronize()
        i = np.arange(n)
        dst = (i >> m << m) + _scramble(i & ((1 << m) - 1), m).astype(np.int64)
        want = np.empty_like(x)
        want[dst] = x
        assert np.array_equal(to_host(out, x), want), (k, m)


@pytest.mark.parametrize("width", [1, 4, 8, 16])
def test_lcg_variant_matches_oracle(width):
    for n in (1, 5, 17, 2049, 65537, 1_000_003):
        x = _payload(n, width, 4)
        y = bs.permute_lcg(to_device(x), 31)
        assert_no_device_error()
        want = x[oracle.indices_lcg(n, 31).astype(np.int64)]
        assert np.array_equal(to_host(y, x), want), n


@pytest.mark.parametrize("variant", [0, 1, 2, 3])
def test_fusion_ablation_variants_match_oracle(variant):
    # Sec. 6: Bijective0 (separate passes), Bijective1 (two-pass scan) and
    # Bijective2 (single pass) compute the same shuffle.
    stream = torch.cuda.current_stream().cuda_stream
    for width in (4, 8, 16):
        for n in (5, 2049, 65537, 1_000_003):
            x = _payload(n, width, variant)
            xd = to_device(x)
            out = torch.empty_like(xd)
            bs.bshuffle_permute_ablation(xd.data_ptr(), out.data_ptr(), n, width, 13, 24, variant, stream)
            assert_no_device_error()
            assert np.array_equal(to_host(out, x), oracle.permute(x, 13)), (width, n)


@pytest.mark.parametrize("width", [32, 64])
def test_rows_both_forms(width):
    # rows of 32 and 64 bytes: up to 4,096 tiles the two-kernel form (a count
    # kernel, then a copy kernel that sums the counts before its tile),
    # beyond it the persistent kernel with the decoupled look-back
    for n in (5_000, 300_001, 2**20 + 3):
        x = _payload(n, width, 1)
        assert np.array_equal(gpu_permute(x, 21), oracle.permute_mt(x, 21)), n
        assert np.array_equal(gpu_inverse(x, 21), oracle.inverse(x, 21)), n
