"""The allocation-free entry point bshuffle_permute_static, called through the
C ABI, against the regular bshuffle_permute.

bshuffle_permute_static serves callers that cannot allocate device memory when
they call (for instance a process that has reserved all device memory for its
own pool): its scratch is a fixed device array inside the library.  Its output
must equal bshuffle_permute's bit for bit, call after call, even though every
call reuses the same scratch.  This file is named so that pytest collects it
last."""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    from paper_2106_06161_gb300 import _lib, build
    build.build()
    return _lib.load()


def _stream() -> int:
    return torch.cuda.current_stream().cuda_stream


def _regular(lib, x: torch.Tensor, elem: int, seed: int) -> torch.Tensor:
    out = torch.empty_like(x)
    assert lib.bshuffle_permute(x.data_ptr(), out.data_ptr(), x.shape[0], elem, seed, 24, _stream()) == 0
    return out


def _static(lib, x: torch.Tensor, elem: int, seed: int) -> torch.Tensor:
    out = torch.full_like(x, -1)
    assert lib.bshuffle_permute_static(x.data_ptr(), out.data_ptr(), x.shape[0], elem, seed, 24, _stream()) == 0
    return out


def test_static_matches_regular_on_two_calls_in_a_row(lib):
    g = torch.Generator(device="cpu").manual_seed(1)
    x = torch.randint(-2**62, 2**62, (1_000_003,), dtype=torch.int64, generator=g).cuda()
    want = _regular(lib, x, 8, 42)
    first = _static(lib, x, 8, 42)
    second = _static(lib, x, 8, 42)
    torch.cuda.synchronize()
    assert torch.equal(first, want)
    assert torch.equal(second, want)


def test_static_matches_regular_across_sizes_and_widths(lib):
    rng = np.random.default_rng(2)
    for n, dt, elem, seed in ((5, torch.int32, 4, 3), (70_001, torch.int32, 4, 9),
                              (2**20 + 1, torch.int64, 8, 11), (4096, torch.int16, 2, 5)):
        x = torch.from_numpy(rng.integers(-1000, 1000, size=n)).to(dt).cuda()
        want = _regular(lib, x, elem, seed)
        for _ in range(2):
            got = _static(lib, x, elem, seed)
            torch.cuda.synchronize()
            assert torch.equal(got, want), (n, elem)


def test_static_rejects_sizes_beyond_its_scratch(lib):
    from paper_2106_06161_gb300 import _lib as L
    x = torch.empty(16, dtype=torch.int64, device="cuda")
    y = torch.empty(16, dtype=torch.int64, device="cuda")
    # n above 2^27 is refused before anything is read
    assert lib.bshuffle_permute_static(x.data_ptr(), y.data_ptr(), 2**27 + 1, 8, 0, 24, _stream()) == \
        L.BSHUFFLE_ERR_TOO_LARGE
    assert lib.bshuffle_permute_static(x.data_ptr(), y.data_ptr(), 16, 32, 0, 24, _stream()) == L.BSHUFFLE_ERR_ELEM


def test_static_at_its_size_limit_and_widest_element(lib):
    # n = 2^27 - 1 and 2^27 use every one of the array's 65,536 tile-status
    # words (domain 2^27, 2,048 indices per tile); 16-byte elements are the
    # widest the entry point takes
    g = torch.Generator(device="cpu").manual_seed(3)
    for n, dt, elem in ((2**27 - 1, torch.int32, 4), (2**27, torch.int32, 4)):
        x = torch.randint(-2**31, 2**31 - 1, (n,), dtype=dt, generator=g).cuda()
        want = _regular(lib, x, elem, 17)
        for _ in range(2):
            got = _static(lib, x, elem, 17)
            torch.cuda.synchronize()
            assert torch.equal(got, want), n
        del x, want, got
    x = torch.randint(-2**62, 2**62, (1_000_003, 2), dtype=torch.int64, generator=g).cuda()
    want = _regular(lib, x, 16, 8)
    for _ in range(2):
        got = _static(lib, x, 16, 8)
        torch.cuda.synchronize()
        assert torch.equal(got, want)
    assert lib.bshuffle_get_error(_stream()) == 0


def test_static_call_allocates_no_device_memory(lib):
    x = torch.arange(3_000_001, dtype=torch.int64, device="cuda")
    out = torch.empty_like(x)
    s = _stream()
    # the first call sets up the array's address and loads the kernel
    assert lib.bshuffle_permute_static(x.data_ptr(), out.data_ptr(), x.numel(), 8, 5, 24, s) == 0
    torch.cuda.synchronize()
    free_before, _ = torch.cuda.mem_get_info()
    for seed in (5, 6):
        assert lib.bshuffle_permute_static(x.data_ptr(), out.data_ptr(), x.numel(), 8, seed, 24, s) == 0
    torch.cuda.synchronize()
    free_after, _ = torch.cuda.mem_get_info()
    assert free_after == free_before


def test_static_device_errors_are_reported_and_cleared(lib):
    # one tile withholds its status (test hook), so the waits of the tiles
    # after it run out after 50 ms: bshuffle_get_error must report it for the
    # static entry point too, clear it, and the next call must be exact
    from paper_2106_06161_gb300 import _lib as L
    n = 10_000                       # domain 2^14: 8 tiles of 2,048 indices
    x = torch.arange(n, dtype=torch.int64, device="cuda")
    want = _regular(lib, x, 8, 3)
    s = _stream()
    assert lib.bshuffle_get_error(s) == 0
    lib.bshuffle_set_lookback_timeout_ns(50_000_000)
    lib.bshuffle_debug_skip_publish(1)
    try:
        out = torch.empty_like(x)
        assert lib.bshuffle_permute_static(x.data_ptr(), out.data_ptr(), n, 8, 3, 24, s) == 0
        code = lib.bshuffle_get_error(s)
    finally:
        lib.bshuffle_debug_skip_publish(-1)
        lib.bshuffle_set_lookback_timeout_ns(2_000_000_000)
    assert code == L.BSHUFFLE_ERR_LOOKBACK_TIMEOUT
    assert lib.bshuffle_get_error(s) == 0          # read once, then cleared
    got = _static(lib, x, 8, 3)
    assert lib.bshuffle_get_error(s) == 0
    assert torch.equal(got, want)
