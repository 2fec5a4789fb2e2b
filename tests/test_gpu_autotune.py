"""Every configuration of the tunable kernels (the plain single pass, the
pipelined single pass and the persistent batched kernel) computes the same
shuffle, checked against the oracle, and the autotuner selects, caches and
re-applies a configuration per kernel and element width."""
import json

import numpy as np
import pytest
import torch

import oracle
import workloads
from tests.gpu_helpers import assert_no_device_error, to_device, to_host

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def bs():
    from paper_2106_06161_gb300 import build
    build.build()
    import paper_2106_06161_gb300
    paper_2106_06161_gb300.load()
    yield paper_2106_06161_gb300
    from paper_2106_06161_gb300 import autotune
    autotune.reset()
    paper_2106_06161_gb300.bshuffle_set_strategy(paper_2106_06161_gb300.BSHUFFLE_STRATEGY_AUTO)


def test_every_configuration_is_exact(bs):
    configs = bs.bshuffle_tuning_configs()
    assert configs[0]["config"] == 0 and len(configs) >= 2
    bs.bshuffle_set_strategy(bs.BSHUFFLE_STRATEGY_SINGLE_PASS)
    try:
        for width in (4, 8, 16):
            for n in (5, 2049, 65537, 1_000_003):
                x = workloads.sweep_payload(n, width, 2)
                want = oracle.permute(x, 6)
                want23 = oracle.permute(x, 6, 23)
                for c in configs:
                    bs.bshuffle_tuning_select(width, c["config"])
                    assert bs.bshuffle_tuning_selected(width) == c["config"]
                    got = to_host(bs.permute(to_device(x), 6), x)
                    assert np.array_equal(got, want), (width, n, c)
                    # a fixed-rounds configuration falls back for other round counts
                    got23 = to_host(bs.permute(to_device(x), 6, 23), x)
                    assert np.array_equal(got23, want23), (width, n, c)
                assert_no_device_error()
    finally:
        for w in (4, 8, 16):
            bs.bshuffle_tuning_select(w, 0)
        bs.bshuffle_set_strategy(bs.BSHUFFLE_STRATEGY_AUTO)
    with pytest.raises(bs.BShuffleError):
        bs.bshuffle_tuning_select(2, 1)
    with pytest.raises(bs.BShuffleError):
        bs.bshuffle_tuning_select(8, len(configs))


def test_every_pipelined_configuration_is_exact(bs):
    from paper_2106_06161_gb300 import _lib as L
    configs = L.bshuffle_kernel_configs(L.BSHUFFLE_KERNEL_PIPELINED)
    assert len(configs) >= 2 and configs[0]["ctas_per_sm"] > 0
    assert {c["rounds_unrolled"] for c in configs} == {0, 24}
    bs.bshuffle_set_strategy(bs.BSHUFFLE_STRATEGY_PIPELINED)
    try:
        for width in (4, 8, 16):
            for n in (5, 65537, 300_007, 2**20 + 1):
                x = workloads.sweep_payload(n, width, 3)
                want = {r: oracle.permute(x, 8, r) for r in (24, 23)}
                for c in configs:
                    L.bshuffle_kernel_select(L.BSHUFFLE_KERNEL_PIPELINED, width, c["config"])
                    assert L.bshuffle_kernel_selected(L.BSHUFFLE_KERNEL_PIPELINED, width) == c["config"]
                    for r in (24, 23):
                        got = to_host(bs.permute(to_device(x), 8, r), x)
                        assert np.array_equal(got, want[r]), (width, n, c, r)
                assert_no_device_error()
            # the index output and the scatter keep the default shape
            idx = bs.indices(300_007, 8, dtype=torch.int64)
            assert np.array_equal(idx.cpu().numpy().view(np.uint64), oracle.indices(300_007, 8))
    finally:
        from paper_2106_06161_gb300 import autotune
        autotune.reset()
        bs.bshuffle_set_strategy(bs.BSHUFFLE_STRATEGY_AUTO)


def test_every_batched_configuration_is_exact(bs):
    from paper_2106_06161_gb300 import _lib as L
    from paper_2106_06161_gb300 import autotune
    configs = L.bshuffle_kernel_configs(L.BSHUFFLE_KERNEL_BATCHED)
    assert len(configs) >= 2
    sizes = np.concatenate([[1, 17, 2048, 2049, 0, 4097], autotune.uneven_sizes(40, 100, 300_000, seed=5)])
    seeds = list(range(100, 100 + len(sizes)))
    try:
        for width in (4, 8, 16):
            host = workloads.sweep_payload(int(sizes.sum()), width, 4)
            data = to_device(host)
            want = np.empty_like(host)
            off = 0
            for m, sd in zip(sizes, seeds):
                want[off:off + m] = oracle.permute(host[off:off + m], sd)
                off += m
            for c in configs:
                L.bshuffle_kernel_select(L.BSHUFFLE_KERNEL_BATCHED, width, c["config"])
                out = torch.empty_like(data)
                descs = bs.packed_descs(data, out, sizes, seeds)
                bs.bshuffle_batched(descs.data_ptr(), len(sizes), width, 24, torch.cuda.current_stream().cuda_stream)
                assert_no_device_error()
                assert np.array_equal(to_host(out, host), want), (width, c)
    finally:
        autotune.reset()
    with pytest.raises(bs.BShuffleError):
        L.bshuffle_kernel_select(L.BSHUFFLE_KERNEL_BATCHED, 2, 1)
    with pytest.raises(bs.BShuffleError):
        L.bshuffle_kernel_select(L.BSHUFFLE_KERNEL_PIPELINED, 8, len(configs) + 5)
    with pytest.raises(bs.BShuffleError):
        L.bshuffle_kernel_select(7, 8, 0)


def test_autotune_caches_and_reapplies(bs, tmp_path):
    from paper_2106_06161_gb300 import _lib as L
    from paper_2106_06161_gb300 import autotune
    cache = str(tmp_path / "tuning.json")
    res = autotune.tune(widths=(4, 8), reps=2, warmup=1, cache=cache, plain_n=2**12 + 1, pipe_n=2**20 + 1,
                        batch_count=64)
    data = json.load(open(cache))
    entry = data[autotune.device_key()]
    for kernel, kid in autotune.KERNELS.items():
        for w in ("4", "8"):
            assert entry[kernel][w]["config"] == res[kernel][w]["config"]
            assert L.bshuffle_kernel_selected(kid, int(w)) == res[kernel][w]["config"]
            assert len(res[kernel][w]["ms"]) >= 2
    autotune.reset()
    assert autotune.apply_cached(cache)
    for kernel, kid in autotune.KERNELS.items():
        for w in ("4", "8"):
            assert L.bshuffle_kernel_selected(kid, int(w)) == res[kernel][w]["config"]
    autotune.reset()
    assert bs.bshuffle_get_strategy() == bs.BSHUFFLE_STRATEGY_AUTO
