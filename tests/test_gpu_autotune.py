"""Every configuration of the tunable single-pass kernel computes the same
shuffle (checked against the oracle), and the autotuner selects, caches and
re-applies a configuration per element width."""
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
    for w in (4, 8, 16):
        paper_2106_06161_gb300.bshuffle_tuning_select(w, 0)
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


def test_autotune_caches_and_reapplies(bs, tmp_path):
    from paper_2106_06161_gb300 import autotune
    cache = str(tmp_path / "tuning.json")
    res = autotune.tune(widths=(4, 8), n=2**20 + 1, reps=2, warmup=1, cache=cache)
    data = json.load(open(cache))
    entry = data[autotune.device_key()]
    for w in ("4", "8"):
        assert entry[w]["config"] == res[w]["config"]
        assert bs.bshuffle_tuning_selected(int(w)) == res[w]["config"]
    for w in (4, 8):
        bs.bshuffle_tuning_select(w, 0)
    assert autotune.apply_cached(cache)
    for w in ("4", "8"):
        assert bs.bshuffle_tuning_selected(int(w)) == res[w]["config"]
    assert bs.bshuffle_get_strategy() == bs.BSHUFFLE_STRATEGY_AUTO
