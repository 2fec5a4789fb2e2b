"""The fused permutation Monte Carlo statistic against the FP64 oracle:
10,000 shuffles of n = 100,000 float32 samples (two groups of 50,000 from
N(0,1) and N(0.05,1)), T_b = mean(first group slots) - mean(second)."""
import multiprocessing as mp
from concurrent.futures import ProcessPoolExecutor

import numpy as np
import pytest
import torch

import oracle
import workloads

pytestmark = pytest.mark.gpu

RTOL, ATOL = 1e-12, 1e-15


@pytest.fixture(scope="module")
def bs():
    from paper_2106_06161_gb300 import build
    build.build()
    import paper_2106_06161_gb300
    paper_2106_06161_gb300.load()
    return paper_2106_06161_gb300


def _oracle_chunk(args):
    start, count = args
    x = workloads.mc_samples()
    return oracle.mc_statistics(x, workloads.MC_GROUP, start, count)


def test_small_instances_match_oracle(bs):
    for group, seed in ((8, 1), (500, 2), (3000, 3)):
        x = workloads.mc_samples(group=group, seed=seed)
        for n1 in (1, group, 2 * group - 1):
            T = bs.mc_group_diff(torch.from_numpy(x).cuda(), n1, 100, 40).cpu().numpy()
            want = oracle.mc_statistics(x, n1, 100, 40)
            np.testing.assert_allclose(T, want, rtol=RTOL, atol=ATOL)


def test_ten_thousand_shuffles_and_p_value(bs):
    x = workloads.mc_samples()
    n1, count = workloads.MC_GROUP, workloads.MC_SHUFFLES
    p, T, t_obs = bs.mc_pvalue(torch.from_numpy(x).cuda(), n1, 0, count)
    T = T.cpu().numpy()
    chunks = [(s, min(250, count - s)) for s in range(0, count, 250)]
    with ProcessPoolExecutor(max_workers=min(16, mp.cpu_count()), mp_context=mp.get_context("spawn")) as ex:
        want = np.concatenate(list(ex.map(_oracle_chunk, chunks)))
    np.testing.assert_allclose(T, want, rtol=RTOL, atol=ATOL)
    t_obs_ref = float(np.mean(x[:n1].astype(np.float64)) - np.mean(x[n1:].astype(np.float64)))
    p_ref = (1 + int(np.sum(np.abs(want) >= abs(t_obs_ref)))) / (count + 1)
    assert abs(p - p_ref) <= 1e-5 * p_ref
    for thr in (0.001, 0.005, 0.01, 0.02):
        assert int(np.sum(np.abs(T) >= thr)) == int(np.sum(np.abs(want) >= thr))
