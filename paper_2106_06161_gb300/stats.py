"""The statistical tests of Sec. 5 on the GPU: permutations sampled with the
library's batched shuffle, the Mallows-kernel MMD^2 estimate from Kendall
discordant-pair counts computed in a CUDA kernel, and the two acceptance
thresholds (Hoeffding and central-limit) from the closed forms of Sec. 5.

    import paper_2106_06161_gb300.stats as st
    r = st.mmd_test(n=1000, count=100_000, rounds=24)   # r["passes_clt"]
"""
from __future__ import annotations

import math

import numpy as np
import torch

from . import _lib

LAMBDA = 5.0   # the Mallows kernel parameter used throughout Sec. 5
ALPHA = 0.05


def sample_ranks(n: int, count: int, seed0: int = 0, rounds: int = 24) -> torch.Tensor:
    """count permutations of [0, n) as ranks sigma (Sec. 2), seeds seed0, seed0+1, ...

    One batched launch shuffles `count` copies of 0..n-1 (slot order), then
    each row is inverted into ranks.  Returns a (count, n) int32 CUDA tensor.
    """
    from . import batched_packed
    dev = torch.device("cuda", torch.cuda.current_device())
    iota = torch.arange(n, dtype=torch.int32, device=dev).repeat(count)
    idx = batched_packed(iota, np.full(count, n), [seed0 + t for t in range(count)], rounds)
    sigma = torch.empty_like(idx)
    _lib.bshuffle_invert_rows(idx.data_ptr(), n, count, sigma.data_ptr(), torch.cuda.current_stream().cuda_stream)
    return sigma.view(count, n)


def kendall_pairs(ranks: torch.Tensor) -> torch.Tensor:
    """n_dis of the consecutive pairs (0,1), (2,3), ... of a (count, n) int32 tensor."""
    ranks = ranks.contiguous()
    count, n = ranks.shape
    out = torch.empty(count // 2, dtype=torch.int64, device=ranks.device)
    _lib.bshuffle_kendall_pairs(ranks.data_ptr(), n, count // 2, out.data_ptr(), torch.cuda.current_stream().cuda_stream)
    return out


def _kernel_mean(n: int, lam: float) -> float:
    c = n * (n - 1) / 2.0
    log_den = math.log(-math.expm1(-lam / c))
    return math.exp(math.fsum(math.log(-math.expm1(-lam * j / c)) - math.log(j) - log_den for j in range(1, n + 1)))


def mallows_expectation(n: int, lam: float = LAMBDA) -> float:
    """E[K(sigma, sigma')] for uniform sigma' (the product formula of Sec. 5)."""
    return _kernel_mean(n, lam)


def mallows_variance(n: int, lam: float = LAMBDA) -> float:
    """Var(K) = E[K^2] - E[K]^2, with K^2 the kernel at 2 lambda."""
    return _kernel_mean(n, 2.0 * lam) - _kernel_mean(n, lam) ** 2


def mmd2_estimate(ranks: torch.Tensor, lam: float = LAMBDA) -> float:
    """(2/|Pi|) sum_i K(Pi_{2i-1}, Pi_{2i}) - E[K]: the unbiased estimate of Sec. 5."""
    count, n = ranks.shape
    if count % 2:
        raise ValueError("the estimate pairs permutations; use an even sample size")
    ndis = kendall_pairs(ranks).to(torch.float64)
    k = torch.exp(-lam * ndis / (n * (n - 1) / 2.0))
    return float(2.0 / count * k.sum().item() - mallows_expectation(n, lam))


def hoeffding_threshold(count: int, alpha: float = ALPHA) -> float:
    return math.sqrt(math.log(2.0 / alpha) / count)


def clt_threshold(n: int, count: int, alpha: float = ALPHA, lam: float = LAMBDA) -> float:
    from scipy import special
    return math.sqrt(2.0 * (2.0 * mallows_variance(n, lam) / count)) * float(special.erfinv(1.0 - alpha))


def mmd_test(n: int, count: int = 100_000, rounds: int = 24, seed0: int = 0, lam: float = LAMBDA,
             alpha: float = ALPHA) -> dict:
    """MMD^2 of `count` shuffles of length n and both acceptance thresholds."""
    ranks = sample_ranks(n, count, seed0, rounds)
    mmd = mmd2_estimate(ranks, lam)
    clt = clt_threshold(n, count, alpha, lam)
    hoeff = hoeffding_threshold(count, alpha)
    return {"n": n, "count": count, "rounds": rounds, "mmd2": mmd, "clt_threshold": clt,
            "hoeffding_threshold": hoeff, "passes_clt": abs(mmd) < clt, "passes_hoeffding": abs(mmd) < hoeff}
