"""Statistical tests for distributions of permutations (Sec. 5 of arXiv 2106.06161).

TEST INFRASTRUCTURE ONLY: used by the test-suite to check that the oracle's
shuffles are uniform, the way Sec. 5 checks VariablePhilox.  All arithmetic is
FP64.

Conventions.  A sample is a (count, n) array of permutations.  The paper's
permutation sigma assigns rank sigma(i) = j to element i (Sec. 2).  A shuffle
output idx (slot j holds element idx[j]) is converted with
:func:`ranks_from_indices`, i.e. sigma = idx^-1.
"""
from __future__ import annotations

import math

import numpy as np
from scipy import special, stats

from . import kendall_pairs

LAMBDA = 5.0   # Mallows kernel parameter used throughout Sec. 5
ALPHA = 0.05   # significance level of the chi-squared test in Sec. 5


def ranks_from_indices(idx: np.ndarray) -> np.ndarray:
    """sigma = idx^-1 row by row: sigma[idx[j]] = j."""
    idx = np.asarray(idx)
    count, n = idx.shape
    sigma = np.empty_like(idx)
    rows = np.arange(count)[:, None]
    sigma[rows, idx.astype(np.int64)] = np.arange(n, dtype=idx.dtype)[None, :]
    return sigma


def lehmer_rank(perms: np.ndarray) -> np.ndarray:
    """Index in [0, n!) of each permutation (Lehmer code, lexicographic order)."""
    perms = np.asarray(perms, dtype=np.int64)
    count, n = perms.shape
    rank = np.zeros(count, dtype=np.int64)
    for pos in range(n):
        smaller_after = (perms[:, pos + 1:] < perms[:, pos:pos + 1]).sum(axis=1)
        rank = rank * (n - pos) + smaller_after
    return rank


def chi2_uniform(perms: np.ndarray, alpha: float = ALPHA):
    """Chi-squared statistic of the permutation frequencies against 1/n!.

    Returns (statistic, degrees of freedom, critical value at level alpha).
    Sec. 5 uses n = 5 (119 degrees of freedom) and 100,000 permutations.
    """
    count, n = perms.shape
    cells = math.factorial(n)
    observed = np.bincount(lehmer_rank(perms), minlength=cells).astype(np.float64)
    expected = count / cells
    chi2 = float(((observed - expected) ** 2 / expected).sum())
    dof = cells - 1
    return chi2, dof, float(stats.chi2.ppf(1.0 - alpha, dof))


def _pairs(n: int) -> float:
    return n * (n - 1) / 2.0


def _kernel_mean(n: int, lam: float) -> float:
    """prod_{j=1..n} (1 - e^{-lam j / C(n,2)}) / (j (1 - e^{-lam / C(n,2)})), in logs."""
    c = _pairs(n)
    log_den = math.log(-math.expm1(-lam / c))
    total = 0.0
    for j in range(1, n + 1):
        total += math.log(-math.expm1(-lam * j / c)) - math.log(j) - log_den
    return math.exp(total)


def mallows_expectation(n: int, lam: float = LAMBDA) -> float:
    """E_{sigma'}[K(sigma, sigma')] under the uniform distribution (Sec. 5)."""
    return _kernel_mean(n, lam)


def mallows_variance(n: int, lam: float = LAMBDA) -> float:
    """Var(K(sigma, sigma')) = E[K^2] - E[K]^2, where K^2 is the kernel at 2 lam."""
    return _kernel_mean(n, 2.0 * lam) - _kernel_mean(n, lam) ** 2


def mallows_kernel_values(perms: np.ndarray, lam: float = LAMBDA) -> np.ndarray:
    """K(Pi_{2i-1}, Pi_{2i}) for the consecutive pairs of the sample."""
    n = perms.shape[1]
    ndis = kendall_pairs(perms).astype(np.float64)
    return np.exp(-lam * ndis / _pairs(n))


def mmd2_estimate(perms: np.ndarray, lam: float = LAMBDA) -> float:
    """Unbiased one-sample MMD^2 estimate of Sec. 5 for an even-sized sample."""
    count, n = perms.shape
    if count % 2:
        raise ValueError("the estimate pairs permutations; use an even sample size")
    k = mallows_kernel_values(perms, lam)
    return float(2.0 / count * k.sum() - mallows_expectation(n, lam))


def hoeffding_threshold(count: int, alpha: float = ALPHA) -> float:
    """Acceptance bound sqrt(log(2/alpha)/|Pi|) from Hoeffding's inequality."""
    return math.sqrt(math.log(2.0 / alpha) / count)


def clt_threshold(n: int, count: int, alpha: float = ALPHA, lam: float = LAMBDA) -> float:
    """Asymptotic acceptance bound sqrt(2 Var(MMD^2)) erf^-1(1 - alpha)."""
    var_mmd = 2.0 * mallows_variance(n, lam) / count
    return math.sqrt(2.0 * var_mmd) * float(special.erfinv(1.0 - alpha))
