"""Exact Shapley values of weighted voting games, the reference values for the
permutation-sampling estimate of Shapley values (an application named in
Sec. 1 of arXiv 2106.06161).

TEST INFRASTRUCTURE ONLY: used by the test-suite and the benchmark's CPU legs.

Game [q; w_0, ..., w_{n-1}]: a coalition S wins when its total weight
w(S) >= q.  Player i's Shapley value is the share of the n! player orders in
which i is pivotal (the players before i weigh less than q and adding w_i
reaches q); summed over the coalitions S of the other players that i turns
from losing to winning, q - w_i <= w(S) < q, each with weight
|S|! (n - 1 - |S|)! / n!.  The coalitions are counted by size and weight with
a dynamic programme over the players, in exact rational arithmetic.
"""
from __future__ import annotations

from fractions import Fraction
from math import factorial


def shapley_shubik(weights, quota: int) -> list[Fraction]:
    """Exact Shapley values of [quota; weights] (non-negative integers)."""
    w = [int(x) for x in weights]
    n = len(w)
    if any(x < 0 for x in w):
        raise ValueError("weights must be non-negative")
    if n == 0:
        return []
    if quota <= 0 or quota > sum(w):
        return [Fraction(0)] * n
    phi = []
    for i in range(n):
        # count[s][t]: coalitions of the other players with s members and
        # weight t, for t < quota (heavier coalitions already win without i)
        count = [[0] * quota for _ in range(n)]
        count[0][0] = 1
        members = 0
        for j in range(n):
            if j == i:
                continue
            for s in range(members, -1, -1):
                row, up = count[s], count[s + 1]
                for t in range(quota - 1 - w[j], -1, -1):
                    if row[t]:
                        up[t + w[j]] += row[t]
            members += 1
        lo = max(quota - w[i], 0)
        value = Fraction(0)
        for s in range(n):
            c = sum(count[s][lo:quota])
            if c:
                value += Fraction(c * factorial(s) * factorial(n - 1 - s), factorial(n))
        phi.append(value)
    return phi
