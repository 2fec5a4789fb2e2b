"""Differentiable row shuffle.

Forward: the fused row gather of :func:`permute` (out[j] = x[f(i_j)]).
Backward: the row scatter of :func:`inverse` (grad_x[f(i_j)] = grad_out[j]),
which regenerates the (source, slot) pairs from (n, seed, rounds) instead of
saving an index tensor.  Each input row receives exactly one output row's
gradient, so the backward is exact in every dtype.
"""
from __future__ import annotations

import torch


class BShuffleRows(torch.autograd.Function):
    """y = x[indices(len(x), seed, rounds)] with a scatter backward."""

    @staticmethod
    def forward(ctx, x: torch.Tensor, seed: int, rounds: int):
        from . import permute
        ctx.seed = seed
        ctx.rounds = rounds
        return permute(x, seed, rounds)

    @staticmethod
    def backward(ctx, grad_out: torch.Tensor):
        from . import inverse
        return inverse(grad_out.contiguous(), ctx.seed, ctx.rounds), None, None


def shuffle_rows(x: torch.Tensor, seed: int, rounds: int = 24) -> torch.Tensor:
    """Shuffle the rows (dim 0) of x; differentiable."""
    return BShuffleRows.apply(x, seed, rounds)
