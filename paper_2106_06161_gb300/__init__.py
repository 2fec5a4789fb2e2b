"""GB300-native bijective shuffle (Mitchell et al., arXiv 2106.06161).

Tensor-level entry points over the C ABI of ``libbshuffle.so``
(``include/bshuffle.h``).  PyTorch supplies device memory and the current
CUDA stream; every step of the shuffle runs in the library's CUDA kernels.
Tensors are shuffled along dim 0: element j of the output is row f(i_j) of
the input, where f is the VariablePhilox bijection (Sec. 3.2) on the padded
power-of-two domain and i_j the j-th domain index whose image is kept
(Algorithm 1, Sec. 4).

    import paper_2106_06161_gb300 as bs
    y = bs.permute(x, seed=42)          # x: CUDA tensor, any dtype
    x2 = bs.inverse(y, seed=42)         # x2 == x
    idx = bs.indices(len(x), seed=42)   # y == x[idx]
"""
from __future__ import annotations

import numpy as np
import torch

from ._lib import (
    DEFAULT_ROUNDS,
    MAX_N,
    MAX_ROUNDS,
    BShuffleError,
    bshuffle_batched,
    bshuffle_count_range,
    bshuffle_cuda_error_name,
    bshuffle_debug_skip_publish,
    bshuffle_last_cuda_error,
    bshuffle_permute_range,
    bshuffle_domain_bits,
    bshuffle_get_error,
    bshuffle_indices,
    bshuffle_inverse,
    bshuffle_mc_group_diff,
    bshuffle_permute,
    bshuffle_shapley_voting,
    bshuffle_random_gather,
    bshuffle_window_scatter,
    bshuffle_release_workspaces,
    bshuffle_round_keys,
    bshuffle_set_lookback_timeout_ns,
    bshuffle_set_strategy,
    bshuffle_get_strategy,
    bshuffle_set_pass_timing,
    bshuffle_last_pass_ms,
    bshuffle_tuning_configs,
    bshuffle_permute_lcg,
    bshuffle_permute_ablation,
    bshuffle_lcg_params,
    bshuffle_tuning_select,
    bshuffle_tuning_selected,
    BSHUFFLE_STRATEGY_AUTO,
    BSHUFFLE_STRATEGY_SINGLE_PASS,
    BSHUFFLE_STRATEGY_STAGED,
    BSHUFFLE_STRATEGY_PIPELINED,
    bshuffle_version,
    error_string,
    load,
)

__all__ = [
    "DEFAULT_ROUNDS", "MAX_N", "MAX_ROUNDS", "BShuffleError", "permute", "inverse", "indices",
    "batched", "batched_packed", "packed_descs", "get_error", "domain_bits", "round_keys", "row_bytes",
    "bshuffle_permute", "bshuffle_indices", "bshuffle_inverse", "bshuffle_batched",
    "bshuffle_get_error", "bshuffle_domain_bits", "bshuffle_round_keys",
    "bshuffle_release_workspaces", "bshuffle_set_lookback_timeout_ns", "bshuffle_set_strategy",
    "bshuffle_get_strategy", "bshuffle_set_pass_timing", "bshuffle_last_pass_ms",
    "bshuffle_tuning_configs", "bshuffle_tuning_select", "bshuffle_tuning_selected",
    "bshuffle_permute_lcg", "bshuffle_lcg_params", "permute_lcg", "bshuffle_permute_ablation", "BSHUFFLE_STRATEGY_AUTO", "BSHUFFLE_STRATEGY_SINGLE_PASS",
    "BSHUFFLE_STRATEGY_STAGED", "BSHUFFLE_STRATEGY_PIPELINED",
    "bshuffle_debug_skip_publish", "bshuffle_version", "error_string", "load",
    "bshuffle_mc_group_diff", "bshuffle_random_gather", "mc_group_diff", "mc_pvalue", "BShuffleRows", "shuffle_rows",
    "bshuffle_shapley_voting", "shapley_voting", "bshuffle_window_scatter",
    "bshuffle_count_range", "bshuffle_permute_range", "bshuffle_last_cuda_error", "bshuffle_cuda_error_name",
]


def _stream_of(t: torch.Tensor) -> int:
    return torch.cuda.current_stream(t.device).cuda_stream


def _require_cuda(t: torch.Tensor, what: str) -> None:
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise ValueError(f"{what} must be a CUDA tensor (there is no CPU path)")
    if t.dim() == 0:
        raise ValueError(f"{what} must have at least one dimension")


def row_bytes(t: torch.Tensor) -> int:
    """Bytes of one element along dim 0 (a scalar or a whole row)."""
    per = 1
    for s in t.shape[1:]:
        per *= s
    return per * t.element_size()


def _out_like(x: torch.Tensor, out: torch.Tensor | None) -> torch.Tensor:
    if out is None:
        return torch.empty_like(x, memory_format=torch.contiguous_format)
    if out.shape != x.shape or out.dtype != x.dtype or out.device != x.device or not out.is_contiguous():
        raise ValueError("out must be a contiguous tensor with the input's shape, dtype and device")
    return out


def _along(fn, x: torch.Tensor, seed: int, rounds: int, out, dim: int) -> torch.Tensor:
    """Apply a dim-0 call along `dim`: the dimension is moved to the front (a
    copy), its slices are shuffled as rows, and it is moved back (a copy)."""
    d = dim % x.dim() if x.dim() else 0
    if d == 0:
        return fn(x, seed, rounds, out)
    y = fn(x.movedim(d, 0).contiguous(), seed, rounds, None).movedim(0, d)
    if out is None:
        return y.contiguous()
    if out.shape != x.shape or out.dtype != x.dtype or out.device != x.device:
        raise ValueError("out must have the input's shape, dtype and device")
    return out.copy_(y)


def _permute0(x: torch.Tensor, seed: int, rounds: int, out) -> torch.Tensor:
    _require_cuda(x, "x")
    x = x.contiguous()
    out = _out_like(x, out)
    bshuffle_permute(x.data_ptr(), out.data_ptr(), x.shape[0], row_bytes(x), seed, rounds, _stream_of(x))
    return out


def permute(x: torch.Tensor, seed: int, rounds: int = DEFAULT_ROUNDS,
            out: torch.Tensor | None = None, dim: int = 0) -> torch.Tensor:
    """Shuffle x along `dim` (default 0): out[j] = x[f(i_j)] (Algorithm 1),
    j and i_j indexing that dimension.  The slices along `dim` are the
    elements shuffled: 1, 2, 4 or 8 bytes, or a multiple of 16 bytes."""
    _require_cuda(x, "x")
    return _along(_permute0, x, seed, rounds, out, dim)


def _inverse0(y: torch.Tensor, seed: int, rounds: int, out) -> torch.Tensor:
    _require_cuda(y, "y")
    y = y.contiguous()
    out = _out_like(y, out)
    bshuffle_inverse(y.data_ptr(), out.data_ptr(), y.shape[0], row_bytes(y), seed, rounds, _stream_of(y))
    return out


def inverse(y: torch.Tensor, seed: int, rounds: int = DEFAULT_ROUNDS,
            out: torch.Tensor | None = None, dim: int = 0) -> torch.Tensor:
    """Undo :func:`permute` along `dim`: out[f(i_j)] = y[j]."""
    _require_cuda(y, "y")
    return _along(_inverse0, y, seed, rounds, out, dim)


def indices(n: int, seed: int, rounds: int = DEFAULT_ROUNDS, dtype: torch.dtype = torch.int64,
            device: torch.device | str | None = None) -> torch.Tensor:
    """Source index of every output slot: permute(x) == x[indices(len(x))]."""
    if dtype not in (torch.int64, torch.int32):
        raise ValueError("indices are int64 or int32")
    dev = torch.device("cuda", torch.cuda.current_device()) if device is None else torch.device(device)
    out = torch.empty(n, dtype=dtype, device=dev)
    if dtype == torch.int32 and n > 2**31:
        raise ValueError("int32 indices cannot hold lengths above 2^31")
    bshuffle_indices(out.data_ptr(), out.element_size(), n, seed, rounds, _stream_of(out))
    return out


def _descs(in_ptrs, out_ptrs, sizes, seeds, device) -> torch.Tensor:
    """Device array of bshuffle_desc {in, out, n, seed} as int64 words."""
    host = np.empty((len(sizes), 4), dtype=np.uint64)
    host[:, 0] = np.asarray(in_ptrs, dtype=np.uint64)
    host[:, 1] = np.asarray(out_ptrs, dtype=np.uint64)
    host[:, 2] = np.asarray(sizes, dtype=np.uint64)
    host[:, 3] = np.asarray([s & (2**64 - 1) for s in seeds], dtype=np.uint64)
    return torch.from_numpy(host.view(np.int64)).to(device, non_blocking=False)


def batched(inputs: list[torch.Tensor], seeds, rounds: int = DEFAULT_ROUNDS,
            outs: list[torch.Tensor] | None = None) -> list[torch.Tensor]:
    """Independent shuffles of several tensors in one launch.

    inputs[t] is shuffled along dim 0 with seeds[t]; the result equals
    permute(inputs[t], seeds[t], rounds).  All inputs share dtype, row width
    and device.
    """
    if len(inputs) == 0:
        return []
    for t in inputs:
        _require_cuda(t, "inputs")
    inputs = [t.contiguous() for t in inputs]
    eb = row_bytes(inputs[0])
    if any(row_bytes(t) != eb or t.dtype != inputs[0].dtype or t.device != inputs[0].device for t in inputs):
        raise ValueError("batched inputs must share dtype, row width and device")
    if outs is None:
        outs = [torch.empty_like(t) for t in inputs]
    seeds = list(seeds)
    if len(seeds) != len(inputs) or len(outs) != len(inputs):
        raise ValueError("one seed and one output per input")
    d = _descs([t.data_ptr() for t in inputs], [o.data_ptr() for o in outs],
               [t.shape[0] for t in inputs], seeds, inputs[0].device)
    bshuffle_batched(d.data_ptr(), len(inputs), eb, rounds, _stream_of(inputs[0]))
    return outs


def packed_descs(data: torch.Tensor, out: torch.Tensor, sizes, seeds) -> torch.Tensor:
    """Device descriptors for segments of `data` shuffled into the same rows of `out`.

    Segment t covers rows offsets[t] .. offsets[t] + sizes[t].  The result can
    be passed to :func:`bshuffle_batched` repeatedly, e.g. inside a captured
    CUDA graph.
    """
    _require_cuda(data, "data")
    if not data.is_contiguous() or not out.is_contiguous() or out.shape != data.shape:
        raise ValueError("data and out must be contiguous tensors of one shape")
    sizes = np.asarray(sizes, dtype=np.int64)
    if sizes.sum() != data.shape[0]:
        raise ValueError("sizes must add up to len(data)")
    eb = row_bytes(data)
    offsets = np.concatenate([[0], np.cumsum(sizes)[:-1]]).astype(np.uint64) * np.uint64(eb)
    return _descs(np.uint64(data.data_ptr()) + offsets, np.uint64(out.data_ptr()) + offsets, sizes,
                  list(seeds), data.device)


def batched_packed(data: torch.Tensor, sizes, seeds, rounds: int = DEFAULT_ROUNDS,
                   out: torch.Tensor | None = None) -> torch.Tensor:
    """Shuffle consecutive segments of data (lengths `sizes`) independently.

    Segment t covers rows offsets[t] .. offsets[t] + sizes[t] of data and is
    shuffled with seeds[t]; one launch for all segments.
    """
    _require_cuda(data, "data")
    data = data.contiguous()
    out = _out_like(data, out)
    d = packed_descs(data, out, sizes, seeds)
    bshuffle_batched(d.data_ptr(), len(d), row_bytes(data), rounds, _stream_of(data))
    return out


def get_error(device=None) -> int:
    """Synchronise the current stream and return its recorded device error (0 = none)."""
    dev = torch.device("cuda", torch.cuda.current_device()) if device is None else torch.device(device)
    return bshuffle_get_error(torch.cuda.current_stream(dev).cuda_stream)


def domain_bits(n: int) -> int:
    return bshuffle_domain_bits(n)


def round_keys(seed: int, rounds: int = DEFAULT_ROUNDS) -> list[int]:
    return bshuffle_round_keys(seed, rounds)


def mc_group_diff(x: torch.Tensor, n1: int, base_seed: int, count: int,
                  rounds: int = DEFAULT_ROUNDS) -> torch.Tensor:
    """T[b] = mean(y[:n1]) - mean(y[n1:]) for y = permute(x, base_seed + b), FP64.

    One fused launch; the shuffled values are never written to memory.
    """
    _require_cuda(x, "x")
    if x.dtype != torch.float32 or x.dim() != 1:
        raise ValueError("x must be a 1-D float32 CUDA tensor")
    x = x.contiguous()
    T = torch.empty(count, dtype=torch.float64, device=x.device)
    bshuffle_mc_group_diff(x.data_ptr(), x.numel(), n1, base_seed, count, rounds, T.data_ptr(), _stream_of(x))
    return T


def mc_pvalue(x: torch.Tensor, n1: int, base_seed: int, count: int, rounds: int = DEFAULT_ROUNDS):
    """Two-sided permutation-test p-value of the group-mean difference.

    p = (1 + #{b : |T_b| >= |T_obs|}) / (count + 1), with T_obs the statistic of
    the unshuffled sample.  Returns (p, T, T_obs).
    """
    T = mc_group_diff(x, n1, base_seed, count, rounds)
    xd = x.double()
    t_obs = float(xd[:n1].mean() - xd[n1:].mean())
    exceed = int((T.abs() >= abs(t_obs)).sum())
    return (1 + exceed) / (count + 1), T, t_obs


def shapley_voting(weights: torch.Tensor, quota: int, seed0: int, samples: int,
                   rounds: int = DEFAULT_ROUNDS) -> torch.Tensor:
    """Pivot counts of the weighted voting game [quota; weights] over `samples`
    player orders (order s = the shuffle with seed seed0 + s), as int64.

    counts / samples estimates the Shapley values.  `weights` is a 1-D CUDA
    tensor of non-negative int32 (or uint32) weights.  One fused launch.
    """
    _require_cuda(weights, "weights")
    if weights.dim() != 1 or weights.dtype not in (torch.int32, getattr(torch, "uint32", torch.int32)):
        raise ValueError("weights must be a 1-D int32 or uint32 CUDA tensor")
    weights = weights.contiguous()
    counts = torch.empty(weights.numel(), dtype=torch.int64, device=weights.device)
    bshuffle_shapley_voting(weights.data_ptr(), weights.numel(), quota, seed0, samples, rounds, counts.data_ptr(),
                            _stream_of(weights))
    return counts


from .autograd import BShuffleRows, shuffle_rows  # noqa: E402


def permute_lcg(x: torch.Tensor, seed: int, out: torch.Tensor | None = None) -> torch.Tensor:
    """Shuffle x along dim 0 with the LCG bijection of Sec. 3.1 (fast, weak)."""
    _require_cuda(x, "x")
    x = x.contiguous()
    out = _out_like(x, out)
    bshuffle_permute_lcg(x.data_ptr(), out.data_ptr(), x.shape[0], row_bytes(x), seed, _stream_of(x))
    return out
