"""One shuffle split across ranks by domain range (one exchange of counts).

Algorithm 1 (Sec. 4) has a single dependency between domain indices: the
exclusive scan of the keep flags.  With the domain [0, 2^k) cut into
`parts` consecutive ranges, part r's kept indices fill the output slots
[offset_r, offset_r + count_r), where offset_r is the sum of the counts of
the ranges before it.  Each rank therefore

  1. counts the kept indices of its range on its GPU (bshuffle_count_range:
     the cipher and the keep test, no data read),
  2. all-gathers the counts (one int64 per rank) and takes its offset
     (exclusive sum in rank order), and
  3. gathers its range's kept elements from the whole input, which every rank
     holds (bshuffle_permute_range), into its part of the output.

For n = 2^k (k >= 4) no domain index is dropped: a range's count is its
length and its offset is its first index, so the ranks need no exchange at
all, and each gathers its range with the scan-free kernel.

Every step of the shuffle runs in the library's kernels; this module only
plans the ranges and moves the counts between ranks.
"""
from __future__ import annotations

import torch

from . import _lib


def ranges(n: int, parts: int) -> list[tuple[int, int]]:
    """Consecutive domain ranges [first, end) covering [0, 2^k) of length n,
    as equal as possible (the first `2^k mod parts` ranges one longer)."""
    if parts < 1:
        raise ValueError("parts must be at least 1")
    domain = 1 << _lib.bshuffle_domain_bits(n) if n else 0
    q, rem = divmod(domain, parts)
    out, first = [], 0
    for r in range(parts):
        end = first + q + (1 if r < rem else 0)
        out.append((first, end))
        first = end
    return out


def offsets(counts: list[int]) -> tuple[list[int], int]:
    """Exclusive sums of the per-range counts in range order, and the total."""
    out, run = [], 0
    for c in counts:
        out.append(run)
        run += int(c)
    return out, run


def count_range(n: int, seed: int, first: int, end: int, rounds: int = _lib.DEFAULT_ROUNDS,
                device=None) -> torch.Tensor:
    """Kept domain indices of [first, end), as a one-element int64 tensor on
    the GPU (written asynchronously on the current stream)."""
    dev = torch.device("cuda", torch.cuda.current_device()) if device is None else torch.device(device)
    c = torch.empty(1, dtype=torch.int64, device=dev)
    _lib.bshuffle_count_range(n, seed, rounds, first, end, c.data_ptr(), torch.cuda.current_stream(dev).cuda_stream)
    return c


def exchange_counts(count: torch.Tensor, group=None) -> tuple[int, int, list[int]]:
    """All-gather one count per rank (int64, on the rank's own device; the
    backend moves it) and return (this rank's offset, total, all counts)."""
    import torch.distributed as dist
    world = dist.get_world_size(group)
    rank = dist.get_rank(group)
    gathered = [torch.empty_like(count) for _ in range(world)]
    dist.all_gather(gathered, count, group=group)
    counts = [int(t.item()) for t in gathered]
    offs, total = offsets(counts)
    return offs[rank], total, counts


def permute_shard(x: torch.Tensor, seed: int, rank: int, world: int, rounds: int = _lib.DEFAULT_ROUNDS,
                  group=None, exchange: bool = True) -> tuple[torch.Tensor, int]:
    """This rank's part of permute(x, seed): (rows [offset, offset + count) of
    the shuffled output, offset).  x (CUDA, rows along dim 0 of 1, 2, 4, 8 or
    16 bytes) is the whole input on every rank.  With exchange=False the
    counts of the ranges before this one are recomputed on this GPU instead of
    being all-gathered (no communication; the count reads no data).  For
    n = 2^k (n >= 16) the counts are the ranges' lengths and nothing is
    exchanged either way."""
    if not x.is_cuda:
        raise ValueError("permute_shard needs a CUDA tensor")
    x = x.contiguous()
    n = x.shape[0]
    elem = x.element_size() * (x.numel() // n if n else 1)
    parts = ranges(n, world)
    first, end = parts[rank]
    if n >= 16 and n & (n - 1) == 0:
        offset, count = first, end - first
    elif exchange:
        mine = count_range(n, seed, first, end, rounds, x.device)
        offset, _, counts = exchange_counts(mine, group)
        count = counts[rank]
    else:
        counts = [count_range(n, seed, f, e, rounds, x.device) for f, e in parts[:rank + 1]]
        offs, _ = offsets([int(c.item()) for c in counts])
        offset, count = offs[rank], int(counts[rank].item())
    out = torch.empty((count,) + tuple(x.shape[1:]), dtype=x.dtype, device=x.device)
    if count:
        _lib.bshuffle_permute_range(x.data_ptr(), out.data_ptr(), n, elem, seed, rounds, first, end, count,
                                    torch.cuda.current_stream(x.device).cuda_stream)
    return out, offset
