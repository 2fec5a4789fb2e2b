"""Host side of one shuffle split across ranks by domain range, on the CPU:
the range plan covers the domain, the offsets are the exclusive sums of the
range counts, and two gloo ranks exchanging their counts (taken from the
oracle's per-range count) get the slot runs that tile [0, n)."""
import multiprocessing as mp
import os
import socket
import sys

import pytest

import oracle

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_ranges_tile_the_domain():
    from paper_2106_06161_gb300 import split
    for n in (1, 5, 17, 1000, 4097, 2**20 + 1, 2**28 + 12345):
        k = oracle.domain_bits(n)
        for parts in (1, 2, 3, 4, 7, 8):
            rs = split.ranges(n, parts)
            assert len(rs) == parts and rs[0][0] == 0 and rs[-1][1] == 2**k
            assert all(a[1] == b[0] for a, b in zip(rs, rs[1:]))
            assert max(e - f for f, e in rs) - min(e - f for f, e in rs) <= 1
    with pytest.raises(ValueError):
        split.ranges(10, 0)


def test_offsets_are_exclusive_sums():
    from paper_2106_06161_gb300 import split
    assert split.offsets([3, 0, 5, 2]) == ([0, 3, 3, 8], 10)
    assert split.offsets([]) == ([], 0)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, n, seed, q):
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import torch
    import torch.distributed as dist

    import oracle as orc
    from paper_2106_06161_gb300 import split
    dist.init_process_group("gloo", rank=rank, world_size=world)
    first, end = split.ranges(n, world)[rank]
    mine = torch.tensor([orc.count_range(n, seed, first, end)], dtype=torch.int64)
    offset, total, counts = split.exchange_counts(mine)
    dist.destroy_process_group()
    q.put((rank, first, end, offset, total, counts))


@pytest.mark.parametrize("world", [2, 3])
def test_count_exchange_over_gloo(world):
    n, seed = 100_003, 9
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, world, port, n, seed, q)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(180)
        assert p.exitcode == 0
    got = sorted(q.get(timeout=10) for _ in range(world))
    idx = oracle.indices(n, seed)
    for rank, first, end, offset, total, counts in got:
        assert total == n and sum(counts) == n
        assert offset == sum(counts[:rank])
        # the rank's slots hold exactly its range's kept images, in order
        k = oracle.domain_bits(n)
        keys = oracle.round_keys(seed, 24)
        import numpy as np
        img = oracle.varphilox(np.arange(first, end, dtype=np.uint64), k, keys)
        assert np.array_equal(idx[offset:offset + counts[rank]], img[img < n])
