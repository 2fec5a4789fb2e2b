"""Autotuner of the plain single-pass permute kernel.

For each element width (4, 8, 16 bytes) every configuration the library
offers (CTA size, domain indices per thread, rounds unrolled at compile time;
see bshuffle_tuning_describe) is timed with CUDA events on the current stream
at a worst-case padded length (n = 2^k + 1: half of the 2^(k+1) domain is
evaluated and dropped), and the fastest is selected.  Every configuration
computes the same output; only speed differs.  The selection applies where
the plain kernel runs: BSHUFFLE_STRATEGY_SINGLE_PASS, and 16-byte gathers
under the default strategy (4- and 8-byte gathers default to the pipelined
kernel, whose shape is fixed: three persistent CTAs of eight compute warps
and one look-back warp per SM measured fastest).

Results are cached as JSON keyed by device name, compute capability and SM
count, then element width.  `apply_cached()` re-selects the cached choices in
a new process.
"""
from __future__ import annotations

import json
import os
import statistics

import torch

from . import _lib

CACHE = os.environ.get("BSHUFFLE_TUNE_CACHE",
                       os.path.join(os.path.expanduser("~"), ".cache", "bshuffle", "tuning.json"))
WIDTHS = (4, 8, 16)


def device_key(device: int | None = None) -> str:
    d = torch.cuda.current_device() if device is None else device
    p = torch.cuda.get_device_properties(d)
    return f"{p.name}|sm_{p.major}{p.minor}|{p.multi_processor_count}SM"


def _payload(n: int, width: int, device) -> torch.Tensor:
    g = torch.Generator(device="cpu").manual_seed(width)
    if width == 4:
        return torch.randint(-2**31, 2**31 - 1, (n,), dtype=torch.int32, generator=g).to(device)
    if width == 8:
        return torch.randint(-2**62, 2**62, (n,), dtype=torch.int64, generator=g).to(device)
    return torch.randint(-2**62, 2**62, (n, 2), dtype=torch.int64, generator=g).to(device)


def _time_ms(fn, reps: int, warmup: int) -> float:
    stream = torch.cuda.current_stream()
    for _ in range(warmup):
        fn()
    times = []
    for _ in range(reps):
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        fn()
        b.record(stream)
        b.synchronize()
        times.append(a.elapsed_time(b))
    return statistics.median(times)


def tune(widths=WIDTHS, n: int = 2**26 + 1, rounds: int = 24, reps: int = 5, warmup: int = 2,
         save: bool = True, cache: str = CACHE) -> dict:
    """Time every configuration per width, select the fastest, optionally cache it."""
    from . import permute
    dev = torch.device("cuda", torch.cuda.current_device())
    configs = _lib.bshuffle_tuning_configs()
    old_strategy = _lib.bshuffle_get_strategy()
    _lib.bshuffle_set_strategy(_lib.BSHUFFLE_STRATEGY_SINGLE_PASS)
    result = {}
    try:
        for w in widths:
            x = _payload(n, w, dev)
            out = torch.empty_like(x)
            timings = {}
            for c in configs:
                if c["rounds_unrolled"] not in (0, rounds):
                    continue
                _lib.bshuffle_tuning_select(w, c["config"])
                timings[c["config"]] = _time_ms(lambda: permute(x, 1, rounds, out=out), reps, warmup)
            best = min(timings, key=timings.get)
            _lib.bshuffle_tuning_select(w, best)
            result[str(w)] = {"config": best, "ms": {str(k): v for k, v in timings.items()}, "n": n,
                              "rounds": rounds}
            del x, out
    finally:
        _lib.bshuffle_set_strategy(old_strategy)
    if save:
        data = {}
        if os.path.exists(cache):
            with open(cache) as fh:
                data = json.load(fh)
        data[device_key()] = result
        os.makedirs(os.path.dirname(cache) or ".", exist_ok=True)
        tmp = cache + f".tmp{os.getpid()}"
        with open(tmp, "w") as fh:
            json.dump(data, fh, indent=1)
        os.replace(tmp, cache)
    return result


def apply_cached(cache: str = CACHE) -> bool:
    """Select the cached configurations for the current device; False if none."""
    if not os.path.exists(cache):
        return False
    with open(cache) as fh:
        data = json.load(fh)
    entry = data.get(device_key())
    if not entry:
        return False
    for w, rec in entry.items():
        _lib.bshuffle_tuning_select(int(w), int(rec["config"]))
    return True
