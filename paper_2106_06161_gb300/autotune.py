"""Autotuner of the kernels the default strategy runs for unstaged shuffles.

Per element width (4, 8 and 16 bytes) and per kernel, every configuration the
library offers (bshuffle_kernel_describe: threads per CTA, domain indices
per thread, resident CTAs per SM targeted, rounds unrolled at compile time)
is timed with CUDA events on the current stream, at the size class where the
default strategy runs that kernel, and the fastest is selected:

* the plain single-pass kernel (BSHUFFLE_KERNEL_SINGLE_PASS) on a domain of
  2^17 (n = 2^16 + 1): below 2^18 domain indices the default runs it, and a
  call is all latency, so a timing is a run of back-to-back calls;
* the pipelined single pass (BSHUFFLE_KERNEL_PIPELINED) at n = 2^24 + 1
  (domain 2^25): from 2^18 domain indices up to the staged path's size, and
  for 16-byte elements of any larger length;
* the persistent batched kernel (BSHUFFLE_KERNEL_BATCHED) on an uneven batch
  of independent shuffles with log-uniform sizes in [100, 2,000,000] (4,096
  instances of 4-byte elements, 1,024 of 8- and 16-byte elements).

Every configuration computes the same output; only speed differs.  Results
are cached as JSON keyed by device name, compute capability and SM count,
then kernel and element width; `apply_cached()` re-selects the cached
choices in a new process.
"""
from __future__ import annotations

import json
import os
import statistics

import numpy as np
import torch

from . import _lib

CACHE = os.environ.get("BSHUFFLE_TUNE_CACHE",
                       os.path.join(os.path.expanduser("~"), ".cache", "bshuffle", "tuning.json"))
WIDTHS = (4, 8, 16)
KERNELS = {"single_pass": _lib.BSHUFFLE_KERNEL_SINGLE_PASS, "pipelined": _lib.BSHUFFLE_KERNEL_PIPELINED,
           "batched": _lib.BSHUFFLE_KERNEL_BATCHED}
PLAIN_N = 2**16 + 1
PIPE_N = 2**24 + 1


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


def uneven_sizes(count: int, lo: int = 100, hi: int = 2_000_000, seed: int = 2024) -> np.ndarray:
    """floor(exp(U(ln lo, ln hi))) per instance: an uneven batch."""
    u = np.random.default_rng(seed).uniform(np.log(lo), np.log(hi), size=count)
    return np.floor(np.exp(u)).astype(np.int64)


def _time_ms(fn, reps: int, warmup: int, calls: int = 1) -> float:
    """Median over reps of the time of `calls` back-to-back calls."""
    stream = torch.cuda.current_stream()
    for _ in range(warmup):
        fn()
    times = []
    for _ in range(reps):
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(calls):
            fn()
        b.record(stream)
        b.synchronize()
        times.append(a.elapsed_time(b) / calls)
    return statistics.median(times)


def _sweep(kernel: int, width: int, fn, rounds: int, reps: int, warmup: int, calls: int = 1) -> dict:
    timings = {}
    for c in _lib.bshuffle_kernel_configs(kernel):
        if c["rounds_unrolled"] not in (0, rounds) and kernel == _lib.BSHUFFLE_KERNEL_SINGLE_PASS:
            continue  # a fixed round count that this call does not use
        _lib.bshuffle_kernel_select(kernel, width, c["config"])
        timings[c["config"]] = _time_ms(fn, reps, warmup, calls)
    best = min(timings, key=timings.get)
    _lib.bshuffle_kernel_select(kernel, width, best)
    return {"config": best, "ms": {str(k): v for k, v in timings.items()}}


def tune(widths=WIDTHS, kernels=tuple(KERNELS), rounds: int = 24, reps: int = 5, warmup: int = 2,
         save: bool = True, cache: str = CACHE, plain_n: int = PLAIN_N, pipe_n: int = PIPE_N,
         batch_count: int | None = None) -> dict:
    """Time every configuration per kernel and width, select the fastest,
    optionally cache it.  Returns {kernel: {width: {"config", "ms", ...}}}."""
    dev = torch.device("cuda", torch.cuda.current_device())
    stream = torch.cuda.current_stream(dev).cuda_stream
    old_strategy = _lib.bshuffle_get_strategy()
    _lib.bshuffle_set_strategy(_lib.BSHUFFLE_STRATEGY_AUTO)
    result = {k: {} for k in kernels}
    try:
        for w in widths:
            if "single_pass" in kernels:
                x = _payload(plain_n, w, dev)
                out = torch.empty_like(x)
                fn = lambda: _lib.bshuffle_permute(x.data_ptr(), out.data_ptr(), plain_n, w, 1, rounds, stream)  # noqa: E731
                rec = _sweep(_lib.BSHUFFLE_KERNEL_SINGLE_PASS, w, fn, rounds, reps, warmup, calls=50)
                result["single_pass"][str(w)] = dict(rec, n=plain_n, rounds=rounds, calls_per_timing=50)
                del x, out
            if "pipelined" in kernels:
                x = _payload(pipe_n, w, dev)
                out = torch.empty_like(x)
                fn = lambda: _lib.bshuffle_permute(x.data_ptr(), out.data_ptr(), pipe_n, w, 1, rounds, stream)  # noqa: E731
                rec = _sweep(_lib.BSHUFFLE_KERNEL_PIPELINED, w, fn, rounds, reps, warmup)
                result["pipelined"][str(w)] = dict(rec, n=pipe_n, rounds=rounds)
                del x, out
            if "batched" in kernels:
                count = batch_count or (4096 if w == 4 else 1024)
                sizes = uneven_sizes(count)
                x = _payload(int(sizes.sum()), w, dev)
                out = torch.empty_like(x)
                from . import packed_descs
                descs = packed_descs(x, out, sizes, list(range(count)))
                fn = lambda: _lib.bshuffle_batched(descs.data_ptr(), count, w, rounds, stream)  # noqa: E731
                rec = _sweep(_lib.BSHUFFLE_KERNEL_BATCHED, w, fn, rounds, reps, warmup)
                result["batched"][str(w)] = dict(rec, instances=count, elements=int(sizes.sum()), rounds=rounds)
                del x, out, descs
            torch.cuda.empty_cache()
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
    for kernel, per_width in entry.items():
        if kernel not in KERNELS:
            continue
        for w, rec in per_width.items():
            _lib.bshuffle_kernel_select(KERNELS[kernel], int(w), int(rec["config"]))
    return True


def reset() -> None:
    """Configuration 0 (the default) for every kernel and width."""
    for k in KERNELS.values():
        for w in WIDTHS:
            _lib.bshuffle_kernel_select(k, w, 0)
