#!/usr/bin/env python3
"""Throughput benchmark of the GB300 bijective shuffle.

Workload (one "step"): one shuffle of n = 2^28 uniform random 64-bit keys
(the paper's Sec. 6 payload) already resident in HBM, through the C ABI with
the library's default strategy.  For this power-of-two length that is the
staged path: pass 1 reads the keys in order, inverts the bijection and
buckets (key, slot) by output window; pass 2 scatters each window while it
sits in L2 (same output as Algorithm 1's fused single pass, which
--strategy single_pass or pipelined times instead).  Inputs (2 GiB) are far
larger than the 129 MB L2, so no flush is needed between steps.

Printed on one JSON line (rank 0):
  value        shuffled elements per second, whole job (all ranks)
  roofline     the dominant kernel of the step: its algorithmic bytes per
               launch over its CUDA-event launch time, against the measured
               HBM copy peak, with its DRAM traffic from the committed ncu
               record while the kernel source is unchanged
  e2e          the same metric through the C ABI from pinned host buffers,
               host-to-device and device-to-host copies inside the timed region,
               with the copies alone timed beside it (the host link's floor)
  cpu_baseline the CPU oracle, as it stands: the whole shuffle once on all
               host threads, the sequential oracle on its first 2^21 slots,
               and a sequential Fisher-Yates shuffle of the same keys
  extra        every strategy at n = 2^28 and at the worst-case padding
               n = 2^28 + 12345, the inverse and index outputs, the Sec. 6
               fusion ablation, the Sec. 5 round-count study, the random
               gather bound, the autograd row shuffle, the Monte Carlo and
               Shapley consumers, and the 4096-instance uneven batch
               (batched launch vs one plain launch per instance, called
               from Python and replayed from a CUDA graph)

`--impl reference` times the CPU oracle on this workload instead (bounded
sample per step) and prints the same line with "impl": "reference".
Multi-GPU (torchrun): every rank shuffles its own array (independent
problems, weak scaling) with no collective on the data path.  `--split`
times one shuffle cut by domain range over the ranks instead (strong
scaling), with each rank's own work at 1, 2, 4 and 8 ranks measured part by
part at one GPU; `--table1` prints the layout of the paper's Table 1.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import workloads  # noqa: E402

N_MAIN = 2**28
N_WORST = 2**28 + 12345
ELEM = 8
SEED = 0
ROUNDS = 24
METRIC = "shuffled elements/s at n=2^28 uint64 (VariablePhilox bijective shuffle)"
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "traffic_full_size_launches.json")
STRATEGIES = {"auto": 0, "single_pass": 1, "staged": 2, "pipelined": 3}


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=200)
    p.add_argument("--warmup", type=int, default=5)
    p.add_argument("--impl", choices=["ours", "reference"], default="ours")
    p.add_argument("--no-extra", action="store_true", help="skip the secondary measurements")
    p.add_argument("--strategy", choices=["auto", "single_pass", "staged", "pipelined"], default="auto",
                   help="how bshuffle_permute moves data (identical output)")
    p.add_argument("--profile-batched", type=int, default=0,
                   help="only run warmup + steps batched launches over this many instances (for ncu)")
    p.add_argument("--profile-rows", type=int, default=0,
                   help="only run warmup + steps forward row shuffles of a [this many x 1024] BF16 matrix (for ncu)")
    p.add_argument("--profile-n", type=int, default=0,
                   help="only run warmup + steps launches of the uint64 shuffle at this n (for ncu)")
    p.add_argument("--table1", action="store_true",
                   help="only print the Table 1 layout: M items/s of 64-bit keys at lengths 2^w + 1")
    p.add_argument("--lookback-share", action="store_true",
                   help="only measure the share of CTA time the single passes wait on the look-back "
                        "(builds the library with BSHUFFLE_LOOKBACK_CLOCKS=1 into its own directory)")
    p.add_argument("--no-tune", action="store_true", help="skip the autotuner (for launch lists)")
    p.add_argument("--split", action="store_true",
                   help="time ONE n=2^28 uint64 shuffle split by domain range across the ranks (strong scaling: "
                        "each rank counts its range, the counts are all-gathered, each rank gathers its slots)")
    return p.parse_args()


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


# ------------------------------------------------------------------ clocks

class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during a region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = os.path.join("/tmp", f"bshuffle_clocks_{os.getpid()}_{index}.csv")

    def start(self):
        try:
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"], stdout=self.fh, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        self.proc.wait()
        self.fh.close()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as fh:
            for line in fh:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) < 7:
                    continue
                try:
                    sm.append(float(parts[0]))
                    smax.append(float(parts[1]))
                except ValueError:
                    continue
                for name, flag in zip(names, parts[3:7]):
                    if flag.lower().startswith("active"):
                        reasons.add(name)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------------ distributed

def dist_setup(gpus: int):
    import torch
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world != gpus and world > 1:
        raise SystemExit(f"--gpus {gpus} but WORLD_SIZE={world}")
    if world > 1:
        import torch.distributed as dist
        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    if torch.cuda.is_available():
        torch.cuda.set_device(local)
    return rank, world, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def job_value(n_per_rank: int, world: int, steps: int, region_ms: float) -> float:
    """Whole-job elements/s: every rank shuffles its own n per step (weak
    scaling), over the slowest rank's timed region."""
    return n_per_rank * world * steps / (region_ms * 1e-3)


def max_over_ranks(value: float, world: int) -> float:
    if world == 1:
        return value
    import torch
    import torch.distributed as dist
    dev = torch.device("cuda", torch.cuda.current_device()) if torch.cuda.is_available() else "cpu"
    t = torch.tensor([value], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ------------------------------------------------------------------ CPU oracle

def cpu_oracle_sample(slots: int, trials: int):
    """The oracle, as it stands, on the first `slots` outputs of the workload."""
    import oracle
    x = workloads.uniform_u64(N_MAIN, SEED)
    oracle.permute_first(x, SEED, 1024)  # load + warm
    times = []
    for _ in range(trials):
        t0 = time.perf_counter()
        oracle.permute_first(x, SEED, slots)
        times.append(time.perf_counter() - t0)
    return times


REF_DOMAIN_SAMPLE = 2**24  # domain indices per reference step: 1/16 of the 2^28 domain


def run_reference(args):
    """The CPU oracle, as it stands, on this workload: every step is a bounded
    sample of the n = 2^28 uint64 shuffle, the first 2^24 domain indices (the
    first ~2^24 output slots), by the threaded oracle on all host cores (count
    per domain range, exclusive scan, gather), so that the default 200 steps
    end within a couple of minutes."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle
    cores = oracle.default_threads()
    host = workloads.uniform_u64(N_MAIN, SEED)
    times, slots = [], 0
    for step in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        out = oracle.permute_range_mt(host, SEED, 0, REF_DOMAIN_SAMPLE, ROUNDS, threads=cores)
        times.append(time.perf_counter() - t0)
        slots = out.shape[0]
    times = times[args.warmup:]
    total = sum(times)
    value = slots * len(times) / total
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "elements/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": total / len(times) * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u64", "data": "synthetic", "config": workload_config(args.gpus),
        "cpu_baseline": {"value": value, "unit": "elements/s", "cores": cores, "kind": "oracle",
                         "sample": f"per step the first {REF_DOMAIN_SAMPLE} domain indices ({slots} output slots) "
                                   f"of the n=2^28 uint64 shuffle, threaded oracle on {cores} host threads"},
        "e2e": {"value": value, "unit": "elements/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ GPU

def timed_launches(fn, steps, stream, torch):
    """Per-launch CUDA-event durations (ms) and the whole region (ms)."""
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    region0 = torch.cuda.Event(enable_timing=True)
    region1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    region0.record(stream)
    for k in range(steps):
        starts[k].record(stream)
        fn()
        ends[k].record(stream)
    region1.record(stream)
    torch.cuda.synchronize()
    per = [s.elapsed_time(e) for s, e in zip(starts, ends)]
    return per, region0.elapsed_time(region1)


def timed_region(fn, steps, stream, torch):
    """Milliseconds per launch of `steps` back-to-back launches, one pair of
    CUDA events around them all (no event between launches: for kernels of
    tens of microseconds an event pair per launch adds a gap of the same
    order as the launch ramp)."""
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(steps):
        fn()
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / steps


def traffic_for(kernel: str, fingerprint: str):
    """DRAM bytes per launch from the committed ncu record, if the kernel is unchanged."""
    if not os.path.exists(TRAFFIC_FILE):
        return None
    with open(TRAFFIC_FILE) as fh:
        d = json.load(fh)
    rec = d.get("kernels", {}).get(kernel)
    if rec is None or rec.get("kernel_fingerprint") != fingerprint:
        return None
    return rec.get("dram_bytes_per_launch")


# Pass 1 of the staged path is bound by integer issue: 2^28 inverse cipher
# evaluations per launch.  ncu on that kernel (n = 2^26 uint64, even k) puts
# the FMA-heavy pipe, which issues the integer multiplies, at the top of the
# pipes (sm__pipe_fmaheavy_cycles_active); its peak rate is one warp
# instruction every two cycles per SM sub-partition (16 lanes).  The derived
# peak is the evaluation rate at which that pipe is busy every cycle:
#   152 SMs x 4 sub-partitions x 16 lanes x 2.07 GHz
#   / (FMA-heavy thread instructions per evaluation, counted by ncu as
#      smsp__inst_executed_pipe_fmaheavy.sum x 32 / evaluations).
SMS, SMSP_PER_SM, FMAHEAVY_LANES, SM_HZ = 152, 4, 16, 2.07e9
FMAHEAVY_INST_PER_INVERSE_EVAL = 80.1  # ncu, n = 2^26 uint64: 72 multiplies + 8 of addressing


def alu_peak_evals_per_s() -> float:
    return SMS * SMSP_PER_SM * FMAHEAVY_LANES * SM_HZ / FMAHEAVY_INST_PER_INVERSE_EVAL


def roofline_for(passes, bsbuild, strategy, window_scatter_ms=None, step_ms=None):
    """Roofline of the dominant kernel of one step, plus every pass's line.

    Algorithmic bytes are the metric's: 2 n elem_bytes per shuffle (one read
    and one write of every element), whichever kernels move them.  The staged
    path's own intermediate traffic (value and slot written by pass 1 and
    read by pass 2: 20 B per uint64 element and pass) is reported beside it,
    not as algorithmic.  The staged scatter pass also gets its fraction of
    the window-scatter kernel (the same sequential reads and random writes
    into 8 MiB windows with nothing else), the L2 random-write ceiling it
    runs into."""
    peak, peak_kind = measured_peaks()
    n = N_MAIN
    algo = 2 * n * ELEM
    if len(passes) == 1 and strategy == STRATEGIES["single_pass"]:
        names = [("elem_tile_kernel<uint64, Gather, even k>", "kernels_elem.cu", "hbm", None)]
    elif len(passes) == 1:
        names = [("pipe_tile_kernel<uint64, even k>", "kernels_pipe.cu", "hbm", None)]
    else:
        names = [("staged_bucket_kernel<uint64, even k>", "kernels_staged.cu", "alu", n * (ELEM + ELEM + 4)),
                 ("staged_scatter_kernel<uint64>", "kernels_staged.cu", "hbm", n * (ELEM + 4 + ELEM))]
    lines = []
    for ms, (name, src, bound, staged_bytes) in zip(passes, names):
        gbps = algo / (ms * 1e-3) / 1e9
        line = {"kernel": name, "bound": bound, "ms": ms, "algorithmic_bytes_per_launch": algo,
                "achieved_gbps": gbps, "frac": gbps / peak}
        if staged_bytes is not None:
            sg = staged_bytes / (ms * 1e-3) / 1e9
            line.update(staged_bytes_per_launch=staged_bytes, staged_gbps=sg, staged_frac=sg / peak)
        if bound == "alu":
            evals = float(2**28)
            pk = alu_peak_evals_per_s()
            line["alu"] = {"evaluations_per_launch": evals, "achieved": evals / (ms * 1e-3), "peak": pk,
                           "unit": "inverse cipher evaluations/s", "frac": evals / (ms * 1e-3) / pk,
                           "peak_kind": "derived: 152 SMs x 4 x 16 FMA-heavy lanes x 2.07 GHz / "
                                        f"{FMAHEAVY_INST_PER_INVERSE_EVAL:g} FMA-heavy instructions per evaluation"}
        line["traffic"] = traffic_for(name, bsbuild.kernel_fingerprint(src))
        if name.startswith("staged_scatter") and window_scatter_ms:
            line["window_scatter_ms"] = window_scatter_ms
            line["l2_random_writes_per_s"] = n / (ms * 1e-3)
            line["frac_of_window_scatter"] = window_scatter_ms / ms
        lines.append(line)
    dom = max(lines, key=lambda d: d["ms"])
    roof = {"bound": "hbm", "achieved": dom["achieved_gbps"], "peak": peak, "unit": "GB/s",
            "frac": dom["frac"], "traffic": dom["traffic"], "kernel": dom["kernel"], "launch_ms": dom["ms"],
            "algorithmic_bytes_per_launch": algo,
            "peak_kind": f"{peak_kind} (MEASURED_PEAKS.json hbm_gbs)",
            "kernel_binding_unit": dom["bound"]}
    if dom["traffic"]:
        roof["traffic_over_algorithmic"] = dom["traffic"] / algo
    if step_ms:
        roof["step_ms"] = step_ms
        roof["step_frac"] = algo / (step_ms * 1e-3) / 1e9 / peak
    traffic = [ln["traffic"] for ln in lines]
    if all(traffic):
        roof["step_traffic"] = sum(traffic)
        roof["step_traffic_over_algorithmic"] = sum(traffic) / algo
    return roof, lines


def run_ours(args):
    import torch
    rank, world, local = dist_setup(args.gpus)
    from paper_2106_06161_gb300 import build as bsbuild
    if rank == 0 or world == 1:
        bsbuild.build()
    barrier(world)
    import paper_2106_06161_gb300 as bs
    bs.load()
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)
    sptr = stream.cuda_stream
    bs.bshuffle_set_strategy(STRATEGIES[args.strategy])
    # the library's autotuner picks, per width, the shapes of the plain and
    # pipelined single passes and of the batched kernel (4 and 8 bytes: the
    # widths the bench runs them at); a few seconds
    from paper_2106_06161_gb300 import autotune
    tuning = None if args.no_tune else autotune.tune(widths=(4, ELEM), reps=3, warmup=1, save=False)

    seed = SEED + rank
    host = workloads.uniform_u64(N_MAIN, seed)
    x = torch.from_numpy(host.view(np.int64)).to(dev)
    y = torch.empty_like(x)
    xp, yp = x.data_ptr(), y.data_ptr()

    def step():
        bs.bshuffle_permute(xp, yp, N_MAIN, ELEM, seed, ROUNDS, sptr)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if bs.get_error() != 0:
        raise SystemExit("device error during warm-up")

    clocks = ClockSampler(local)
    barrier(world)
    clocks.start()
    per, region_ms = timed_launches(step, args.steps, stream, torch)
    clk = clocks.stop()
    barrier(world)
    if bs.get_error() != 0:
        raise SystemExit("device error during the timed region")
    region_ms = max_over_ranks(region_ms, world)
    ms_per_step = region_ms / args.steps
    value = job_value(N_MAIN, world, args.steps, region_ms)

    # per-kernel durations, live: the same step with the library's per-pass
    # CUDA events on this stream, read back after every step
    bs.bshuffle_set_pass_timing(True)
    rsteps = max(3, min(args.steps, 30))
    pass_ms = []
    for _ in range(rsteps):
        step()
        pass_ms.append(bs.bshuffle_last_pass_ms(sptr))
    bs.bshuffle_set_pass_timing(False)
    passes = [statistics.mean(col) for col in zip(*pass_ms)]
    # the round trip is exact
    if rank == 0:
        idx = torch.randint(0, N_MAIN, (1 << 16,), device=dev)
        src = bs.indices(N_MAIN, seed)[idx]
        assert torch.equal(y[idx], x[src]), "shuffle output does not match its index sequence"
    # the ceiling of the staged scatter pass, live: sequential reads and
    # random writes inside 8 MiB windows (2^20 uint64), nothing else
    ws = lambda: bs.bshuffle_window_scatter(xp, yp, N_MAIN, ELEM, 20, sptr)  # noqa: E731
    for _ in range(3):
        ws()
    _, ws_region = timed_launches(ws, 10, stream, torch)
    roofline, pass_lines = roofline_for(passes, bsbuild, bs.bshuffle_get_strategy(), ws_region / 10,
                                        ms_per_step)

    e2e = e2e_pipeline(bs, torch, dev, host, seed, args, world)

    extra = {}
    if not args.no_extra and rank == 0:
        extra = secondary(bs, torch, dev, stream)
        extra["sweep"] = sweep(bs, torch, dev, stream)
        bs.bshuffle_set_strategy(STRATEGIES[args.strategy])

    cpu = cpu_baseline(host) if rank == 0 and world == 1 else None

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "elements/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_per_step,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64",
            "data": "synthetic", "config": workload_config(world),
            "logical_gbps": 2 * N_MAIN * ELEM / (ms_per_step * 1e-3) / 1e9,
            "strategy": {0: "auto", 1: "single_pass", 2: "staged", 3: "pipelined"}[bs.bshuffle_get_strategy()],
            "kernels_per_step": len(passes), "passes": pass_lines,
            "tuning": tuning, "extra": extra,
            "e2e": e2e, "gpu_launches": args.steps * len(passes), "clocks": clk,
            "cpu_baseline": cpu, "roofline": roofline,
        }
        # the last key holds the figures a reader of the line's tail needs
        line["summary"] = summary(line)
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def workload_config(world: int) -> dict:
    """The bench line's config, the same for the GPU arm and the reference arm."""
    return {"workload": "bijective shuffle of n=2^28 uniform uint64 keys per GPU, seed 0, 24 rounds",
            "n": N_MAIN, "elem_bytes": ELEM, "rounds": ROUNDS,
            "l2": "inputs (2 GiB) larger than L2, no flush",
            "parallelism": f"independent shuffles, {world} GPU(s)"}


def cpu_baseline(host):
    """The oracle on the host cores: Algorithm 1 on every core over the whole
    workload (count per domain range, exclusive scan, gather: the multi-core
    form of the method), the sequential oracle on the first slots, and a
    sequential Fisher-Yates shuffle (the classical method of Sec. 1) of the
    same n = 2^28 uint64 keys."""
    import oracle
    cores = oracle.default_threads()
    t0 = time.perf_counter()
    out = oracle.permute_mt(host, SEED, ROUNDS, threads=cores)
    mt_s = time.perf_counter() - t0
    del out
    slots = 2**21
    st = cpu_oracle_sample(slots, 4)
    fy = []
    for t in range(2):
        t0 = time.perf_counter()
        oracle.fisher_yates(host, t)
        fy.append(time.perf_counter() - t0)
    return {"value": N_MAIN / mt_s, "unit": "elements/s", "cores": cores, "kind": "oracle",
            "sample": f"the whole n=2^28 uint64 shuffle (seed 0) once, threaded oracle on {cores} host threads "
                      "(count per domain range, exclusive scan, gather)",
            "seconds": mt_s,
            "single_thread": {"value": slots * len(st) / sum(st), "unit": "elements/s", "cores": 1,
                              "sample": f"first {slots} output slots of the same shuffle, {len(st)} trials"},
            "fisher_yates": {"value": N_MAIN / min(fy), "unit": "elements/s", "cores": 1,
                             "sample": "sequential Fisher-Yates (mt19937_64) of the same 2^28 uint64 keys, "
                                       f"best of {len(fy)}"}}


def summary(line: dict) -> dict:
    """Compact figures, printed last so that the tail of the line shows them."""
    ex = line.get("extra") or {}
    roof = line["roofline"]
    out = {"elements_per_s": line["value"], "ms_per_step": line["ms_per_step"],
           "hbm_frac_step": roof.get("step_frac"), "hbm_frac_dominant_kernel": roof["frac"],
           "dominant_kernel": roof["kernel"]}
    for key in ("2p28_u64", "worst_case_2p28_plus_12345_u64"):
        row = {name: round(ex[f"{key}_{name}"]["ms"], 3) for name in ("single_pass", "pipelined", "staged")
               if f"{key}_{name}" in ex}
        if row:
            out[f"{key}_ms"] = row
    sw = ex.get("sweep")
    if sw:
        out["sweep_gelem_per_s"] = {w: {n: round(r["elements_per_s_mean"] / 1e9, 2) for n, r in rows.items()}
                                    for w, rows in sw["rows"].items()}
    b = ex.get("batched_4096_uneven_int32")
    if b:
        out["batched_speedup"] = round(b["speedup"], 2)
        if "speedup_vs_graph" in b:
            out["batched_speedup_vs_graph"] = round(b["speedup_vs_graph"], 2)
    cpu = line.get("cpu_baseline")
    if cpu:
        out["cpu_elements_per_s"] = {"oracle_threads": cpu["value"], "cores": cpu["cores"],
                                     "oracle_1_thread": cpu["single_thread"]["value"],
                                     "fisher_yates": cpu["fisher_yates"]["value"]}
    out["e2e_elements_per_s"] = line["e2e"]["value"]
    if "frac_of_copy_floor" in line["e2e"]:
        out["e2e_frac_of_copy_floor"] = round(line["e2e"]["frac_of_copy_floor"], 3)
    return out


SWEEP_LABELS = {2**10: "2^10", 2**16: "2^16", 2**20: "2^20", 2**24: "2^24", 2**28: "2^28",
                2**28 + 12345: "2^28+12345"}


def sweep(bs, torch, dev, stream, trials=5):
    """Config 2's sweep through the default strategy: 4, 8 and 16-byte
    elements at n in {2^10, 2^16, 2^20, 2^24, 2^28, 2^28 + 12345}.  A trial
    times a run of back-to-back launches (at least about 2 ms of work, so
    that small lengths measure throughput, not one launch); the line gives
    the mean and median of 5 trials (Sec. 6 reports means of 5 trials).
    Inputs below the 129 MB L2 stay resident between launches, as in any
    repeated-launch measurement; payload values do not affect the timing."""
    peak, _ = measured_peaks()
    sptr = stream.cuda_stream
    rows = {}
    for width in (4, 8, 16):
        wrow = {}
        for n in workloads.SWEEP_SIZES:
            cols = width // 8 if width == 16 else 1
            dt = torch.int32 if width == 4 else torch.int64
            shape = (n, cols) if width == 16 else (n,)
            x = torch.randint(-2**31, 2**31 - 1, shape, dtype=dt, device=dev)
            y = torch.empty_like(x)
            xp, yp = x.data_ptr(), y.data_ptr()
            f = lambda: bs.bshuffle_permute(xp, yp, n, width, 0, ROUNDS, sptr)  # noqa: E731
            reps = max(3, min(2000, (2**22 * 16) // (n * width) + 1))
            for _ in range(3):
                f()
            per_elem = []
            for _ in range(trials):
                _, region = timed_launches(f, reps, stream, torch)
                per_elem.append(n * reps / (region * 1e-3))
            mean = statistics.mean(per_elem)
            med = statistics.median(per_elem)
            wrow[SWEEP_LABELS[n]] = {
                "elements_per_s_mean": mean, "elements_per_s_median": med, "launches_per_trial": reps,
                "logical_gbps_mean": mean * 2 * width / 1e9, "hbm_frac_mean": mean * 2 * width / 1e9 / peak}
            del x, y
        rows[f"{width}B"] = wrow
    if bs.get_error() != 0:
        raise SystemExit("device error during the sweep")
    return {"strategy": "auto", "trials": trials, "rows": rows,
            "note": "elements/s = n x launches / region time; logical bytes 2 n elem_bytes per launch"}


def e2e_pipeline(bs, torch, dev, host, seed, args, world):
    """The same shuffle end to end from pinned host memory, through the C ABI.

    Every step copies its input host->device, shuffles it and copies the
    result device->host, all inside the timed region.  Steps are pipelined on
    three streams with two device buffer pairs, so the copy-in of step i+1 and
    the copy-out of step i-1 overlap the shuffle of step i.
    """
    steps = max(3, min(40, args.steps // 5))
    hin = torch.from_numpy(host.view(np.int64)).pin_memory()
    hout = torch.empty_like(hin).pin_memory()
    xs = [torch.empty(N_MAIN, dtype=torch.int64, device=dev) for _ in range(2)]
    ys = [torch.empty(N_MAIN, dtype=torch.int64, device=dev) for _ in range(2)]
    s_in, s_run, s_out = (torch.cuda.Stream(dev) for _ in range(3))
    ev = lambda: torch.cuda.Event(enable_timing=False)  # noqa: E731
    copied_in = [ev(), ev()]
    shuffled = [ev(), ev()]
    copied_out = [ev(), ev()]

    def run(count):
        for i in range(count):
            b = i % 2
            if i >= 2:
                s_in.wait_event(shuffled[b])       # x[b] is free once step i-2 has shuffled it
            with torch.cuda.stream(s_in):
                xs[b].copy_(hin, non_blocking=True)
            copied_in[b].record(s_in)
            s_run.wait_event(copied_in[b])
            if i >= 2:
                s_run.wait_event(copied_out[b])    # y[b] is free once step i-2 has been copied out
            bs.bshuffle_permute(xs[b].data_ptr(), ys[b].data_ptr(), N_MAIN, ELEM, seed, ROUNDS, s_run.cuda_stream)
            shuffled[b].record(s_run)
            s_out.wait_event(shuffled[b])
            with torch.cuda.stream(s_out):
                hout.copy_(ys[b], non_blocking=True)
            copied_out[b].record(s_out)

    run(2)
    torch.cuda.synchronize()
    barrier(world)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(s_in)
    s_run.wait_event(e0)
    s_out.wait_event(e0)
    run(steps)
    s_out.wait_stream(s_run)
    s_out.wait_stream(s_in)
    e1.record(s_out)
    torch.cuda.synchronize()
    ms = max_over_ranks(e0.elapsed_time(e1), world)
    # The copy floor: the same copies alone, both directions at once (the
    # host link, not the shuffle, bounds the end-to-end rate); the best of
    # three trials, since the host link is shared with the machine's other
    # GPUs and a transfer of theirs slows a trial down.
    trials = []
    for _ in range(3):
        c0 = torch.cuda.Event(enable_timing=True)
        c1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        c0.record(s_in)
        s_out.wait_event(c0)
        for i in range(steps):
            with torch.cuda.stream(s_in):
                xs[i % 2].copy_(hin, non_blocking=True)
            with torch.cuda.stream(s_out):
                hout.copy_(ys[i % 2], non_blocking=True)
        s_out.wait_stream(s_in)
        c1.record(s_out)
        torch.cuda.synchronize()
        trials.append(max_over_ranks(c0.elapsed_time(c1), world) / steps)
    floor_ms = min(trials)
    del xs, ys, hin, hout
    return {"value": N_MAIN * world * steps / (ms * 1e-3), "unit": "elements/s",
            "h2d_bytes_per_step": N_MAIN * ELEM, "d2h_bytes_per_step": N_MAIN * ELEM,
            "ms_per_step": ms / steps, "steps": steps,
            "copy_floor_ms_per_step": floor_ms, "copy_floor_trials_ms": trials,
            "frac_of_copy_floor": floor_ms / (ms / steps),
            "pipeline": "copy-in, shuffle and copy-out of consecutive steps overlap on three streams"}


def secondary(bs, torch, dev, stream):
    """Worst-case padding and the uneven batch (one-off measurements)."""
    out = {}
    sptr = stream.cuda_stream
    # every strategy at n = 2^28 and at n = 2^28 + 12345 (domain 2^29, about
    # half of the images dropped: the paper's worst case)
    for label, n_, seed_ in (("2p28_u64", N_MAIN, 0), ("worst_case_2p28_plus_12345_u64", N_WORST, 1)):
        host = workloads.uniform_u64(n_, seed_)
        x = torch.from_numpy(host.view(np.int64)).to(dev)
        y = torch.empty_like(x)
        xp, yp = x.data_ptr(), y.data_ptr()
        f = lambda: bs.bshuffle_permute(xp, yp, n_, ELEM, seed_, ROUNDS, sptr)  # noqa: E731
        for name, strat in (("single_pass", bs.BSHUFFLE_STRATEGY_SINGLE_PASS),
                            ("pipelined", bs.BSHUFFLE_STRATEGY_PIPELINED), ("staged", bs.BSHUFFLE_STRATEGY_STAGED)):
            bs.bshuffle_set_strategy(strat)
            for _ in range(3):
                f()
            per, region = timed_launches(f, 20, stream, torch)
            out[f"{label}_{name}"] = {
                "elements_per_s": n_ * 20 / (region * 1e-3), "ms": statistics.mean(per),
                "logical_gbps": 2 * n_ * ELEM / (statistics.mean(per) * 1e-3) / 1e9}
        bs.bshuffle_set_strategy(bs.BSHUFFLE_STRATEGY_AUTO)
        del x, y

    # the inverse shuffle (staged with the forward cipher at 2^28, the
    # pipelined single pass at 2^28 + 12345) and the index output
    for label, n_ in (("2p28", N_MAIN), ("2p28_plus_12345", N_WORST)):
        x = torch.empty(n_, dtype=torch.int64, device=dev).random_()
        y = torch.empty_like(x)
        inv = lambda: bs.bshuffle_inverse(x.data_ptr(), y.data_ptr(), n_, ELEM, 5, ROUNDS, sptr)  # noqa: E731
        idx = lambda: bs.bshuffle_indices(y.data_ptr(), 8, n_, 5, ROUNDS, sptr)  # noqa: E731
        for fn, name in ((inv, "inverse"), (idx, "indices64")):
            for _ in range(3):
                fn()
            per, region = timed_launches(fn, 10, stream, torch)
            out[f"{name}_{label}_u64"] = {"ms": region / 10, "elements_per_s": n_ * 10 / (region * 1e-3)}
        del x, y

    # the fusion experiment of Sec. 6 at worst-case padding: Bijective0
    # (separate passes), Bijective1 (two-pass scan), Bijective2 (single pass)
    for w in (20, 24, 28):
        n_ = 2**w + 1
        host = workloads.uniform_u64(n_, 3)
        x = torch.from_numpy(host.view(np.int64)).to(dev)
        y = torch.empty_like(x)
        xp, yp = x.data_ptr(), y.data_ptr()
        row = {}
        for variant, name in ((0, "bijective0"), (1, "bijective1"), (2, "bijective2"), (3, "bijective2_pipelined")):
            f = lambda: bs.bshuffle_permute_ablation(xp, yp, n_, ELEM, 3, ROUNDS, variant, sptr)  # noqa: E731
            for _ in range(3):
                f()
            per, region = timed_launches(f, 10, stream, torch)
            row[name] = {"ms": region / 10, "m_items_per_s": n_ * 10 / (region * 1e-3) / 1e6}
        out[f"fusion_ablation_2p{w}_plus_1_u64"] = row
        del x, y

    # Sec. 5's round-count study on the GPU: MMD^2 of 100,000 shuffles per point
    from paper_2106_06161_gb300 import stats as gst
    study = {}
    t0 = time.perf_counter()
    for n_ in (5, 100, 1000):
        for r_ in (4, 8, 12, 16, 20, 24):
            res_ = gst.mmd_test(n_, 100_000, rounds=r_)
            study[f"n{n_}_r{r_}"] = {"mmd2": res_["mmd2"], "clt": res_["clt_threshold"],
                                     "passes_clt": res_["passes_clt"]}
    torch.cuda.synchronize()
    study["seconds"] = time.perf_counter() - t0
    out["mmd_round_study_100000"] = study

    # the paper's throughput bound: a random gather of the same size (no cipher, no scan)
    host = workloads.uniform_u64(N_MAIN, 2)
    x = torch.from_numpy(host.view(np.int64)).to(dev)
    y = torch.empty_like(x)
    xp, yp = x.data_ptr(), y.data_ptr()
    g = lambda: bs.bshuffle_random_gather(xp, yp, N_MAIN, ELEM, sptr)  # noqa: E731
    for _ in range(3):
        g()
    per, region = timed_launches(g, 20, stream, torch)
    out["random_gather_2p28_u64"] = {
        "elements_per_s": N_MAIN * 20 / (region * 1e-3), "launch_ms": statistics.mean(per),
        "logical_gbps": 2 * N_MAIN * ELEM / (statistics.mean(per) * 1e-3) / 1e9}
    del x, y

    # rows: [65536 x 1024] FP32 and BF16 (4 KiB and 2 KiB rows), forward
    # gather and backward scatter of the autograd row shuffle; 65537 rows run
    # the count and copy kernels instead of the scan-free launch.  Each is
    # timed over 50 back-to-back calls between one pair of events, and a
    # plain device copy of the same bytes (torch's copy_) the same way: at
    # 0.1-0.3 GB per call the launch and ramp take a share that the 2 GiB
    # copy behind the measured peak does not see.
    for n_rows in (workloads.ROWS_SHAPE[0], workloads.ROWS_SHAPE[0] + 1):
        for dtype, name in ((torch.float32, "fp32"), (torch.bfloat16, "bf16")):
            rows = torch.randn(n_rows, workloads.ROWS_SHAPE[1], device=dev).to(dtype)
            res = torch.empty_like(rows)
            rb = rows.shape[1] * rows.element_size()
            fwd = lambda: bs.bshuffle_permute(rows.data_ptr(), res.data_ptr(), rows.shape[0], rb, 7, ROUNDS, sptr)  # noqa: E731
            bwd = lambda: bs.bshuffle_inverse(res.data_ptr(), rows.data_ptr(), rows.shape[0], rb, 7, ROUNDS, sptr)  # noqa: E731
            cpy = lambda: res.copy_(rows)  # noqa: E731
            for _ in range(3):
                fwd()
                bwd()
                cpy()
            tf = timed_region(fwd, 50, stream, torch)
            tb = timed_region(bwd, 50, stream, torch)
            tc = timed_region(cpy, 50, stream, torch)
            nbytes = 2 * rows.numel() * rows.element_size()
            out[f"rows_{n_rows}x1024_{name}"] = {
                "forward_ms": tf, "backward_ms": tb,
                "forward_gbps": nbytes / (tf * 1e-3) / 1e9, "backward_gbps": nbytes / (tb * 1e-3) / 1e9,
                "forward_frac": nbytes / (tf * 1e-3) / 1e9 / measured_peaks()[0],
                "backward_frac": nbytes / (tb * 1e-3) / 1e9 / measured_peaks()[0],
                "same_size_copy_ms": tc, "forward_over_copy": tc / tf}
            del rows, res

    # permutation Monte Carlo: 10,000 shuffles of 100,000 float32 + group-mean difference
    xmc = torch.from_numpy(workloads.mc_samples()).to(dev)
    T = torch.empty(workloads.MC_SHUFFLES, dtype=torch.float64, device=dev)
    mc = lambda: bs.bshuffle_mc_group_diff(xmc.data_ptr(), xmc.numel(), workloads.MC_GROUP, 0,  # noqa: E731
                                           workloads.MC_SHUFFLES, ROUNDS, T.data_ptr(), sptr)
    for _ in range(2):
        mc()
    _, tmc = timed_launches(mc, 5, stream, torch)
    out["mc_10000x100000_fp32"] = {"ms": tmc / 5, "shuffles_per_s": workloads.MC_SHUFFLES / (tmc / 5 * 1e-3)}

    # Shapley values of a weighted voting game by permutation sampling:
    # 10,000 players, simple majority, 100,000 sampled orders
    wv = workloads.voting_weights()
    wt = torch.from_numpy(wv.view(np.int32)).to(dev)
    counts = torch.empty(wv.size, dtype=torch.int64, device=dev)
    qv = workloads.majority_quota(wv)
    sv = lambda: bs.bshuffle_shapley_voting(wt.data_ptr(), wv.size, qv, 0, workloads.VOTING_SAMPLES,  # noqa: E731
                                            ROUNDS, counts.data_ptr(), sptr)
    for _ in range(2):
        sv()
    _, tsv = timed_launches(sv, 5, stream, torch)
    out["shapley_voting_10000_players_100000_orders"] = {
        "ms": tsv / 5, "orders_per_s": workloads.VOTING_SAMPLES / (tsv / 5 * 1e-3),
        "pivots": int(counts.sum().item())}

    # 4096 uneven instances, int32: one batched launch vs one plain launch each
    sizes = workloads.batched_sizes()
    data = torch.from_numpy(workloads.batched_payloads(sizes)).to(dev)
    res = torch.empty_like(data)
    descs = bs.packed_descs(data, res, sizes, list(range(len(sizes))))
    count = len(sizes)
    dptr = descs.data_ptr()
    fb = lambda: bs.bshuffle_batched(dptr, count, 4, ROUNDS, sptr)  # noqa: E731
    offs = np.concatenate([[0], np.cumsum(sizes)[:-1]]) * 4
    ins = [data.data_ptr() + int(o) for o in offs]
    outs = [res.data_ptr() + int(o) for o in offs]
    ns = [int(n) for n in sizes]

    def plain_all():
        for t in range(count):
            bs.bshuffle_permute(ins[t], outs[t], ns[t], 4, t, ROUNDS, sptr)

    # the batched kernel's default shape against the autotuner's choice
    from paper_2106_06161_gb300 import _lib as L
    tuned = L.bshuffle_kernel_selected(L.BSHUFFLE_KERNEL_BATCHED, 4)
    by_config = {}
    for config in sorted({0, tuned}):
        L.bshuffle_kernel_select(L.BSHUFFLE_KERNEL_BATCHED, 4, config)
        for _ in range(3):
            fb()
        _, tcfg = timed_launches(fb, 10, stream, torch)
        by_config[config] = tcfg / 10
    L.bshuffle_kernel_select(L.BSHUFFLE_KERNEL_BATCHED, 4, tuned)
    for _ in range(3):
        fb()
    _, tb = timed_launches(fb, 10, stream, torch)
    batched_ref = res.clone()
    plain_all()
    torch.cuda.synchronize()
    _, tp = timed_launches(plain_all, 3, stream, torch)
    same = bool(torch.equal(res, batched_ref))
    # the same 4096 launches captured once in a CUDA graph: their GPU-side
    # time without the host's per-call cost (the first pass on the capture
    # stream sizes its workspace)
    gs = torch.cuda.Stream(dev)
    gptr = gs.cuda_stream
    with torch.cuda.stream(gs):
        for t in range(count):
            bs.bshuffle_permute(ins[t], outs[t], ns[t], 4, t, ROUNDS, gptr)
        gs.synchronize()
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph, stream=gs):
            for t in range(count):
                bs.bshuffle_permute(ins[t], outs[t], ns[t], 4, t, ROUNDS, gptr)
    torch.cuda.synchronize()
    res.zero_()
    for _ in range(2):
        graph.replay()
    torch.cuda.synchronize()
    same_graph = bool(torch.equal(res, batched_ref))
    _, tg = timed_launches(graph.replay, 3, stream, torch)
    del graph
    out["batched_4096_uneven_int32"] = {
        "batched_ms": tb / 10, "plain_ms": tp / 3, "speedup": (tp / 3) / (tb / 10),
        "plain_graph_ms": tg / 3, "speedup_vs_graph": (tg / 3) / (tb / 10),
        "batched_shuffles_per_s": count / (tb / 10 * 1e-3), "plain_shuffles_per_s": count / (tp / 3 * 1e-3),
        "total_elements": int(sizes.sum()), "batched_equals_plain": same, "graph_equals_batched": same_graph,
        "batched_ms_default_shape": by_config[0], "batched_ms_tuned_shape": by_config[tuned],
        "tuned_config": tuned}
    return out


def profile_case(args):
    """warmup + steps plain launches of the uint64 shuffle at n = --profile-n."""
    import torch
    from paper_2106_06161_gb300 import build as bsbuild
    bsbuild.build()
    import paper_2106_06161_gb300 as bs
    bs.bshuffle_set_strategy(STRATEGIES[args.strategy])
    n = args.profile_n
    x = torch.from_numpy(workloads.uniform_u64(n, SEED).view(np.int64)).cuda()
    y = torch.empty_like(x)
    sptr = torch.cuda.current_stream().cuda_stream
    f = lambda: bs.bshuffle_permute(x.data_ptr(), y.data_ptr(), n, ELEM, SEED, ROUNDS, sptr)  # noqa: E731
    for _ in range(args.warmup):
        f()
    per, region = timed_launches(f, args.steps, torch.cuda.current_stream(), torch)
    if bs.get_error() != 0:
        raise SystemExit("device error")
    print(json.dumps({"profile_n": n, "launch_ms": per, "elements_per_s": n * args.steps / (region * 1e-3)}))


def profile_batched(args):
    """warmup + steps batched launches over the first --profile-batched instances."""
    import torch
    from paper_2106_06161_gb300 import build as bsbuild
    bsbuild.build()
    import paper_2106_06161_gb300 as bs
    sizes = workloads.batched_sizes()[:args.profile_batched]
    data = torch.from_numpy(workloads.batched_payloads(sizes)).cuda()
    res = torch.empty_like(data)
    descs = bs.packed_descs(data, res, sizes, list(range(len(sizes))))
    sptr = torch.cuda.current_stream().cuda_stream
    f = lambda: bs.bshuffle_batched(descs.data_ptr(), len(sizes), 4, ROUNDS, sptr)  # noqa: E731
    for _ in range(args.warmup):
        f()
    per, region = timed_launches(f, args.steps, torch.cuda.current_stream(), torch)
    if bs.get_error() != 0:
        raise SystemExit("device error")
    print(json.dumps({"profile_batched": len(sizes), "elements": int(sizes.sum()), "launch_ms": per}))


def profile_rows(args):
    """warmup + steps forward row shuffles of a [--profile-rows x 1024] BF16 matrix."""
    import torch
    from paper_2106_06161_gb300 import build as bsbuild
    bsbuild.build()
    import paper_2106_06161_gb300 as bs
    n_rows, cols = args.profile_rows, workloads.ROWS_SHAPE[1]
    rows = torch.from_numpy(workloads.normal_rows(n_rows, cols)).to(torch.bfloat16).cuda()
    res = torch.empty_like(rows)
    sptr = torch.cuda.current_stream().cuda_stream
    f = lambda: bs.bshuffle_permute(rows.data_ptr(), res.data_ptr(), n_rows, cols * 2,  # noqa: E731
                                    workloads.ROWS_SEED, ROUNDS, sptr)
    for _ in range(args.warmup):
        f()
    ms = timed_region(f, args.steps, torch.cuda.current_stream(), torch)
    if bs.get_error() != 0:
        raise SystemExit("device error")
    print(json.dumps({"profile_rows": n_rows, "row_bytes": cols * 2, "launch_ms": ms,
                      "gbps": 2 * n_rows * cols * 2 / (ms * 1e-3) / 1e9}))


TABLE1_W = (8, 11, 14, 17, 20, 23, 26, 29)


def table1(args):
    """Tables 1 and 2 of Sec. 6 on this GPU: millions of 64-bit keys shuffled
    per second at the worst-case lengths 2^w + 1, for the random-gather bound
    (2^w elements: the measurement kernel takes powers of two), the library's
    default shuffle (the ranked staged form from 256 MiB of input, single-pass
    kernels below), the paper's
    fused single pass (Bijective2) and the LCG bijection through the same
    kernel.  Every launch reuses the same buffers, so lengths up to about
    2^23 stay resident in the 129 MB L2 between launches.  varphilox_graph is
    the default shuffle's calls replayed from a CUDA graph (no host cost per
    call)."""
    import torch
    from paper_2106_06161_gb300 import build as bsbuild
    bsbuild.build()
    import paper_2106_06161_gb300 as bs
    bs.load()
    stream = torch.cuda.current_stream()
    sptr = stream.cuda_stream
    rows = {}
    for w in TABLE1_W:
        n = 2**w + 1
        x = torch.from_numpy(workloads.uniform_u64(n, w).view(np.int64)).cuda()
        y = torch.empty_like(x)
        xp, yp = x.data_ptr(), y.data_ptr()
        reps = max(10, min(2000, 2**26 // n))
        cases = (
            ("gather", 2**w, lambda: bs.bshuffle_random_gather(xp, yp, 2**w, ELEM, sptr)),
            ("varphilox", n, lambda: bs.bshuffle_permute(xp, yp, n, ELEM, w, ROUNDS, sptr)),
            ("varphilox_bijective2", n, lambda: bs.bshuffle_permute_ablation(xp, yp, n, ELEM, w, ROUNDS, 2, sptr)),
            ("lcg", n, lambda: bs.bshuffle_permute_lcg(xp, yp, n, ELEM, w, sptr)),
        )
        row = {"reps": reps}
        for name, items, fn in cases:
            for _ in range(max(3, args.warmup)):
                fn()
            _, region = timed_launches(fn, reps, stream, torch)
            row[name] = items * reps / (region * 1e-3) / 1e6
        # the default shuffle's calls replayed from one CUDA graph: the GPU's
        # rate without the per-call cost of a call from Python (the first
        # call on the capture stream creates its workspace)
        gcalls = min(reps, 200)
        gs = torch.cuda.Stream()
        with torch.cuda.stream(gs):
            bs.bshuffle_permute(xp, yp, n, ELEM, w, ROUNDS, gs.cuda_stream)
            gs.synchronize()
            graph = torch.cuda.CUDAGraph()
            with torch.cuda.graph(graph, stream=gs):
                for _ in range(gcalls):
                    bs.bshuffle_permute(xp, yp, n, ELEM, w, ROUNDS, gs.cuda_stream)
        torch.cuda.synchronize()
        graph.replay()
        _, gregion = timed_launches(graph.replay, 3, stream, torch)
        row["varphilox_graph"] = n * gcalls * 3 / (gregion * 1e-3) / 1e6
        del graph
        if bs.get_error() != 0:
            raise SystemExit("device error")
        rows[f"2^{w}+1"] = row
        del x, y
    print(json.dumps({"table": "M items/s, 64-bit keys, lengths 2^w + 1, 24 rounds, mean over reps launches",
                      "gpu": torch.cuda.get_device_name(), "rows": rows}), flush=True)


def lookback_share(args):
    """Share of CTA time the plain and the pipelined single pass wait on the
    inter-tile look-back, from SM clock cycles counted on the device by a
    measurement build of the library (BSHUFFLE_LOOKBACK_CLOCKS=1), at the
    worst-case padding n = 2^28 + 12345 and at n = 2^28 (uint64)."""
    import ctypes

    import torch
    from paper_2106_06161_gb300 import build as bsbuild
    path = bsbuild.build(defines=("BSHUFFLE_LOOKBACK_CLOCKS=1",),
                         build_dir=os.path.join(bsbuild.HERE, "_build_clocks"))
    lib = ctypes.CDLL(path)
    lib.bshuffle_permute.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint32,
                                     ctypes.c_uint64, ctypes.c_uint32, ctypes.c_void_p]
    lib.bshuffle_debug_lookback_cycles.argtypes = [ctypes.c_void_p, ctypes.POINTER(ctypes.c_uint64),
                                                   ctypes.POINTER(ctypes.c_uint64)]
    lib.bshuffle_get_error.argtypes = [ctypes.c_void_p]
    stream = torch.cuda.current_stream()
    sptr = stream.cuda_stream
    rows = {}
    for n in (N_WORST, N_MAIN):
        x = torch.from_numpy(workloads.uniform_u64(n, 1).view(np.int64)).cuda()
        y = torch.empty_like(x)
        for name, strat in (("single_pass", 1), ("pipelined", 3)):
            lib.bshuffle_set_strategy(strat)
            f = lambda: lib.bshuffle_permute(x.data_ptr(), y.data_ptr(), n, ELEM, 1, ROUNDS, sptr)  # noqa: E731
            for _ in range(max(3, args.warmup)):
                f()
            lb, cta = ctypes.c_uint64(0), ctypes.c_uint64(0)
            rc = lib.bshuffle_debug_lookback_cycles(sptr, ctypes.byref(lb), ctypes.byref(cta))
            if rc != 0:
                raise SystemExit(f"measurement build not active ({rc})")
            _, region = timed_launches(f, args.steps, stream, torch)
            rc = lib.bshuffle_debug_lookback_cycles(sptr, ctypes.byref(lb), ctypes.byref(cta))
            if rc != 0 or lib.bshuffle_get_error(sptr) != 0:
                raise SystemExit("device error")
            rows[f"n={n} {name}"] = {"lookback_share": lb.value / cta.value if cta.value else None,
                                     "lookback_cycles": lb.value, "cta_cycles": cta.value,
                                     "ms_per_launch_measurement_build": region / args.steps}
        lib.bshuffle_set_strategy(0)
        del x, y
    print(json.dumps({"lookback_share": rows, "launches": args.steps,
                      "definition": "plain kernel: cycles of each tile's look-back (its other warps wait at the "
                                    "barrier) / cycles of its CTAs; pipelined kernel: cycles its compute warps "
                                    "wait for a tile's rank / cycles of its persistent CTAs"}), flush=True)


def run_split(args):
    """One shuffle split across the ranks by domain range (strong scaling).
    Every rank holds the whole input and gathers its range's kept elements
    into its run of output slots; the timed region is the slowest rank's.
    For n = 2^28 nothing is dropped, so a range's count is its length and the
    ranks exchange nothing (other lengths count their ranges and all-gather
    the counts).  Exactness is checked against the library's own unsplit
    shuffle on rank 0's slots."""
    import torch
    rank, world, local = dist_setup(args.gpus)
    from paper_2106_06161_gb300 import build as bsbuild
    if rank == 0 or world == 1:
        bsbuild.build()
    barrier(world)
    import paper_2106_06161_gb300 as bs
    from paper_2106_06161_gb300 import split
    bs.load()
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)
    x = torch.from_numpy(workloads.uniform_u64(N_MAIN, SEED).view(np.int64)).to(dev)
    exchange = world > 1
    step = lambda: split.permute_shard(x, SEED, rank, world, ROUNDS, exchange=exchange)  # noqa: E731
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    barrier(world)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        part, offset = step()
    e1.record(stream)
    torch.cuda.synchronize()
    if bs.get_error() != 0:
        raise SystemExit("device error")
    region_ms = max_over_ranks(e0.elapsed_time(e1), world)
    whole = bs.permute(x, SEED, ROUNDS)
    ok = bool(torch.equal(whole[offset:offset + part.shape[0]], part))
    emulated = emulated_ranks(bs, split, torch, stream) if world == 1 else None
    if rank == 0:
        ms = region_ms / args.steps
        line = {"metric": METRIC, "value": N_MAIN * args.steps / (region_ms * 1e-3), "unit": "elements/s",
                "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
                "higher_is_better": True, "scaling": "strong", "vs_baseline": None, "dtype": "u64",
                "data": "synthetic",
                "config": dict(workload_config(world), parallelism=f"one shuffle split by domain range over "
                                                                  f"{world} GPU(s); n = 2^k keeps every index, "
                                                                  f"so no exchange"),
                "split_equals_unsplit_on_rank0": ok, "gpu_launches": args.steps}
        if emulated is not None:
            line["emulated_ranks"] = emulated
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def emulated_ranks(bs, split, torch, stream, reps=5):
    """Each rank's own work at P ranks, measured part by part on this GPU: its
    range count (not for n = 2^k), the host read of the count, and its range
    gather from the whole input, as one rank would run them alone on its own
    GPU; the slowest part bounds a step at P GPUs, the all-gather of the
    counts aside.  Every part's output is checked against the unsplit
    shuffle."""
    sptr = stream.cuda_stream
    out = {}
    for n in (N_MAIN, N_MAIN + 12345):
        x = torch.from_numpy(workloads.uniform_u64(n, SEED).view(np.int64)).cuda()
        whole = bs.permute(x, SEED, ROUNDS)
        y = torch.empty_like(x)
        pow2 = n & (n - 1) == 0
        rows, exact = {}, True
        for parts in (1, 2, 4, 8):
            ranges = split.ranges(n, parts)
            offset, times = 0, []
            for first, end in ranges:
                def work(first=first, end=end):
                    count = end - first if pow2 else int(split.count_range(n, SEED, first, end, ROUNDS).item())
                    bs.bshuffle_permute_range(x.data_ptr(), y.data_ptr(), n, ELEM, SEED, ROUNDS, first, end, count,
                                              sptr)
                    return count
                count = work()
                torch.cuda.synchronize()
                exact = exact and bool(torch.equal(y[:count], whole[offset:offset + count]))
                offset += count
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                for _ in range(reps):
                    work()
                e1.record(stream)
                torch.cuda.synchronize()
                times.append(e0.elapsed_time(e1) / reps)
            exact = exact and offset == n
            rows[str(parts)] = {"max_part_ms": max(times), "parts_ms": times}
        if bs.get_error() != 0:
            raise SystemExit("device error")
        out["2^28" if pow2 else "2^28+12345"] = {"parts_equal_unsplit": exact, "by_parts": rows}
        del x, y, whole
        torch.cuda.empty_cache()
    return out


def main():
    args = parse()
    if args.split:
        run_split(args)
    elif args.lookback_share:
        lookback_share(args)
    elif args.table1:
        table1(args)
    elif args.profile_batched:
        profile_batched(args)
    elif args.profile_rows:
        profile_rows(args)
    elif args.profile_n:
        profile_case(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
