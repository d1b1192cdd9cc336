#!/usr/bin/env python3
"""Benchmark of the in-place Knuth shuffle on one GB300 (one JSON line).

Workload (default): n = 10^9 uint64 keys A[i] = i, hashed targets with seed 2,
eps = 0.25; one step is one complete shuffle of the array (every round of the
deterministic-reservation driver, in one persistent launch).  The array (8 GB)
is far larger than L2 (126 MB), so no flush is needed between steps; each step
shuffles the previous step's output, which is an equally valid input.

Reported: elements/s (value), the roofline of the round kernel against the
measured HBM copy bandwidth, the same metric end to end from pinned host
memory, an eps sweep (0.5 and 0.75), the scratch bytes against the
c * n^(1-eps) bound, and the CPU oracle timed on a bounded sample.

``--impl reference`` times the CPU oracle (the sequential Knuth shuffle) on a
bounded sample of the same workload instead.  With N > 1 GPUs (torchrun) every
rank shuffles its own replica (a single shuffle does not shard), and the time
is the maximum over ranks.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

PAPER_RP_FINAL_1E9_MS = 3960.0  # RP-Final, n = 1000M 64-bit ints, 72 cores + HT (Table "rp-runtime")
BYTES_PER_ELEM = {"u32": 72, "u64": 80, "rec128": 96}  # i side r+w + one 32-B sector read + write
ELEM_BYTES = {"u32": 4, "u64": 8, "rec128": 16}
KERNEL_SOURCES = ["paper_2103_01216_gb300/csrc/grid_driver.cu", "paper_2103_01216_gb300/csrc/device.cuh"]
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "rounds_kernel_traffic.txt")


def kernel_hash() -> str:
    h = hashlib.sha256()
    for p in KERNEL_SOURCES:
        with open(os.path.join(ROOT, p), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def recorded_traffic(n: int, dtype: str, eps: float):
    """DRAM bytes per launch from the committed ncu summary, scaled to n, if it
    was taken on the current kernel source; else None."""
    if not os.path.exists(TRAFFIC_FILE):
        return None
    vals = {}
    with open(TRAFFIC_FILE) as f:
        for line in f:
            if ":" in line and not line.startswith("#"):
                k, _, v = line.partition(":")
                vals[k.strip()] = v.strip()
    try:
        if vals.get("kernel_source_hash") != kernel_hash():
            return None
        if vals.get("dtype") != dtype or abs(float(vals.get("eps", -1)) - eps) > 1e-9:
            return None
        per_elem = float(vals["dram_bytes_per_launch"]) / float(vals["n"])
        return per_elem * n
    except (KeyError, ValueError):
        return None


class ClockSampler:
    """nvidia-smi clocks and throttle reasons, sampled every 200 ms in the background."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.dev = device_index
        self.proc = None
        self.lines = []
        self.thread = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.dev), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, ValueError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
        if self.thread is not None:
            self.thread.join(timeout=2)
        return False

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.lines:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for name, v in zip(names, parts[3:7]):
                if v.lower().startswith("active"):
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def measured_peak_hbm():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        if d.get("hbm_gbs"):
            return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def dist_info():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def cpu_oracle_sample(dtype: str, seed: int, n_sample: int):
    """Times the oracle (single thread) on n_sample elements; returns elems/s and seconds."""
    import numpy as np

    import oracle
    import workloads

    oracle.build()
    arr = workloads.make(n_sample, dtype)
    t0 = time.perf_counter()
    oracle.knuth_hash(arr, seed)
    dt = time.perf_counter() - t0
    del np
    return n_sample / dt, dt


def run_reference(args):
    rank, world, _ = dist_info()
    if rank != 0:
        return 0
    n_sample = args.cpu_sample
    # warmup steps and timed steps, each a bounded sample of the workload
    for _ in range(args.warmup):
        cpu_oracle_sample(args.dtype, args.seed, max(1, n_sample // 8))
    times = []
    for _ in range(args.steps):
        _, dt = cpu_oracle_sample(args.dtype, args.seed, n_sample)
        times.append(dt)
    mean_t = sum(times) / len(times)
    value = n_sample / mean_t
    line = {
        "impl": "reference",
        "metric": "shuffled elems/s",
        "value": value,
        "unit": "elems/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": mean_t * 1e3,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": args.dtype,
        "data": "synthetic",
        "config": workload_config(args),
        "cpu_baseline": {"value": value, "unit": "elems/s", "cores": 1, "kind": "oracle",
                         "sample": f"sequential Knuth shuffle (oracle/knuth.c) of {n_sample} {args.dtype} "
                                   f"elements A[i]=i, seed {args.seed}, one host thread"},
        "e2e": {"value": value, "unit": "elems/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def workload_config(args):
    return {
        "workload": f"knuth_shuffle_n{args.n}_{args.dtype}_seed{args.seed}_eps{args.eps}",
        "n": args.n,
        "elem": args.dtype,
        "eps": args.eps,
        "seed": args.seed,
        "targets": "H[i]=mulhi64(splitmix64(seed^i), i+1)",
        "input": "A[i]=i" if args.dtype != "rec128" else "{key=i, payload=splitmix64(i)}",
        "l2": "inputs larger than L2 (no flush)",
        "global_batch": 1,
        "parallelism": "replicas" if dist_info()[1] > 1 else "single",
    }


def make_device_input(torch, n, dtype, device):
    if dtype == "u32":
        return torch.arange(n, dtype=torch.int32, device=device)
    if dtype == "u64":
        return torch.arange(n, dtype=torch.int64, device=device)
    A = torch.empty((n, 2), dtype=torch.int64, device=device)
    A[:, 0] = torch.arange(n, dtype=torch.int64, device=device)
    A[:, 1] = A[:, 0] * 3 + 1  # payload content is irrelevant to the timing
    return A


def time_steps(torch, pip, A, seed, eps, steps, warmup, stream, opts):
    for _ in range(warmup):
        pip.shuffle(A, seed=seed, eps=eps, stream=stream, **opts)
    pip.check(stream)
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    torch.cuda.synchronize()
    for s, e in evs:
        s.record(stream)
        pip.shuffle(A, seed=seed, eps=eps, stream=stream, **opts)
        e.record(stream)
    pip.check(stream)
    torch.cuda.synchronize()
    return [s.elapsed_time(e) for s, e in evs]


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=10**9)
    ap.add_argument("--dtype", default="u64", choices=["u32", "u64", "rec128"])
    ap.add_argument("--seed", type=int, default=2)
    ap.add_argument("--eps", type=float, default=0.25)
    ap.add_argument("--sweep", default="0.5,0.75", help="extra eps values timed (1 step each); '' to skip")
    ap.add_argument("--e2e-steps", type=int, default=3)
    ap.add_argument("--cpu-sample", type=int, default=1 << 27, help="elements in the oracle's timed sample")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--prefix-c", type=float, default=0.0)
    ap.add_argument("--fresh", type=int, default=0)
    ap.add_argument("--slot-factor", type=int, default=0)
    ap.add_argument("--grid-blocks", type=int, default=0)
    ap.add_argument("--block-threads", type=int, default=0)
    ap.add_argument("--flags", type=int, default=0, help="PIP_FLAG_* bits (2 = L2 prefetch of the next block)")
    args = ap.parse_args()

    if args.impl == "reference":
        return run_reference(args)

    import torch

    import paper_2103_01216_gb300 as pip
    from paper_2103_01216_gb300 import _build

    rank, world, local = dist_info()
    if world > 1:
        import torch.distributed as dist

        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        dist = None
        torch.cuda.set_device(0)
    if rank == 0:
        _build.build()
    if dist is not None:
        dist.barrier()
    pip.lib()
    device = torch.device("cuda", torch.cuda.current_device())
    stream = torch.cuda.current_stream()
    opts = {}
    if args.prefix_c:
        opts["prefix_c"] = args.prefix_c
    if args.fresh:
        opts["fresh_per_round"] = args.fresh
    if args.slot_factor:
        opts["slot_factor"] = args.slot_factor
    if args.grid_blocks:
        opts["grid_blocks"] = args.grid_blocks
    if args.block_threads:
        opts["block_threads"] = args.block_threads
    if args.flags:
        opts["flags"] = args.flags

    n, dtype, seed, eps = args.n, args.dtype, args.seed, args.eps
    plan = pip.plan(n, dtype, eps, **opts)
    A = make_device_input(torch, n, dtype, device)
    torch.cuda.synchronize()

    # device-resident timing, with clocks sampled during the timed region
    free_before, _ = torch.cuda.mem_get_info()
    with ClockSampler(torch.cuda.current_device()) as clk:
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()
        ms = time_steps(torch, pip, A, seed, eps, args.steps, args.warmup, stream, opts)
        torch.cuda.synchronize()
    clocks = clk.summary()
    total_ms = sum(ms)
    if dist is not None:
        t = torch.tensor([total_ms], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
    ms_per_step = total_ms / args.steps
    value = world * n * args.steps / (total_ms / 1e3)

    # aux bytes as seen by the allocator while a shuffle is in flight
    side = torch.cuda.Stream()
    with torch.cuda.stream(side):
        pip.shuffle(A, seed=seed, eps=eps, stream=side, **opts)
        free_during, _ = torch.cuda.mem_get_info()
    pip.check(side)
    aux_delta = max(0, free_before - free_during)

    # stats of one run
    st_buf = torch.zeros(pip.STATS_BYTES, dtype=torch.uint8, device=device)
    pip.shuffle(A, seed=seed, eps=eps, stats=st_buf, **opts)
    pip.check()
    st = pip.read_stats(st_buf)

    # end to end: pinned host -> device, shuffle, device -> host, every step
    e2e = None
    if args.e2e_steps > 0:
        host = A.cpu().pin_memory()
        out = torch.empty_like(host).pin_memory()
        dev = torch.empty_like(A)
        nbytes = host.numel() * host.element_size()
        for _ in range(1):
            dev.copy_(host, non_blocking=True)
            pip.shuffle(dev, seed=seed, eps=eps, **opts)
            out.copy_(dev, non_blocking=True)
        torch.cuda.synchronize()
        s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        if dist is not None:
            dist.barrier()
        s.record()
        for _ in range(args.e2e_steps):
            dev.copy_(host, non_blocking=True)
            pip.shuffle(dev, seed=seed, eps=eps, **opts)
            out.copy_(dev, non_blocking=True)
        e.record()
        pip.check()
        e2e_ms = s.elapsed_time(e)
        if dist is not None:
            t = torch.tensor([e2e_ms], dtype=torch.float64, device=device)
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            e2e_ms = float(t.item())
        e2e = {"value": world * n * args.e2e_steps / (e2e_ms / 1e3), "unit": "elems/s",
               "h2d_bytes_per_step": nbytes, "d2h_bytes_per_step": nbytes,
               "ms_per_step": e2e_ms / args.e2e_steps}
        del host, out, dev

    # eps sweep (one timed step each, one warm-up)
    sweep = {}
    for tok in [t for t in args.sweep.split(",") if t.strip()]:
        e_ = float(tok)
        p_ = pip.plan(n, dtype, e_, **opts)
        ms_ = time_steps(torch, pip, A, seed, e_, 1, 1, stream, opts)
        t_s = ms_[0] / 1e3
        ach = BYTES_PER_ELEM[dtype] * n / t_s / 1e9
        sweep[str(e_)] = {"value": n / t_s, "unit": "elems/s", "ms": ms_[0], "fresh_per_round": p_["fresh_per_round"],
                          "aux_bytes": p_["aux_bytes"], "aux_bound_bytes": p_["aux_bound_bytes"],
                          "roofline_frac": ach / measured_peak_hbm()[0]}

    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return 0

    peak, peak_kind = measured_peak_hbm()
    alg_bytes = BYTES_PER_ELEM[dtype] * n
    achieved = alg_bytes / (ms_per_step / 1e3) / 1e9
    traffic = recorded_traffic(n, dtype, eps)
    cpu = None
    if not args.no_cpu:
        v, dt = cpu_oracle_sample(dtype, seed, args.cpu_sample)
        cpu = {"value": v, "unit": "elems/s", "cores": 1, "kind": "oracle",
               "sample": f"sequential Knuth shuffle (oracle/knuth.c) of {args.cpu_sample} {dtype} elements A[i]=i, "
                         f"seed {seed}, one host thread, {dt:.1f} s"}
    line = {
        "metric": "shuffled elems/s",
        "value": value,
        "unit": "elems/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": ms_per_step,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": (value / world) / (n / (PAPER_RP_FINAL_1E9_MS / 1e3)) if (n == 10**9 and dtype == "u64") else None,
        "dtype": dtype,
        "data": "synthetic",
        "config": workload_config(args),
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                     "traffic": traffic, "peak_kind": peak_kind,
                     "algorithmic_bytes_per_elem": BYTES_PER_ELEM[dtype]},
        "cpu_baseline": cpu,
        "e2e": e2e,
        "gpu_launches": args.steps,
        "clocks": clocks,
        "plan": {k: plan[k] for k in ("fresh_per_round", "max_active", "slots", "grid_blocks", "block_threads",
                                      "aux_bytes", "aux_bound_bytes", "min_rounds")},
        "aux_alloc_delta_bytes": aux_delta,
        "rounds": st.rounds,
        "loser_fraction": st.losers / max(1, st.attempts),
        "eps_sweep": sweep,
        "step_ms": ms,
    }
    print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
