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
# Work queues from the host to the GPU, read when CUDA starts: the serving
# workload runs a stream per lane next to the tick stream, and streams beyond
# the queues (8 by default) would wait behind each other's launches.
os.environ.setdefault("CUDA_DEVICE_MAX_CONNECTIONS", "32")

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


def max_over_ranks(value: float, dist, device) -> float:
    """Maximum of a per-rank time over all ranks (identity without a process
    group).  Replicas run independently; only the timing is combined."""
    if dist is None:
        return value
    import torch

    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_throughput(n_per_rank: int, world: int, steps: int, max_ms: float) -> float:
    """Whole-job elements/s: every rank shuffled n_per_rank elements per step."""
    return world * n_per_rank * steps / (max_ms / 1e3)


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


def cpu_oracle_workload(kind: str, eps: float, seed: int, n_sample: int, dtype: str = "u64",
                        min_seconds: float = 5.0, max_reps: int = 10):
    """The oracle of a list, tree or scan workload, timed as it stands on one
    host thread over a bounded sample of the same shape (one random list, one
    random binary tree of n_sample leaves, or n_sample integers below 2^20).
    The oracle works in place, so it runs on a fresh copy of the one input
    each time (copies and input generation outside the timed region), until
    min_seconds of timed work or max_reps runs.  Returns the ``cpu_baseline``
    object."""
    import numpy as np

    import oracle
    import workloads

    oracle.build()
    if kind == "list":
        src = workloads.random_lists(n_sample, rng_seed=seed)
        run = oracle.list_contract
        units, unit = n_sample, "nodes/s"
        what = f"sequential splice in index order (oracle/listc.c) of one random list of {n_sample} nodes"
    elif kind == "tree":
        import paper_2103_01216_gb300 as pip

        src = workloads.random_tree(n_sample, rng_seed=seed)
        F = pip.tree_plan(src.shape[0], eps)["fresh_per_round"]
        run = lambda rec: oracle.tree_contract(rec, F, F * 5 // 2 + 2)  # noqa: E731
        units, unit = src.shape[0], "nodes/s"
        what = (f"round schedule (oracle/treec.c) of one random binary tree of {src.shape[0]} nodes, "
                f"F = {F}, eps {eps}")
    elif kind == "scan":
        npdt = np.uint32 if dtype == "u32" else np.uint64
        src = np.random.default_rng(seed).integers(0, 1 << 20, size=n_sample, dtype=npdt)
        run = oracle.scan_exclusive
        units, unit = n_sample, "elems/s"
        what = f"up-sweep / down-sweep recursion (oracle/scanc.c) of {n_sample} {dtype} values"
    else:
        raise ValueError(kind)
    total, reps = 0.0, 0
    while reps < max_reps and (reps == 0 or total < min_seconds):
        work = src.copy()
        t0 = time.perf_counter()
        run(work)
        total += time.perf_counter() - t0
        reps += 1
    return {"value": units * reps / total, "unit": unit, "cores": 1, "kind": "oracle",
            "sample": f"{what}, {reps} runs on copies of one input, one host thread, {total:.1f} s"}


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


def time_steps(torch, pip, A, seed, eps, steps, warmup, stream, opts, flush=None):
    """CUDA-event times of `steps` shuffles of A on `stream` after `warmup`
    untimed ones.  `flush` (a CUDA tensor larger than L2) is rewritten
    between timed steps, outside the timed region, for inputs that L2 holds."""
    for _ in range(warmup):
        pip.shuffle(A, seed=seed, eps=eps, stream=stream, **opts)
    pip.check(stream)
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    torch.cuda.synchronize()
    for s, e in evs:
        if flush is not None:
            with torch.cuda.stream(stream):
                flush.add_(1)
        s.record(stream)
        pip.shuffle(A, seed=seed, eps=eps, stream=stream, **opts)
        e.record(stream)
    pip.check(stream)
    torch.cuda.synchronize()
    return [s.elapsed_time(e) for s, e in evs]


def floor_ms(torch, pip, A, seed, stream, reps=3, mode=0):
    """Bare swap traffic of the same shuffle with no conflict resolution
    (pip_calibrate_swap_floor, which destroys A): the practical floor of the
    round drivers, with the random side as an exchange (mode 0) or a load and
    a store (mode 1)."""
    for _ in range(2):
        pip.calibrate_swap_floor(A, seed=seed, stream=stream, mode=mode)
    torch.cuda.synchronize()
    out = []
    for _ in range(reps):
        s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s.record(stream)
        pip.calibrate_swap_floor(A, seed=seed, stream=stream, mode=mode)
        e.record(stream)
        e.synchronize()
        out.append(s.elapsed_time(e))
    return min(out)


def cuda_runtime():
    """A CUDA runtime library for the default memory pool's counters (the
    pool is a driver object shared by every runtime in the process), or None."""
    import ctypes
    import ctypes.util
    import glob

    import torch

    cands = [ctypes.util.find_library("cudart")]
    for root in [os.path.dirname(torch.__file__), "/usr/local/cuda/lib64"]:
        cands += sorted(glob.glob(os.path.join(root, "**", "libcudart.so*"), recursive=True))
    for c in [c for c in cands if c]:
        try:
            return ctypes.CDLL(c)
        except OSError:
            continue
    return None


def pool_bytes(rt, device):
    """(reserved, used) bytes of the device's default memory pool."""
    import ctypes

    if rt is None:
        return None
    pool = ctypes.c_void_p()
    if rt.cudaDeviceGetDefaultMemPool(ctypes.byref(pool), device) != 0:
        return None
    out = []
    for attr in (5, 7):  # cudaMemPoolAttrReservedMemCurrent, cudaMemPoolAttrUsedMemCurrent
        v = ctypes.c_uint64()
        if rt.cudaMemPoolGetAttribute(pool, attr, ctypes.byref(v)) != 0:
            return None
        out.append(v.value)
    return tuple(out)


def aux_accounting(torch, pip, A, n, dtype, seed, eps, stream):
    """Scratch of one shuffle three ways: the plan's exact bytes against the
    c * n^(1-eps) bound; what the stream-ordered pool holds and what
    cudaMemGetInfo loses while a shuffle that allocates its own scratch runs;
    and the cudaMemGetInfo delta of a shuffle given caller scratch of exactly
    the planned size (the library then allocates nothing)."""
    dev = torch.cuda.current_device()
    rt = cuda_runtime()
    p = pip.plan(n, dtype, eps)
    torch.cuda.synchronize()
    pool_before = pool_bytes(rt, dev)
    free0, _ = torch.cuda.mem_get_info()
    pip.shuffle(A, seed=seed, eps=eps, stream=stream)
    free1, _ = torch.cuda.mem_get_info()
    pool_during = pool_bytes(rt, dev)
    pip.check(stream)
    aux = torch.empty(max(256, p["aux_bytes"]), dtype=torch.uint8, device=A.device)
    pip.shuffle(A, seed=seed, eps=eps, stream=stream, aux=aux)  # warm
    pip.check(stream)
    free2, _ = torch.cuda.mem_get_info()
    pip.shuffle(A, seed=seed, eps=eps, stream=stream, aux=aux)
    free3, _ = torch.cuda.mem_get_info()
    pip.check(stream)
    del aux
    return {"plan_aux_bytes": p["aux_bytes"], "plan_smem_bytes": p["smem_bytes"],
            "aux_bound_bytes": p["aux_bound_bytes"], "driver": p["driver"], "fresh_per_round": p["fresh_per_round"],
            "pool_reserved_during": None if pool_during is None else pool_during[0] - pool_before[0],
            "pool_used_during": None if pool_during is None else pool_during[1] - pool_before[1],
            "mem_get_info_delta_pool": max(0, free0 - free1),
            "mem_get_info_delta_caller_scratch": free2 - free3}


def batch_case(torch, pip, count, steps, warmup, plain_steps, bopts):
    """Batched workload: `count` uint32 arrays A[i]=i, sizes log-uniform in
    [2^8, 2^22] (stream seed 7), per-array seed = index, eps = 0.5.  One
    launch (and its CUDA-graph replay) against one pip_shuffle per array.
    Returns the measurements as a dict."""
    import numpy as np

    import workloads

    sizes, seeds = workloads.batch_workload(count=count)
    offs = np.zeros(len(sizes) + 1, dtype=np.int64)
    offs[1:] = np.cumsum((sizes + 3) // 4 * 4)  # 16-byte aligned arrays in one buffer
    buf = torch.empty(int(offs[-1]), dtype=torch.int32, device="cuda")
    arrays = [buf[int(offs[j]):int(offs[j]) + int(sizes[j])] for j in range(len(sizes))]
    for a in arrays:
        a.copy_(torch.arange(a.shape[0], dtype=torch.int32, device="cuda"))
    total = int(sizes.sum())
    eps = 0.5
    b = pip.Batch(arrays, [int(x) for x in seeds], eps=eps, **bopts)
    stream = torch.cuda.current_stream()
    for _ in range(warmup):
        b.run()
    pip.check()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    with ClockSampler(torch.cuda.current_device()) as clk:
        for s_, e_ in ev:
            s_.record(stream)
            b.run()
            e_.record(stream)
        pip.check()
    batched_ms = [s_.elapsed_time(e_) for s_, e_ in ev]
    # the same launch captured once and replayed
    g = torch.cuda.CUDAGraph()
    side = torch.cuda.Stream()
    side.wait_stream(stream)
    with torch.cuda.stream(side):
        b.run(stream=side)
    side.synchronize()
    with torch.cuda.graph(g, stream=side):
        b.run(stream=side)
    g.replay()
    torch.cuda.synchronize()
    gs, ge = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    gs.record()
    for _ in range(steps):
        g.replay()
    ge.record()
    torch.cuda.synchronize()
    pip.check()
    graph_ms = gs.elapsed_time(ge) / steps
    del g
    # plain path: one launch per array, FIFO on one stream
    plain_ms = []
    for _ in range(plain_steps):
        ps, pe = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ps.record()
        for a, sd in zip(arrays, seeds):
            pip.shuffle(a, seed=int(sd), eps=eps)
        pe.record()
        pip.check()
        plain_ms.append(ps.elapsed_time(pe))
    # identical output: a sample of arrays through both paths from A[i] = i
    chk = [j for j in range(0, len(sizes), max(1, len(sizes) // 64))]
    ref = [torch.arange(int(sizes[j]), dtype=torch.int32, device="cuda") for j in chk]
    bb = [torch.arange(int(sizes[j]), dtype=torch.int32, device="cuda") for j in chk]
    pip.Batch(bb, [int(seeds[j]) for j in chk], eps=eps).run()
    for r_, j in zip(ref, chk):
        pip.shuffle(r_, seed=int(seeds[j]), eps=eps)
    pip.check()
    identical = all(bool(torch.equal(x, y)) for x, y in zip(ref, bb))
    bms = sum(batched_ms) / len(batched_ms)
    pms = sum(plain_ms) / len(plain_ms) if plain_ms else float("nan")
    out = {
        "workload": f"batch_{len(sizes)}_u32_log_uniform_2^8_2^22_seed7_eps0.5", "arrays": len(sizes),
        "total_elems": total, "fmax": b.plan.fmax, "block_threads": b.plan.block_threads,
        "ms_per_step": bms, "value": total / (bms / 1e3), "unit": "elems/s",
        "graph_ms_per_step": graph_ms, "graph_value": total / (graph_ms / 1e3),
        "plain": {"ms_per_step": pms, "value": total / (pms / 1e3), "launches_per_step": len(sizes),
                  "path": "pip_shuffle per array, FIFO on one stream"},
        "speedup_vs_plain": pms / bms, "graph_speedup_vs_plain": pms / graph_ms,
        "identical_output_sample": identical, "steps": steps, "warmup": warmup,
        "clocks": clk.summary(), "step_ms": batched_ms,
    }
    del arrays, buf, b
    torch.cuda.empty_cache()
    return out


def run_batch(args):
    import torch

    import paper_2103_01216_gb300 as pip
    from paper_2103_01216_gb300 import _build

    _build.build()
    torch.cuda.set_device(0)
    bopts = {}
    if args.block_threads:
        bopts["block_threads"] = args.block_threads
    if args.prefix_c:
        bopts["prefix_c"] = args.prefix_c
    if args.flags:
        bopts["flags"] = args.flags
    r = batch_case(torch, pip, args.batch_count, args.steps, args.warmup, args.plain_steps, bopts)
    line = {
        "metric": "shuffled elems/s (batched, 8192 arrays)",
        "value": r["value"],
        "unit": "elems/s",
        "n_gpus": 1,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": r["ms_per_step"],
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "u32",
        "data": "synthetic",
        "config": {"workload": r["workload"], "arrays": r["arrays"], "total_elems": r["total_elems"],
                   "fmax": r["fmax"], "block_threads": r["block_threads"], "l2": "inputs larger than L2 (no flush)"},
        **{k: r[k] for k in ("graph_ms_per_step", "graph_value", "plain", "speedup_vs_plain",
                             "graph_speedup_vs_plain", "identical_output_sample", "clocks", "step_ms")},
        "gpu_launches": args.steps,
    }
    print(json.dumps(line), flush=True)
    return 0


def run_floor(args):
    """The bare swap traffic of the workload (pip_calibrate_swap_floor): the
    n-1 swaps with no conflict resolution, timed like a shuffle step."""
    import torch

    import paper_2103_01216_gb300 as pip
    from paper_2103_01216_gb300 import _build

    _build.build()
    torch.cuda.set_device(0)
    A = make_device_input(torch, args.n, args.dtype, "cuda")
    stream = torch.cuda.current_stream()
    f = floor_ms(torch, pip, A, args.seed, stream, reps=max(1, args.steps), mode=pip.FLOOR_EXCHANGE)
    fl = floor_ms(torch, pip, A, args.seed, stream, reps=max(1, args.steps), mode=pip.FLOOR_LOADSTORE)
    print(json.dumps({"metric": "bare swap floor", "value": args.n / (f / 1e3), "unit": "swaps/s", "ms": f,
                      "loadstore_ms": fl, "n": args.n, "dtype": args.dtype,
                      "bytes_algorithmic_per_swap": BYTES_PER_ELEM[args.dtype]}),
          flush=True)
    return 0


LIST_BYTES_PER_NODE = 144  # own 16-byte record read, two random 8-byte writes (32-B sector read + written each)
PAPER_LIST_PIP_200M_MS = 418.0  # PIP list contraction, 200M nodes, 72 cores + HT (Table "lt-runtime")


def run_list(args):
    """List contraction (Section 4.2, Algorithm 2): n nodes of two 64-bit
    pointers forming one random doubly-linked list (the paper's workload
    shape, 10 to 200 million nodes), node i contracting once both current
    neighbours are larger.  The list is rebuilt before every step (outside the
    timed region) because contraction consumes it; the order comes from
    torch.randperm with a fixed seed, and the output of the last step is
    checked on a sample against the nearest-larger definition."""
    import torch

    import paper_2103_01216_gb300 as pip
    from paper_2103_01216_gb300 import _build

    _build.build()
    torch.cuda.set_device(0)
    n, eps = args.n, args.eps
    gen = torch.Generator(device="cuda")
    gen.manual_seed(args.seed)
    order = torch.randperm(n, device="cuda", generator=gen)
    base = torch.full((n, 2), -1, dtype=torch.int64, device="cuda")
    base[order[1:], 0] = order[:-1]
    base[order[:-1], 1] = order[1:]
    nodes = torch.empty_like(base)
    opts = {}
    if args.fresh:
        opts["fresh_per_round"] = args.fresh
    if args.block_threads:
        opts["block_threads"] = args.block_threads
    if args.grid_blocks:
        opts["grid_blocks"] = args.grid_blocks
    plan = pip.list_plan(n, eps, **opts)
    stream = torch.cuda.current_stream()
    for _ in range(args.warmup):
        nodes.copy_(base)
        pip.list_contract(nodes, eps=eps, **opts)
    pip.check()
    times = []
    with ClockSampler(torch.cuda.current_device()) as clk:
        for _ in range(args.steps):
            nodes.copy_(base)
            s_, e_ = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            s_.record(stream)
            pip.list_contract(nodes, eps=eps, **opts)
            e_.record(stream)
            e_.synchronize()
            times.append(s_.elapsed_time(e_))
    pip.check()
    st_buf = torch.zeros(pip.STATS_BYTES, dtype=torch.uint8, device="cuda")
    nodes.copy_(base)
    pip.list_contract(nodes, eps=eps, stats=st_buf, **opts)
    pip.check()
    st = pip.read_stats(st_buf)
    # sampled check: every neighbour at contraction is larger, and one node per
    # list (the maximum) is left with none
    out = nodes[::max(1, n // 100000)].cpu()
    idx = torch.arange(0, n, max(1, n // 100000))
    ok_larger = bool(torch.all((out == -1) | (out > idx[:, None])))
    ms = sorted(times)[len(times) // 2]
    # list ranking (contraction with link weights, then the reconstruction
    # step) on the same list: the k-th node of the visiting order has k nodes
    # before it, checked on a sample
    rank_times = []
    for k in range(args.warmup + args.steps):
        nodes.copy_(base)
        s_, e_ = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s_.record(stream)
        pip.list_rank(nodes, eps=eps, **opts)
        e_.record(stream)
        e_.synchronize()
        if k >= args.warmup:
            rank_times.append(s_.elapsed_time(e_))
    pip.check()
    ks = torch.arange(0, n, max(1, n // 100000), device="cuda")
    got = nodes[order[ks]]
    rank_ok = bool(torch.equal(got[:, 0], ks) and torch.equal(got[:, 1], n - 1 - ks))
    rms = sorted(rank_times)[len(rank_times) // 2]
    ranking = {"ms": rms, "value": n / (rms / 1e3), "unit": "ranked nodes/s", "step_ms": rank_times,
               "sample_check": rank_ok,
               "what": "pip_list_rank: weighted contraction, then the reconstruction rounds from the largest index "
                       "down; record i ends as (nodes before i, nodes after i)"}
    ach = LIST_BYTES_PER_NODE * n / (ms / 1e3) / 1e9
    peak, peak_kind = measured_peak_hbm()
    line = {
        "metric": "contracted list nodes/s", "value": n / (ms / 1e3), "unit": "nodes/s", "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u64", "data": "synthetic",
        "config": {"workload": f"list_contraction_n{n}_one_random_list_eps{eps}", "n": n, "eps": eps,
                   "record": "2 x 64-bit pointers", "l2": "inputs larger than L2 (no flush)"},
        "roofline": {"bound": "hbm", "achieved": ach, "peak": peak, "unit": "GB/s", "frac": ach / peak,
                     "traffic": None, "peak_kind": peak_kind, "algorithmic_bytes_per_node": LIST_BYTES_PER_NODE},
        "plan": {k: plan[k] for k in ("fresh_per_round", "max_active", "grid_blocks", "block_threads", "aux_bytes",
                                      "smem_bytes", "aux_bound_bytes", "min_rounds")},
        "rounds": st.rounds, "carried_fraction": st.losers / max(1, st.attempts),
        "sample_check": ok_larger,
        "list_ranking": ranking,
        "paper_context": {"pip_72cores_ht_200M_ms": PAPER_LIST_PIP_200M_MS},
        "gpu_launches": args.steps, "clocks": clk.summary(), "step_ms": times,
    }
    if not args.no_cpu:
        line["cpu_baseline"] = cpu_oracle_workload("list", eps, args.seed, min(n, 1 << 25))
    print(json.dumps(line), flush=True)
    return 0


# one rake touches the 32-B sectors of its leaf, parent, sibling and
# grandparent (read) and writes three of them; an internal node is read once
# when admitted: (4 + 3) * 32 + 32 bytes per leaf-internal pair
TREE_BYTES_PER_NODE = 128
PAPER_TREE_PIP_200M_MS = 680.0  # PIP tree contraction, 200M entries, 72 cores + HT (Table "lt-runtime")


def _random_tree_on_device(leaves, seed):
    """The bench's forest on the GPU: one random binary tree over ``leaves``
    leaves built bottom-up (the current roots shuffled by torch.randperm and
    joined in pairs, level after level, depth about log2 of the leaves), then
    every node id renamed by a uniform permutation -- the construction of
    workloads.random_tree, drawn with torch's generator."""
    import torch

    dev = "cuda"
    gen = torch.Generator(device=dev)
    gen.manual_seed(seed)
    n = 2 * leaves - 1
    par = torch.full((n,), -1, dtype=torch.int64, device=dev)
    lft = torch.full((n,), -1, dtype=torch.int64, device=dev)
    rgt = torch.full((n,), -1, dtype=torch.int64, device=dev)
    roots = torch.arange(leaves, dtype=torch.int64, device=dev)
    nxt = leaves
    while roots.numel() > 1:
        roots = roots[torch.randperm(roots.numel(), device=dev, generator=gen)]
        k = roots.numel() // 2
        new = torch.arange(nxt, nxt + k, dtype=torch.int64, device=dev)
        nxt += k
        lft[new] = roots[:k]
        rgt[new] = roots[k:2 * k]
        par[roots[:k]] = new
        par[roots[k:2 * k]] = new
        roots = torch.cat([new, roots[2 * k:]])
    perm = torch.randperm(n, device=dev, generator=gen)

    def ren(a):
        return torch.where(a >= 0, perm[a.clamp(min=0)], a)

    rec = torch.empty((n, 4), dtype=torch.int64, device=dev)
    rec[perm, 0] = ren(par)
    rec[perm, 1] = ren(lft)
    rec[perm, 2] = ren(rgt)
    rec[:, 3] = 0
    del par, lft, rgt, perm, roots
    return rec


def run_tree(args):
    """Tree contraction (Section 4.2): a random binary tree of n = 2L - 1
    nodes of 32 bytes (the paper's inputs hold 10 to 200 million entries),
    contracted by rounds over a prefix of the nodes.  The tree is restored
    before every step (outside the timed region) because contraction
    consumes it; the last step's output is checked on a sample: each sampled
    raked leaf's parent still lists the leaf and the recorded sibling as its
    children, and one leaf is left as the root."""
    import torch

    import paper_2103_01216_gb300 as pip
    from paper_2103_01216_gb300 import _build

    _build.build()
    torch.cuda.set_device(0)
    leaves, eps = args.n, args.eps
    base = _random_tree_on_device(leaves, args.seed)
    n = base.shape[0]
    nodes = torch.empty_like(base)
    opts = {}
    if args.fresh:
        opts["fresh_per_round"] = args.fresh
    if args.block_threads:
        opts["block_threads"] = args.block_threads
    if args.grid_blocks:
        opts["grid_blocks"] = args.grid_blocks
    plan = pip.tree_plan(n, eps, **opts)
    stream = torch.cuda.current_stream()
    for _ in range(args.warmup):
        nodes.copy_(base)
        pip.tree_contract(nodes, eps=eps, **opts)
    pip.check()
    times = []
    with ClockSampler(torch.cuda.current_device()) as clk:
        for _ in range(args.steps):
            nodes.copy_(base)
            s_, e_ = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            s_.record(stream)
            pip.tree_contract(nodes, eps=eps, **opts)
            e_.record(stream)
            e_.synchronize()
            times.append(s_.elapsed_time(e_))
    pip.check()
    st_buf = torch.zeros(pip.STATS_BYTES, dtype=torch.uint8, device="cuda")
    nodes.copy_(base)
    pip.tree_contract(nodes, eps=eps, stats=st_buf, **opts)
    pip.check()
    st = pip.read_stats(st_buf)
    leaf = base[:, 1] < 0
    raked = leaf & (nodes[:, 1] >= 0)
    idx = torch.nonzero(raked).flatten()
    idx = idx[::max(1, idx.numel() // 100000)]
    p, s_ = nodes[idx, 0], nodes[idx, 1]
    kids = nodes[p][:, 1:3]
    ok = bool(torch.all(((kids[:, 0] == idx) & (kids[:, 1] == s_)) | ((kids[:, 1] == idx) & (kids[:, 0] == s_))))
    ok = ok and int((leaf & ~raked).sum()) == 1 and int(raked.sum()) == leaves - 1
    ms = sorted(times)[len(times) // 2]
    ach = TREE_BYTES_PER_NODE * n / (ms / 1e3) / 1e9
    peak, peak_kind = measured_peak_hbm()
    line = {
        "metric": "contracted tree nodes/s", "value": n / (ms / 1e3), "unit": "nodes/s", "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u64", "data": "synthetic",
        "config": {"workload": f"tree_contraction_n{n}_one_random_binary_tree_eps{eps}", "n": n, "leaves": leaves,
                   "eps": eps, "record": "4 x 64-bit words (parent, left, right, round)",
                   "l2": "inputs larger than L2 (no flush)"},
        "roofline": {"bound": "hbm", "achieved": ach, "peak": peak, "unit": "GB/s", "frac": ach / peak,
                     "traffic": None, "peak_kind": peak_kind, "algorithmic_bytes_per_node": TREE_BYTES_PER_NODE},
        "plan": {k: plan[k] for k in ("fresh_per_round", "max_active", "grid_blocks", "block_threads", "aux_bytes",
                                      "smem_bytes", "aux_bound_bytes", "min_rounds")},
        "rounds": st.rounds, "carried_fraction": st.losers / max(1, st.attempts),
        "sample_check": ok,
        "paper_context": {"pip_72cores_ht_200M_ms": PAPER_TREE_PIP_200M_MS},
        "gpu_launches": args.steps, "clocks": clk.summary(), "step_ms": times,
    }
    if not args.no_cpu:
        line["cpu_baseline"] = cpu_oracle_workload("tree", eps, args.seed, min(leaves, 1 << 23))
    print(json.dumps(line), flush=True)
    return 0


SCAN_BYTES_PER_ELEM = {"u32": 8, "u64": 16}  # each element read once and written once


def run_scan(args):
    """In-place exclusive scan (Section 5.1) of n unsigned integers (the
    paper's scan input is 10^9 integers), values below 2^20 from a fixed
    seed; each step scans the previous step's output (an equally valid
    input).  Bound by HBM bandwidth: 2 x element bytes per element."""
    import torch

    import paper_2103_01216_gb300 as pip
    from paper_2103_01216_gb300 import _build

    _build.build()
    torch.cuda.set_device(0)
    n, dt = args.n, ("u32" if args.dtype == "u32" else "u64")
    tdt = torch.int32 if dt == "u32" else torch.int64
    gen = torch.Generator(device="cuda")
    gen.manual_seed(args.seed)
    A = torch.randint(0, 1 << 20, (n,), dtype=tdt, device="cuda", generator=gen)
    tot = torch.zeros(1, dtype=tdt, device="cuda")
    aux = torch.empty(pip.scan_aux_bytes(), dtype=torch.uint8, device="cuda")
    stream = torch.cuda.current_stream()
    for _ in range(args.warmup):
        pip.scan(A, total=tot, aux=aux)
    pip.check()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    with ClockSampler(torch.cuda.current_device()) as clk:
        for s_, e_ in evs:
            s_.record(stream)
            pip.scan(A, total=tot, aux=aux)
            e_.record(stream)
        pip.check()
    times = [s_.elapsed_time(e_) for s_, e_ in evs]
    ms = sorted(times)[len(times) // 2]
    ach = SCAN_BYTES_PER_ELEM[dt] * n / (ms / 1e3) / 1e9
    peak, peak_kind = measured_peak_hbm()
    line = {
        "metric": "scanned elems/s", "value": n / (ms / 1e3), "unit": "elems/s", "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": dt, "data": "synthetic",
        "config": {"workload": f"inplace_exclusive_scan_n{n}_{dt}", "n": n, "l2": "inputs larger than L2 (no flush)"},
        "roofline": {"bound": "hbm", "achieved": ach, "peak": peak, "unit": "GB/s", "frac": ach / peak,
                     "traffic": None, "peak_kind": peak_kind,
                     "algorithmic_bytes_per_elem": SCAN_BYTES_PER_ELEM[dt]},
        "aux_bytes": pip.scan_aux_bytes(), "gpu_launches": args.steps, "clocks": clk.summary(), "step_ms": times,
    }
    if not args.no_cpu:
        line["cpu_baseline"] = cpu_oracle_workload("scan", 0.0, args.seed, min(n, 1 << 28), dt)
    print(json.dumps(line), flush=True)
    return 0


def _percentile(xs, q):
    xs = sorted(xs)
    if not xs:
        return None
    k = min(len(xs) - 1, max(0, int(round(q / 100.0 * (len(xs) - 1)))))
    return xs[k]


def serve_case(torch, pip, N, opts, plain_N, plain_open=False):
    """Served workload: the first N of the 20,000-request stream -- sizes
    log-uniform in [2^12, 2^28] (stream 5), uint32/uint64 by a seeded coin,
    seed = request id, eps = 0.5 -- under a 120 GB device budget.  Closed
    loop first (saturation throughput), then Poisson arrivals at 80 % of it.
    The plain FIFO path (allocate, initialise, pip_shuffle, synchronize, one
    request at a time) runs back to back over the first plain_N requests of
    the same stream (its saturation), and with plain_open also on their
    arrival schedule.  Throughputs are compared per element, since the
    plain path's prefix has its own size mix."""
    import threading as th

    import workloads

    sizes_all, dtypes_all, seeds_all, _ = workloads.serve_workload(count=20000)
    sizes, dtypes, seeds = sizes_all[:N], dtypes_all[:N], seeds_all[:N]
    total = int(sizes.sum())
    budget = 120 * 10**9
    eps = 0.5

    def closed_loop(k):
        with pip.Server(budget, **opts) as srv:
            t0 = time.perf_counter()
            for n, d, sd in zip(sizes[:k], dtypes[:k], seeds[:k]):
                srv.submit(int(n), str(d), seed=int(sd), eps=eps)
            for _ in range(k):  # release each request as soon as it finishes
                srv.release(srv.next_done())
            dt = time.perf_counter() - t0
            info = srv.info()
        return dt, info

    closed_loop(min(N, 200))  # warm-up (kernel attributes, pools)
    with ClockSampler(torch.cuda.current_device()) as clk:
        t_sat, info_sat = closed_loop(N)
    rate = 0.8 * N / t_sat
    _, _, _, arrivals = workloads.serve_workload(count=20000, rate_per_s=rate)
    arrivals = arrivals[:N]

    # open loop through the server
    lat, done_at = [], []
    with pip.Server(budget, **opts) as srv:
        tickets = []
        start = time.perf_counter()
        start_ns = time.monotonic_ns()

        def submitter():
            for j in range(N):
                delay = arrivals[j] - (time.perf_counter() - start)
                if delay > 0:
                    time.sleep(delay)
                tickets.append(srv.submit(int(sizes[j]), str(dtypes[j]), seed=int(seeds[j]), eps=eps))

        thr = th.Thread(target=submitter)
        thr.start()
        for _ in range(N):  # completion order: each request is released as soon as it is done
            t = srv.next_done()
            _, st = srv.poll(t)
            lat.append((st.done_ns - st.submit_ns) / 1e6)
            done_at.append(st.done_ns)
            srv.release(t)
        thr.join()
        served_span = (max(done_at) - start_ns) / 1e9
        info = srv.info()

    def plain_one(j):
        n = int(sizes_all[j])
        A = torch.arange(n, dtype=torch.int64 if dtypes_all[j] == "u64" else torch.int32, device="cuda")
        pip.shuffle(A, seed=int(seeds_all[j]), eps=eps)
        torch.cuda.synchronize()
        del A

    plain = {"requests": plain_N, "path": "allocate, initialise, pip_shuffle, synchronize; one request at a time"}
    if plain_N > 0:
        plain_total = int(sizes_all[:plain_N].sum())
        t1 = time.perf_counter()
        for j in range(plain_N):
            plain_one(j)
        plain_sat = time.perf_counter() - t1
        plain.update({"total_elems": plain_total, "saturation_req_s": plain_N / plain_sat,
                      "saturation_elems_s": plain_total / plain_sat})
        if plain_open:
            plain_lat = []
            t0 = time.perf_counter()
            for j in range(plain_N):
                delay = arrivals[j] - (time.perf_counter() - t0)
                if delay > 0:
                    time.sleep(delay)
                plain_one(j)
                plain_lat.append((time.perf_counter() - t0 - arrivals[j]) * 1e3)
            plain.update({"p50_ms": _percentile(plain_lat, 50), "p99_ms": _percentile(plain_lat, 99),
                          "throughput_req_s": plain_N / (time.perf_counter() - t0)})
        torch.cuda.empty_cache()
    served = {"requests": N, "total_elems": total, "p50_ms": _percentile(lat, 50), "p99_ms": _percentile(lat, 99),
              "throughput_req_s": N / served_span, "elems_s": total / served_span,
              "saturation_req_s": N / t_sat, "saturation_elems_s": total / t_sat,
              "arrival_rate_per_s": rate, "peak_used_bytes": info.peak_used_bytes, "ticks": info.ticks,
              "lane_requests": info.lane_requests, "clocks": clk.summary()}
    out = {"workload": f"serve_{N}_of_20000_requests_log_uniform_2^12_2^28_u32_u64_eps0.5_budget120GB",
           "served": served, "plain_fifo": plain, "options": dict(opts)}
    if plain.get("saturation_elems_s"):
        out["speedup_saturation_elems"] = served["saturation_elems_s"] / plain["saturation_elems_s"]
    return out


def run_serve(args):
    import torch

    import paper_2103_01216_gb300 as pip
    from paper_2103_01216_gb300 import _build

    _build.build()
    torch.cuda.set_device(0)
    opts = dict(rounds_per_tick=args.rounds_per_tick, fresh_cap=args.fresh_cap, tick_us=args.tick_us)
    N = args.requests
    r = serve_case(torch, pip, N, opts, 0 if args.no_plain else min(N, args.plain_requests),
                   plain_open=not args.no_plain)
    line = {
        "metric": "served requests/s and p50/p99 latency vs FIFO plain path",
        "value": r["served"]["throughput_req_s"],
        "unit": "requests/s",
        "n_gpus": 1,
        "steps": 1,
        "warmup": 1,
        "ms_per_step": r["served"]["requests"] / r["served"]["throughput_req_s"] * 1e3,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "u32/u64",
        "data": "synthetic",
        "config": {"workload": r["workload"], "requests": N, **opts},
        **{k: v for k, v in r.items() if k not in ("workload",)},
    }
    print(json.dumps(line), flush=True)
    return 0


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
    ap.add_argument("--e2e-steps", type=int, default=16)
    ap.add_argument("--cpu-sample", type=int, default=1 << 27, help="elements in the oracle's timed sample")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--prefix-c", type=float, default=0.0)
    ap.add_argument("--fresh", type=int, default=0)
    ap.add_argument("--slot-factor", type=int, default=0)
    ap.add_argument("--grid-blocks", type=int, default=0)
    ap.add_argument("--block-threads", type=int, default=0)
    ap.add_argument("--flags", type=int, default=0, help="PIP_FLAG_* bits (2 = L2 prefetch of the next block)")
    ap.add_argument("--workload", default="single",
                    choices=["single", "batch", "serve", "floor", "list", "tree", "scan"])
    ap.add_argument("--batch-count", type=int, default=8192)
    ap.add_argument("--plain-steps", type=int, default=1)
    ap.add_argument("--requests", type=int, default=20000)
    ap.add_argument("--plain-requests", type=int, default=2000,
                    help="serve: requests of the stream's prefix timed through the plain FIFO path")
    ap.add_argument("--rounds-per-tick", type=int, default=0)
    ap.add_argument("--tick-us", type=int, default=0)
    ap.add_argument("--fresh-cap", type=int, default=1024)
    ap.add_argument("--no-floor", action="store_true")
    ap.add_argument("--no-rules", dest="rules", action="store_false",
                    help="skip the two-reservation rule ablation step")
    ap.add_argument("--no-plain", action="store_true", help="serve: skip the plain FIFO comparison")
    ap.add_argument("--no-configs", dest="configs", action="store_false",
                    help="single workload: skip the other configurations (records, batch, serving, 2^20)")
    args = ap.parse_args()

    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "batch":
        return run_batch(args)
    if args.workload == "serve":
        return run_serve(args)
    if args.workload == "floor":
        return run_floor(args)
    if args.workload == "scan":
        return run_scan(args)
    if args.workload == "list":
        if args.n == 10**9:
            args.n = 2 * 10**8  # the paper's largest list
        return run_list(args)
    if args.workload == "tree":
        if args.n == 10**9:
            args.n = 10**8  # leaves: 2 * 10^8 - 1 nodes, the paper's largest tree input
        return run_tree(args)

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
    with ClockSampler(torch.cuda.current_device()) as clk:
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()
        ms = time_steps(torch, pip, A, seed, eps, args.steps, args.warmup, stream, opts)
        torch.cuda.synchronize()
    clocks = clk.summary()
    total_ms = max_over_ranks(sum(ms), dist, device)
    ms_per_step = total_ms / args.steps
    value = replica_throughput(n, world, args.steps, total_ms)

    # scratch accounting: the plan, the stream-ordered pool while a shuffle
    # runs, and caller-provided scratch (where nothing is allocated)
    aux = {str(eps): aux_accounting(torch, pip, A, n, dtype, seed, eps, stream)}

    # stats of one run
    st_buf = torch.zeros(pip.STATS_BYTES, dtype=torch.uint8, device=device)
    pip.shuffle(A, seed=seed, eps=eps, stats=st_buf, **opts)
    pip.check()
    st = pip.read_stats(st_buf)

    # end to end through the host-memory entry point (pip_shuffle_host_stream):
    # every step copies its input from pinned host memory to the device,
    # shuffles it and copies the result back to pinned host memory; the
    # copies of one step overlap the shuffles of its neighbours.  The copy
    # stages are then timed alone on the same buffers.
    e2e = None
    if args.e2e_steps > 0:
        host = A.cpu().pin_memory()
        out = torch.empty(host.shape, dtype=host.dtype, pin_memory=True)
        nbytes = host.numel() * host.element_size()
        slot = (nbytes + 255) // 256 * 256
        buf = torch.empty(4 * slot, dtype=torch.uint8, device=device)
        pip.shuffle_host_stream([host] * 4, [out] * 4, [seed] * 4, eps=eps, dev_buf=buf)
        pip.check()
        s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        if dist is not None:
            dist.barrier()
        s.record()
        pip.shuffle_host_stream([host] * args.e2e_steps, [out] * args.e2e_steps, [seed] * args.e2e_steps,
                                eps=eps, dev_buf=buf)
        e.record()
        pip.check()
        e2e_ms = max_over_ranks(s.elapsed_time(e), dist, device)
        hv, ov = host.view(-1).view(torch.uint8), out.view(-1).view(torch.uint8)
        d0, d1 = buf[:nbytes], buf[slot:slot + nbytes]
        s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()

        def stage(fn):
            torch.cuda.synchronize()
            a_, b_ = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a_.record()
            fn()
            b_.record()
            torch.cuda.synchronize()
            return a_.elapsed_time(b_)

        def h2d():
            with torch.cuda.stream(s1):
                d0.copy_(hv, non_blocking=True)
            torch.cuda.current_stream().wait_stream(s1)

        def d2h():
            with torch.cuda.stream(s2):
                ov.copy_(d1, non_blocking=True)
            torch.cuda.current_stream().wait_stream(s2)

        def both():
            h2d()
            d2h()

        h2d_ms, d2h_ms, both_ms = stage(h2d), stage(d2h), stage(both)
        # one shuffle (of the third buffer, a valid array) while both copies run
        s3 = torch.cuda.Stream()
        d2 = buf[2 * slot:2 * slot + nbytes].view(torch.int64 if dtype != "u32" else torch.int32)
        if dtype == "rec128":
            d2 = d2.view(-1, 2)
        torch.cuda.synchronize()
        a3, b3 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ce = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
        with torch.cuda.stream(s1):
            ce[0].record(s1)
            d0.copy_(hv, non_blocking=True)
            ce[1].record(s1)
        with torch.cuda.stream(s2):
            ce[2].record(s2)
            ov.copy_(d1, non_blocking=True)
            ce[3].record(s2)
        a3.record(s3)
        pip.shuffle(d2, seed=seed, eps=eps, stream=s3, **opts)
        b3.record(s3)
        torch.cuda.synchronize()
        pip.check(s3)
        under_ms = a3.elapsed_time(b3)
        # the two copies while that shuffle runs (the shuffle's random traffic
        # shares HBM with them)
        copies_under_ms = max(ce[0].elapsed_time(ce[1]), ce[2].elapsed_time(ce[3]))
        k = args.e2e_steps
        # steady state: no stage runs faster than it does alone, the two
        # copies together no faster than measured together, and neither the
        # shuffle nor the copies faster than when they ran at once
        model = (h2d_ms + d2h_ms + k * max(under_ms, copies_under_ms, both_ms, h2d_ms, d2h_ms)) / k
        e2e = {"value": replica_throughput(n, world, k, e2e_ms), "unit": "elems/s",
               "h2d_bytes_per_step": nbytes, "d2h_bytes_per_step": nbytes,
               "ms_per_step": e2e_ms / k, "steps": k,
               "api": "pip_shuffle_host_stream (pinned host buffers, copies overlapped with neighbouring shuffles)",
               "stages": {"h2d_ms": h2d_ms, "d2h_ms": d2h_ms, "h2d_and_d2h_together_ms": both_ms,
                          "shuffle_ms": ms_per_step, "shuffle_while_copying_ms": under_ms,
                          "copies_while_shuffling_ms": copies_under_ms,
                          "h2d_GB_s": nbytes / h2d_ms / 1e6,
                          "d2h_GB_s": nbytes / d2h_ms / 1e6,
                          "model_ms_per_step": model,
                          "model": "(h2d + d2h + steps * max(shuffle while copying, copies while shuffling, "
                                   "h2d and d2h together, h2d, d2h)) / steps: the first copy in and the last "
                                   "copy out are not overlapped"}}
        del host, out, buf, hv, ov, d0, d1, d2

    # eps sweep (one timed step each, one warm-up) and its scratch accounting
    sweep = {}
    for tok in [t for t in args.sweep.split(",") if t.strip()]:
        e_ = float(tok)
        p_ = pip.plan(n, dtype, e_, **opts)
        ms_ = time_steps(torch, pip, A, seed, e_, 1, 1, stream, opts)
        t_s = ms_[0] / 1e3
        ach = BYTES_PER_ELEM[dtype] * n / t_s / 1e9
        sweep[str(e_)] = {"value": n / t_s, "unit": "elems/s", "ms": ms_[0], "fresh_per_round": p_["fresh_per_round"],
                          "driver": p_["driver"], "aux_bytes": p_["aux_bytes"], "smem_bytes": p_["smem_bytes"],
                          "aux_bound_bytes": p_["aux_bound_bytes"], "roofline_frac": ach / measured_peak_hbm()[0]}
        if ms_[0] < 1000.0:
            aux[str(e_)] = aux_accounting(torch, pip, A, n, dtype, seed, e_, stream)

    # reservation-rule ablation (Algorithm 1 as printed: two reservations per
    # step, against the one-reservation rule of the default path), one step
    rules = None
    if args.rules:
        o2 = dict(opts)
        o2["flags"] = o2.get("flags", 0) | pip.FLAG_TWO_RES
        ms2 = time_steps(torch, pip, A, seed, eps, 1, 1, stream, o2)
        st2 = torch.zeros(pip.STATS_BYTES, dtype=torch.uint8, device=device)
        pip.shuffle(A, seed=seed, eps=eps, stats=st2, **o2)
        pip.check()
        s2 = pip.read_stats(st2)
        rules = {"two_reservation": {"ms": ms2[0], "value": n / (ms2[0] / 1e3), "rounds": s2.rounds,
                                     "loser_fraction": s2.losers / max(1, s2.attempts)},
                 "one_reservation": {"ms": ms_per_step, "value": value, "rounds": st.rounds,
                                     "loser_fraction": st.losers / max(1, st.attempts)}}

    # commit-mode ablation: the planner's mode against the other one, one step
    modes = None
    if args.rules:
        other = pip.FLAG_SWAP_LOADSTORE if plan["flags"] & pip.FLAG_SWAP_EXCHANGE else pip.FLAG_SWAP_EXCHANGE
        o3 = dict(opts)
        o3["flags"] = o3.get("flags", 0) | other
        ms3 = time_steps(torch, pip, A, seed, eps, 1, 1, stream, o3)
        name = lambda f: "exchange" if f & pip.FLAG_SWAP_EXCHANGE else "loadstore"  # noqa: E731
        modes = {"planned": name(plan["flags"]), name(plan["flags"]): ms_per_step,
                 name(pip.plan(n, dtype, eps, **o3)["flags"]): ms3[0]}

    # bare swap traffic of the same shuffle (destroys A; nothing reads it after)
    floor = None
    if not args.no_floor:
        f_x = floor_ms(torch, pip, A, seed, stream, mode=pip.FLOOR_EXCHANGE)
        f_l = floor_ms(torch, pip, A, seed, stream, mode=pip.FLOOR_LOADSTORE)
        floor = {"ms": f_x, "elems_s": n / (f_x / 1e3), "frac_of_floor": f_x / ms_per_step,
                 "loadstore_ms": f_l, "frac_of_loadstore_floor": f_l / ms_per_step,
                 "what": "pip_calibrate_swap_floor: the n-1 swaps with no conflict resolution; ms with the "
                         "random side as one exchange at L2, loadstore_ms as a load and a store"}
    del A
    torch.cuda.empty_cache()

    # the other configurations of the workload set, one GPU only
    configs = None
    if args.configs and world == 1:
        configs = run_configs(torch, pip, args, stream)

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
        "plan": {k: plan[k] for k in ("driver", "fresh_per_round", "max_active", "slots", "grid_blocks",
                                      "block_threads", "aux_bytes", "smem_bytes", "aux_bound_bytes", "min_rounds",
                                      "flags")},
        "aux": aux,
        "rounds": st.rounds,
        "loser_fraction": st.losers / max(1, st.attempts),
        "eps_sweep": sweep,
        "reservation_rules": rules,
        "commit_modes": modes,
        "random_swap_floor": floor,
        "configs": configs,
        "step_ms": ms,
        "median_ms_per_step": statistics.median(ms),
    }
    print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


def oracle_pool_baseline(jobs, what):
    """The oracle on all host cores over a bounded sample of independent
    arrays: one sequential Knuth shuffle (oracle/knuth.c) per array of
    A[i] = i, the arrays spread over host threads (the C oracle runs outside
    the GIL), largest first.  jobs: (n, dtype, seed) triples.  The arrays are
    built before the clock starts."""
    import concurrent.futures as cf

    import oracle
    import workloads

    cores = os.cpu_count() or 1
    jobs = sorted(jobs, key=lambda j: -j[0])
    arrs = [(workloads.iota(n, dt), int(sd)) for n, dt, sd in jobs]
    t0 = time.perf_counter()
    with cf.ThreadPoolExecutor(max_workers=cores) as ex:
        list(ex.map(lambda a: oracle.knuth_hash(a[0], a[1]), arrs))
    sec = time.perf_counter() - t0
    total = sum(n for n, _, _ in jobs)
    return {"value": total / sec, "unit": "elems/s", "req_s": len(jobs) / sec, "cores": cores, "kind": "oracle",
            "sample": f"{what}: {len(jobs)} arrays, {total} elements, {sec:.1f} s on {cores} host threads"}


def run_configs(torch, pip, args, stream):
    """The rest of the workload set, each at its stated size, in this process:
    the 2^20 shuffle (L2-resident, so L2 is flushed between timed steps), the
    2^30 16-byte records, the 8192-array batch and the 20,000-request serving
    stream."""
    out = {}
    peak = measured_peak_hbm()[0]
    # configuration 1: n = 2^20 uint64, seed 1, eps = 0.5
    n1 = 1 << 20
    A1 = torch.arange(n1, dtype=torch.int64, device="cuda")
    flush = torch.zeros(256 << 20, dtype=torch.int32, device="cuda")  # 1 GiB, larger than L2
    p1 = pip.plan(n1, "u64", 0.5)
    ms1 = time_steps(torch, pip, A1, 1, 0.5, max(args.steps, 10), args.warmup, stream, {}, flush=flush)
    st1 = torch.zeros(pip.STATS_BYTES, dtype=torch.uint8, device="cuda")
    pip.shuffle(A1, seed=1, eps=0.5, stats=st1)
    pip.check()
    s1 = pip.read_stats(st1)
    m1 = statistics.median(ms1)
    out["shuffle_2^20_u64_seed1_eps0.5"] = {
        "ms": m1, "value": n1 / (m1 / 1e3), "unit": "elems/s", "driver": p1["driver"],
        "fresh_per_round": p1["fresh_per_round"], "rounds": s1.rounds, "steps": len(ms1),
        "l2": "8 MiB input held by L2: a 1 GiB buffer is rewritten between timed steps",
        "note": "round-latency-bound (about n / F rounds of a few microseconds); not an HBM case"}
    del A1, flush
    torch.cuda.empty_cache()

    # configuration 3: n = 2^30 16-byte records, seed 3, eps = 0.5
    n3 = 1 << 30
    A3 = make_device_input(torch, n3, "rec128", "cuda")
    p3 = pip.plan(n3, "rec128", 0.5)
    k3 = min(args.steps, 5)
    ms3 = time_steps(torch, pip, A3, 3, 0.5, k3, min(args.warmup, 3), stream, {})
    st3 = torch.zeros(pip.STATS_BYTES, dtype=torch.uint8, device="cuda")
    pip.shuffle(A3, seed=3, eps=0.5, stats=st3)
    pip.check()
    s3 = pip.read_stats(st3)
    m3 = sum(ms3) / len(ms3)
    f3 = floor_ms(torch, pip, A3, 3, stream, mode=pip.FLOOR_EXCHANGE)
    f3l = floor_ms(torch, pip, A3, 3, stream, mode=pip.FLOOR_LOADSTORE)
    ach3 = BYTES_PER_ELEM["rec128"] * n3 / (m3 / 1e3) / 1e9
    out["records_2^30_rec128_seed3_eps0.5"] = {
        "ms": m3, "value": n3 / (m3 / 1e3), "unit": "elems/s", "driver": p3["driver"],
        "fresh_per_round": p3["fresh_per_round"], "rounds": s3.rounds, "steps": k3, "step_ms": ms3,
        "roofline": {"bound": "hbm", "achieved": ach3, "peak": peak, "unit": "GB/s", "frac": ach3 / peak,
                     "algorithmic_bytes_per_elem": BYTES_PER_ELEM["rec128"]},
        "random_swap_floor": {"ms": f3, "loadstore_ms": f3l, "frac_of_floor": f3 / m3},
        "aux_bytes": p3["aux_bytes"], "aux_bound_bytes": p3["aux_bound_bytes"]}
    del A3
    torch.cuda.empty_cache()

    # configuration 4: the 8192-array batch
    out["batch_8192_u32"] = batch_case(torch, pip, 8192, min(args.steps, 5), min(args.warmup, 3), 1, {})
    if not args.no_cpu:
        import workloads

        bsz, bsd = workloads.batch_workload(count=8192)
        out["batch_8192_u32"]["cpu_baseline"] = oracle_pool_baseline(
            [(int(bsz[j]), "u32", int(bsd[j])) for j in range(0, 8192, 16)], "every 16th array of the batch")
    # configuration 5: the serving stream
    if args.requests > 0:
        out["serve"] = serve_case(torch, pip, args.requests, {}, min(args.requests, args.plain_requests))
        if not args.no_cpu:
            import workloads

            ssz, sdt, ssd, _ = workloads.serve_workload(count=args.requests)
            jobs, tot = [], 0
            for j in range(len(ssz)):
                if tot >= 4 * 10**8:
                    break
                jobs.append((int(ssz[j]), str(sdt[j]), int(ssd[j])))
                tot += int(ssz[j])
            out["serve"]["cpu_baseline"] = oracle_pool_baseline(
                jobs, "the stream's first requests up to 4e8 elements")
    return out


if __name__ == "__main__":
    sys.exit(main())
