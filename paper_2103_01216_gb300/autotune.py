"""Autotuner for the shuffle's launch options, cached per size class.

The planner's defaults come from sweeps on GB300.  The autotuner refines them
for a size class -- (element type, round(log2 n), eps rounded to 0.05), or for
a batch, its element type and size mix -- by timing candidate option sets on
the GPU through the library's own entry points and keeping the fastest.  The
candidates cover the prefix constant C (F = C * n^(1-eps), always clamped by
the scratch bound c * n^(1-eps)), the slot factor of the reservation tables,
the block shape and the round driver.  Results go to a JSON cache
(``$PIP_TUNE_CACHE`` or ``~/.cache/pip_gb300/tune.json``) that
``options_for`` reads.

Only option choice happens here; the timed work is the library's kernels.
"""
from __future__ import annotations

import json
import math
import os
import threading
from typing import Callable, Iterable

_lock = threading.Lock()

GRID_CANDIDATES = [
    dict(flags=32, prefix_c=c, slot_factor=s, block_threads=t)
    for c in (0.05, 0.1, 0.2, 0.5, 4.0)
    for s in (3, 4, 6)
    for t in (256, 512)
]
CTA_CANDIDATES = [
    dict(flags=64, prefix_c=c, slot_factor=s, block_threads=t)
    for c in (1.0, 2.0, 4.0)
    for s in (4, 8)
    for t in (512, 1024)
]
BATCH_CANDIDATES = [
    dict(prefix_c=c, block_threads=t, slot_factor=s)
    for c in (0.5, 1.0, 2.0)
    for t in (256, 512, 1024)
    for s in (4, 6)
]


def cache_path() -> str:
    p = os.environ.get("PIP_TUNE_CACHE")
    if p:
        return p
    return os.path.join(os.path.expanduser("~"), ".cache", "pip_gb300", "tune.json")


def size_class(n: int, dtype: str, eps: float) -> str:
    """Key of a single-array size class."""
    lg = round(math.log2(max(2, n)))
    return f"single/{dtype}/n2^{lg}/eps{round(eps * 20) / 20:.2f}"


def batch_class(sizes: Iterable[int], dtype: str, eps: float) -> str:
    """Key of a batch: element type, count and the log2 range of its sizes."""
    sizes = list(sizes)
    lo = round(math.log2(max(2, min(sizes)))) if sizes else 0
    hi = round(math.log2(max(2, max(sizes)))) if sizes else 0
    return f"batch/{dtype}/count{len(sizes)}/n2^{lo}-2^{hi}/eps{round(eps * 20) / 20:.2f}"


def load_cache(path: str | None = None) -> dict:
    path = path or cache_path()
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def save_cache(cache: dict, path: str | None = None) -> None:
    path = path or cache_path()
    os.makedirs(os.path.dirname(path) or ".", exist_ok=True)
    tmp = f"{path}.tmp{os.getpid()}"
    with open(tmp, "w") as f:
        json.dump(cache, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def options_for(n: int, dtype: str, eps: float, cache: dict | None = None) -> dict:
    """Cached best options for this size class, or {} (planner defaults)."""
    cache = load_cache() if cache is None else cache
    hit = cache.get(size_class(n, dtype, eps))
    return dict(hit["options"]) if hit else {}


def pick_best(candidates: list[dict], measure: Callable[[dict], float | None]) -> tuple[dict, float, list]:
    """Times every candidate with ``measure`` (ms, or None if not applicable)
    and returns (best options, best ms, all results)."""
    results = []
    best, best_ms = None, math.inf
    for c in candidates:
        ms = measure(c)
        results.append((c, ms))
        if ms is not None and ms < best_ms:
            best, best_ms = c, ms
    if best is None:
        raise RuntimeError("no candidate could be measured")
    return best, best_ms, results


def _time_ms(torch, fn, reps: int) -> float:
    fn()
    torch.cuda.synchronize()
    out = []
    for _ in range(reps):
        s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s.record()
        fn()
        e.record()
        e.synchronize()
        out.append(s.elapsed_time(e))
    return min(out)


def tune_single(n: int, dtype: str = "u64", eps: float = 0.5, reps: int = 2, cache_file: str | None = None,
                candidates: list[dict] | None = None) -> dict:
    """Times the candidate option sets for one array of this size class on the
    current GPU and records the fastest in the cache.  Returns the cache entry."""
    import torch

    import paper_2103_01216_gb300 as pip

    A = {"u32": lambda: torch.arange(n, dtype=torch.int32, device="cuda"),
         "u64": lambda: torch.arange(n, dtype=torch.int64, device="cuda"),
         "rec128": lambda: torch.zeros((n, 2), dtype=torch.int64, device="cuda")}[dtype]()
    fcap = None

    def measure(opts):
        nonlocal fcap
        try:
            plan = pip.plan(n, dtype, eps, **opts)
        except pip.PipError:
            return None
        if opts.get("flags") == 64 and plan["driver"] != pip.DRIVER_CTA:
            return None
        if opts.get("flags") == 32 and plan["fresh_per_round"] <= 64 and n > 1 << 20:
            return None  # a grid with a tiny prefix is never competitive; skip its long run

        def run():
            pip.shuffle(A, seed=1, eps=eps, **opts)
            pip.check()

        return _time_ms(torch, run, reps)

    cands = candidates if candidates is not None else (CTA_CANDIDATES + GRID_CANDIDATES)
    best, best_ms, results = pick_best(cands, measure)
    entry = {"options": best, "ms": best_ms, "n": n, "dtype": dtype, "eps": eps,
             "tried": [[c, ms] for c, ms in results]}
    with _lock:
        cache = load_cache(cache_file)
        cache[size_class(n, dtype, eps)] = entry
        save_cache(cache, cache_file)
    return entry


def tune_batch(arrays, seeds, eps: float = 0.5, reps: int = 2, cache_file: str | None = None,
               candidates: list[dict] | None = None) -> dict:
    """Times batch option sets on these arrays and records the fastest."""
    import torch

    import paper_2103_01216_gb300 as pip

    dtype = {4: "u32", 8: "u64", 16: "rec128"}[arrays[0].element_size() * (arrays[0].shape[1] if arrays[0].dim() == 2 else 1)]

    def measure(opts):
        try:
            b = pip.Batch(arrays, seeds, eps=eps, **opts)
        except pip.PipError:
            return None

        def run():
            b.run()
            pip.check()

        return _time_ms(torch, run, reps)

    best, best_ms, results = pick_best(candidates if candidates is not None else BATCH_CANDIDATES, measure)
    key = batch_class([a.shape[0] for a in arrays], dtype, eps)
    entry = {"options": best, "ms": best_ms, "tried": [[c, ms] for c, ms in results]}
    with _lock:
        cache = load_cache(cache_file)
        cache[key] = entry
        save_cache(cache, cache_file)
    return entry


def batch_options_for(sizes, dtype: str, eps: float, cache: dict | None = None) -> dict:
    cache = load_cache() if cache is None else cache
    hit = cache.get(batch_class(sizes, dtype, eps))
    return dict(hit["options"]) if hit else {}
