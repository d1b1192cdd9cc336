"""Seeded synthetic inputs shared by the tests and the benchmark.

This module generates workload data only: initial arrays, record payloads,
explicit target sequences drawn from numpy's generator, and the size mixes of
the batched and served workloads.  It holds none of the shuffle's arithmetic
(no swap-target generator, no swapping) and imports neither ``oracle`` nor the
CUDA package, so both sides can take their inputs from here.

The paper measures on synthetic arrays of 10 million to 1 billion 64-bit
integers (Section 7.2); the shapes below follow that: A[i] = i keys of 4 or 8
bytes, and 16-byte records {key = i, payload = mix(i)}.  For list contraction
it uses 10 to 200 million nodes of two 64-bit pointers (Section 7.3): random
doubly-linked lists over node ids 0..n-1, NIL = 2^64 - 1 at the ends.  For
tree contraction (same section, same sizes) it uses forests of rooted binary
trees in which every internal node has two children, one 32-byte record
(parent, left, right, round) per node, with node ids in random order.
"""
from __future__ import annotations

import numpy as np

_M64 = np.uint64(0xFFFFFFFFFFFFFFFF)


def _mix64(x: np.ndarray) -> np.ndarray:
    """SplitMix64 output step applied elementwise (uint64, wraps mod 2^64).

    Used here only to make record payloads and workload size draws; the
    library's swap targets are computed independently on each side.
    """
    with np.errstate(over="ignore"):
        z = x.astype(np.uint64) + np.uint64(0x9E3779B97F4A7C15)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        return z ^ (z >> np.uint64(31))


def iota(n: int, dtype: str = "u64") -> np.ndarray:
    """A[i] = i as uint32 ("u32") or uint64 ("u64")."""
    return np.arange(n, dtype=np.uint32 if dtype == "u32" else np.uint64)


def record_payload(keys: np.ndarray) -> np.ndarray:
    """Payload of record i: the SplitMix64 mix of i (the record workload's pattern)."""
    return _mix64(keys)


def records(n: int) -> np.ndarray:
    """(n, 2) uint64 array of 16-byte records {key = i, payload = mix(i)}."""
    keys = np.arange(n, dtype=np.uint64)
    out = np.empty((n, 2), dtype=np.uint64)
    out[:, 0] = keys
    out[:, 1] = record_payload(keys)
    return out


def make(n: int, dtype: str) -> np.ndarray:
    """The standard input of a dtype: iota for u32/u64, records for rec128."""
    if dtype == "rec128":
        return records(n)
    return iota(n, dtype)


def random_targets(n: int, rng_seed: int) -> np.ndarray:
    """Explicit uniform targets H[i] in [0, i] (H[0] = 0) from numpy's PCG64."""
    rng = np.random.default_rng(rng_seed)
    if n == 0:
        return np.zeros(0, dtype=np.uint32)
    i = np.arange(n, dtype=np.float64)
    H = np.floor(rng.random(n) * (i + 1)).astype(np.int64)
    H = np.minimum(H, np.arange(n))
    return H.astype(np.uint32)


def uniforms(stream_seed: int, count: int) -> np.ndarray:
    """u_j = (mix(S ^ j) >> 11) * 2^-53 for j < count: a counter-based stream on [0, 1)."""
    j = np.arange(count, dtype=np.uint64)
    z = _mix64(np.uint64(stream_seed) ^ j)
    return (z >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def log_uniform_sizes(count: int, lo_exp: float, hi_exp: float, stream_seed: int) -> np.ndarray:
    """floor(2^(lo + (hi-lo) u_j)) clamped to [2^lo, 2^hi], as int64."""
    u = uniforms(stream_seed, count)
    s = np.floor(np.exp2(lo_exp + (hi_exp - lo_exp) * u)).astype(np.int64)
    return np.clip(s, int(2 ** lo_exp), int(2 ** hi_exp))


def batch_workload(count: int = 8192, lo_exp: int = 8, hi_exp: int = 22, stream_seed: int = 7):
    """Batched workload: sizes log-uniform in [2^lo, 2^hi] from stream seed 7,
    per-array target seed = array index, uint32 iota arrays."""
    sizes = log_uniform_sizes(count, lo_exp, hi_exp, stream_seed)
    seeds = np.arange(count, dtype=np.uint64)
    return sizes, seeds


def serve_workload(count: int = 20000, lo_exp: int = 12, hi_exp: int = 28, size_seed: int = 5,
                   arrival_seed: int = 11, rate_per_s: float = 1.0):
    """Served workload: sizes log-uniform in [2^lo, 2^hi] (stream 5), dtype u64
    when the low bit of mix(5 ^ j ^ 0xD1) is 1 else u32, per-request target
    seed = request id, exponential inter-arrival times at ``rate_per_s``
    (stream 11).  Returns (sizes, dtypes, seeds, arrival_times_s)."""
    sizes = log_uniform_sizes(count, lo_exp, hi_exp, size_seed)
    j = np.arange(count, dtype=np.uint64)
    coin = _mix64(np.uint64(size_seed) ^ j ^ np.uint64(0xD1)) & np.uint64(1)
    dtypes = np.where(coin == 1, "u64", "u32")
    seeds = np.arange(count, dtype=np.uint64)
    u = uniforms(arrival_seed, count)
    gaps = -np.log1p(-u) / rate_per_s
    arrivals = np.cumsum(gaps)
    return sizes, dtypes, seeds, arrivals


LIST_NIL = np.uint64(0xFFFFFFFFFFFFFFFF)


def lists_from_order(order: np.ndarray, nlists: int = 1) -> np.ndarray:
    """(n, 2) uint64 records (prev, next) of the lists that visit the node ids
    of ``order`` in turn, cut into ``nlists`` lists of near-equal length."""
    order = np.asarray(order, dtype=np.uint64)
    n = order.shape[0]
    rec = np.full((n, 2), LIST_NIL, dtype=np.uint64)
    if n == 0:
        return rec
    cuts = np.linspace(0, n, max(1, min(nlists, n)) + 1).astype(np.int64)
    for a, b in zip(cuts[:-1], cuts[1:]):
        seg = order[a:b]
        if seg.shape[0] > 1:
            rec[seg[1:], 0] = seg[:-1]
            rec[seg[:-1], 1] = seg[1:]
    return rec


def random_lists(n: int, rng_seed: int, nlists: int = 1) -> np.ndarray:
    """Records of ``nlists`` random lists over 0..n-1: the visiting order is a
    uniform permutation from numpy's PCG64 seeded with ``rng_seed``."""
    order = np.random.default_rng(rng_seed).permutation(n).astype(np.uint64)
    return lists_from_order(order, nlists)


TREE_NIL = LIST_NIL


def tree_records(parent: np.ndarray, left: np.ndarray, right: np.ndarray, perm: np.ndarray | None = None,
                 round_fill: int = 0) -> np.ndarray:
    """(n, 4) uint64 records (parent, left, right, round) of a forest given by
    parent / child arrays over ids 0..n-1 (NIL = 2^64 - 1), with every id x
    renamed perm[x] when ``perm`` is given; the round words hold ``round_fill``."""
    parent = np.asarray(parent, dtype=np.uint64)
    left = np.asarray(left, dtype=np.uint64)
    right = np.asarray(right, dtype=np.uint64)
    n = parent.shape[0]
    rec = np.full((n, 4), TREE_NIL, dtype=np.uint64)
    rec[:, 3] = np.uint64(round_fill)
    if n == 0:
        return rec
    if perm is None:
        perm = np.arange(n, dtype=np.uint64)
    perm = np.asarray(perm, dtype=np.uint64)

    def ren(a):
        out = np.full(n, TREE_NIL, dtype=np.uint64)
        ok = a != TREE_NIL
        out[ok] = perm[a[ok].astype(np.int64)]
        return out

    idx = perm.astype(np.int64)
    rec[idx, 0] = ren(parent)
    rec[idx, 1] = ren(left)
    rec[idx, 2] = ren(right)
    return rec


def random_tree(leaves: int, rng_seed: int, trees: int = 1, round_fill: int = 0) -> np.ndarray:
    """A forest of ``trees`` random binary trees with ``leaves`` leaves in all
    (every internal node has two children; 2 * leaves - trees nodes).  Each
    tree is built bottom-up: its current roots are shuffled and joined in
    pairs under new internal nodes, level after level, which gives trees of
    depth about log2 of their leaves; then all node ids are renamed by a
    uniform permutation, so that priorities (ids) carry no information about
    the shape.  numpy's PCG64 seeded with ``rng_seed`` drives both steps."""
    rng = np.random.default_rng(rng_seed)
    trees = max(1, min(trees, leaves))
    n = 2 * leaves - trees
    parent = np.full(n, TREE_NIL, dtype=np.uint64)
    left = np.full(n, TREE_NIL, dtype=np.uint64)
    right = np.full(n, TREE_NIL, dtype=np.uint64)
    cuts = np.linspace(0, leaves, trees + 1).astype(np.int64)
    nxt = leaves
    for a, b in zip(cuts[:-1], cuts[1:]):
        roots = np.arange(a, b, dtype=np.int64)
        while roots.shape[0] > 1:
            roots = roots[rng.permutation(roots.shape[0])]
            k = roots.shape[0] // 2
            x, y = roots[:k], roots[k:2 * k]
            new = np.arange(nxt, nxt + k, dtype=np.int64)
            nxt += k
            left[new] = x.astype(np.uint64)
            right[new] = y.astype(np.uint64)
            parent[x] = new.astype(np.uint64)
            parent[y] = new.astype(np.uint64)
            roots = np.concatenate([new, roots[2 * k:]])
    assert nxt == n
    perm = rng.permutation(n).astype(np.uint64)
    return tree_records(parent, left, right, perm, round_fill)


def caterpillar_tree(leaves: int, order: np.ndarray | None = None, round_fill: int = 0) -> np.ndarray:
    """A caterpillar: internal nodes form one path (the spine) and each holds
    one leaf, the deepest holding two.  Ids: leaves 0..leaves-1 from the
    bottom of the spine up (renamed through ``order`` when given), internal
    nodes after them from the bottom up."""
    n = 2 * leaves - 1
    parent = np.full(n, TREE_NIL, dtype=np.uint64)
    left = np.full(n, TREE_NIL, dtype=np.uint64)
    right = np.full(n, TREE_NIL, dtype=np.uint64)
    if leaves > 1:
        below = 0  # the subtree under the next spine node
        for j in range(leaves - 1):
            v = leaves + j
            left[v] = np.uint64(below)
            right[v] = np.uint64(j + 1)
            parent[below] = np.uint64(v)
            parent[j + 1] = np.uint64(v)
            below = v
    perm = np.arange(n, dtype=np.uint64)
    if order is not None:
        perm[:leaves] = np.asarray(order, dtype=np.uint64)
    return tree_records(parent, left, right, perm, round_fill)
