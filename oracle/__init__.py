"""CPU oracle for the parallel in-place random permutation, list and tree contraction and scan.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package.  The product library never links, loads or calls it, and it shares no
code with the CUDA path (see ``knuth.c`` for the arithmetic, written out from
Section 4.1 of the paper and from the published SplitMix64 definition, and
``listc.c`` for list contraction and ``treec.c`` for tree contraction,
Section 4.2, and ``scanc.c`` for the in-place scan, Section 5.1).

The C part (``knuth.c``, ``listc.c``, ``treec.c``, ``scanc.c``) is compiled with the host C compiler
into ``_liboracle.so`` next to this file; :func:`build` does that and
:func:`lib` loads it.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRCS = [os.path.join(_HERE, f) for f in ("knuth.c", "listc.c", "treec.c", "scanc.c")]
_SO = os.path.join(_HERE, "_liboracle.so")
_lock = threading.Lock()
_lib = None

ELEM_BYTES = {"u32": 4, "u64": 8, "rec128": 16}


def build(force: bool = False) -> str:
    """Compile the C sources into ``_liboracle.so`` (plain C, -O2, no CPU-specific flags)."""
    if not force and os.path.exists(_SO) and all(os.path.getmtime(_SO) >= os.path.getmtime(s) for s in _SRCS):
        return _SO
    tmp = _SO + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-o", tmp, *_SRCS])
    os.replace(tmp, _SO)
    return _SO


def lib() -> ctypes.CDLL:
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = ctypes.CDLL(_SO)
            u64, u32, vp = ctypes.c_uint64, ctypes.c_uint32, ctypes.c_void_p
            L.oracle_splitmix64.argtypes = [u64]
            L.oracle_splitmix64.restype = u64
            L.oracle_mulhi64.argtypes = [u64, u64]
            L.oracle_mulhi64.restype = u64
            L.oracle_swap_target.argtypes = [u64, u64]
            L.oracle_swap_target.restype = u64
            L.oracle_fill_targets.argtypes = [u64, u64, vp]
            L.oracle_fill_targets.restype = None
            L.oracle_knuth_hash.argtypes = [vp, u64, u32, u64]
            L.oracle_knuth_hash.restype = ctypes.c_int
            L.oracle_knuth_explicit.argtypes = [vp, u64, u32, vp]
            L.oracle_knuth_explicit.restype = ctypes.c_int
            L.oracle_perm_histogram.argtypes = [u32, u64, u64, vp]
            L.oracle_perm_histogram.restype = ctypes.c_int
            L.oracle_list_contract.argtypes = [vp, u64]
            L.oracle_list_contract.restype = ctypes.c_int
            L.oracle_list_check.argtypes = [vp, u64]
            L.oracle_list_check.restype = ctypes.c_int
            L.oracle_list_nearest_larger.argtypes = [vp, u64, vp]
            L.oracle_list_nearest_larger.restype = ctypes.c_int
            L.oracle_list_rank.argtypes = [vp, u64, vp]
            L.oracle_list_rank.restype = ctypes.c_int
            L.oracle_tree_contract.argtypes = [vp, u64, u64, u64]
            L.oracle_tree_contract.restype = ctypes.c_int64
            L.oracle_tree_contract_seq.argtypes = [vp, u64]
            L.oracle_tree_contract_seq.restype = ctypes.c_int
            L.oracle_tree_check.argtypes = [vp, u64]
            L.oracle_tree_check.restype = ctypes.c_int
            L.oracle_tree_uncontract.argtypes = [vp, u64, vp, u64, vp]
            L.oracle_tree_uncontract.restype = ctypes.c_int
            L.oracle_scan_u32.argtypes = [vp, u64, vp]
            L.oracle_scan_u32.restype = None
            L.oracle_scan_u64.argtypes = [vp, u64, vp]
            L.oracle_scan_u64.restype = None
            _lib = L
    return _lib


def splitmix64(x: int) -> int:
    return int(lib().oracle_splitmix64(x))


def mulhi64(a: int, b: int) -> int:
    return int(lib().oracle_mulhi64(a, b))


def swap_target(seed: int, i: int) -> int:
    """H[i] for the hashed generator (0-based, in [0, i])."""
    return int(lib().oracle_swap_target(seed, i))


def swap_targets(seed: int, n: int) -> np.ndarray:
    """H[0..n) as uint64 (H[0] == 0)."""
    out = np.empty(n, dtype=np.uint64)
    if n:
        lib().oracle_fill_targets(seed, n, out.ctypes.data)
    return out


def _elem_bytes(arr: np.ndarray) -> int:
    if arr.ndim == 1:
        return arr.dtype.itemsize
    if arr.ndim == 2:
        return arr.dtype.itemsize * arr.shape[1]
    raise ValueError("array must be 1-D (scalar elements) or 2-D (records)")


def knuth_hash(arr: np.ndarray, seed: int) -> np.ndarray:
    """Sequential Knuth shuffle of ``arr`` in place with hashed targets.

    ``arr`` is 1-D of 4- or 8-byte scalars, or 2-D (n, w) whose rows are
    16-byte records.  Returns ``arr``.
    """
    assert arr.flags["C_CONTIGUOUS"]
    eb = _elem_bytes(arr)
    rc = lib().oracle_knuth_hash(arr.ctypes.data, arr.shape[0], eb, seed)
    if rc != 0:
        raise ValueError(f"oracle_knuth_hash failed ({rc}); element size {eb}")
    return arr


def knuth_explicit(arr: np.ndarray, H) -> np.ndarray:
    """Sequential Knuth shuffle of ``arr`` in place with explicit targets ``H``."""
    assert arr.flags["C_CONTIGUOUS"]
    h = np.ascontiguousarray(H, dtype=np.uint32)
    if h.shape[0] != arr.shape[0]:
        raise ValueError("H must have one entry per element")
    eb = _elem_bytes(arr)
    rc = lib().oracle_knuth_explicit(arr.ctypes.data, arr.shape[0], eb, h.ctypes.data)
    if rc == -2:
        raise ValueError("H[i] > i for some i")
    if rc != 0:
        raise ValueError(f"oracle_knuth_explicit failed ({rc})")
    return arr


def perm_histogram(n: int, count: int, seed_stride: int) -> np.ndarray:
    """Counts of each of the n! output permutations of [0..n) over ``count`` seeds."""
    import math

    counts = np.zeros(math.factorial(n), dtype=np.uint64)
    rc = lib().oracle_perm_histogram(n, count, seed_stride, counts.ctypes.data)
    if rc != 0:
        raise ValueError("n must be in [1, 10]")
    return counts


# ------------------------------------------------------------------ list contraction
NIL = 0xFFFFFFFFFFFFFFFF


def _records(rec) -> np.ndarray:
    rec = np.asarray(rec)
    if rec.dtype != np.uint64 or rec.ndim != 2 or rec.shape[1] != 2 or not rec.flags["C_CONTIGUOUS"]:
        raise ValueError("records must be a C-contiguous (n, 2) uint64 array of (prev, next)")
    return rec


def list_contract(rec: np.ndarray) -> np.ndarray:
    """Contract every node of the lists in ``rec`` in place (Section 4.2): each
    record ends up holding the neighbours its node had when spliced out."""
    rec = _records(rec)
    if lib().oracle_list_contract(rec.ctypes.data, rec.shape[0]) != 0:
        raise ValueError("pointer out of range")
    return rec


def list_check(rec: np.ndarray) -> int:
    """0 when ``rec`` holds valid acyclic doubly-linked lists, else a negative code."""
    rec = _records(rec)
    return int(lib().oracle_list_check(rec.ctypes.data, rec.shape[0]))


def list_nearest_larger(rec: np.ndarray) -> np.ndarray:
    """For every node, the nearest node with a larger index before and after it
    in its list (NIL if none), as an (n, 2) array."""
    rec = _records(rec)
    out = np.empty_like(rec)
    if lib().oracle_list_nearest_larger(rec.ctypes.data, rec.shape[0], out.ctypes.data) != 0:
        raise MemoryError("oracle_list_nearest_larger")
    return out


def list_rank(rec: np.ndarray) -> np.ndarray:
    """List ranking by definition (Section 4.2: the value list contraction and
    its reconstruction step compute): for every node, the number of nodes
    before it and after it in its list, as an (n, 2) uint64 array.  ``rec``
    must hold valid acyclic lists (:func:`list_check`)."""
    rec = _records(rec)
    out = np.empty_like(rec)
    if lib().oracle_list_rank(rec.ctypes.data, rec.shape[0], out.ctypes.data) != 0:
        raise ValueError("a list is longer than n (a cycle)")
    return out


# ------------------------------------------------------------------ tree contraction
def _tree_records(rec) -> np.ndarray:
    rec = np.asarray(rec)
    if rec.dtype != np.uint64 or rec.ndim != 2 or rec.shape[1] != 4 or not rec.flags["C_CONTIGUOUS"]:
        raise ValueError("records must be a C-contiguous (n, 4) uint64 array of (parent, left, right, round)")
    return rec


def tree_contract(rec: np.ndarray, F: int, kmax: int) -> int:
    """Contract the forest in ``rec`` in place by the round schedule with fresh
    block ``F`` and active-set cap ``kmax`` (Section 4.2); returns the rounds."""
    rec = _tree_records(rec)
    r = int(lib().oracle_tree_contract(rec.ctypes.data, rec.shape[0], F, kmax))
    if r == -2:
        raise MemoryError("oracle_tree_contract")
    if r < 0:
        raise ValueError(f"inconsistent tree input ({r})")
    return r


def tree_contract_seq(rec: np.ndarray) -> np.ndarray:
    """Rake every leaf in increasing index order (leaf i in round i + 1)."""
    rec = _tree_records(rec)
    if lib().oracle_tree_contract_seq(rec.ctypes.data, rec.shape[0]) != 0:
        raise ValueError("inconsistent tree input")
    return rec


def tree_check(rec: np.ndarray) -> int:
    """0 when ``rec`` holds a valid forest of full binary trees, else a negative code."""
    rec = _tree_records(rec)
    return int(lib().oracle_tree_check(rec.ctypes.data, rec.shape[0]))


def tree_uncontract(out: np.ndarray, orig: np.ndarray) -> tuple[int, np.ndarray]:
    """Undo the rakes recorded in ``out`` (a copy is modified) in decreasing
    round order; returns (status, records), status 0 when every step was
    consistent.  ``orig`` is the input the contraction started from: its
    leaves whose left word is no longer NIL are the raked ones (a raked leaf
    records its sibling there), and its round words are put back."""
    rec = np.ascontiguousarray(_tree_records(out).copy())
    orig = _tree_records(orig)
    n = rec.shape[0]
    raked = np.nonzero((orig[:, 1] == NIL) & (rec[:, 1] != NIL))[0].astype(np.uint64)
    raked = np.ascontiguousarray(raked)
    orr = np.ascontiguousarray(orig[:, 3])
    rc = int(lib().oracle_tree_uncontract(rec.ctypes.data, n, raked.ctypes.data, raked.shape[0], orr.ctypes.data))
    return rc, rec


# ------------------------------------------------------------------ scan
def scan_exclusive(arr: np.ndarray) -> int:
    """In-place exclusive scan of a 1-D uint32 or uint64 array by the
    up-sweep / down-sweep of Algorithm 3 (Section 5.1), modulo 2^w; returns
    the total."""
    if arr.ndim != 1 or not arr.flags["C_CONTIGUOUS"] or arr.dtype not in (np.uint32, np.uint64):
        raise ValueError("expected a contiguous 1-D uint32 or uint64 array")
    tot = np.zeros(1, dtype=arr.dtype)
    fn = lib().oracle_scan_u32 if arr.dtype == np.uint32 else lib().oracle_scan_u64
    fn(arr.ctypes.data, arr.shape[0], tot.ctypes.data)
    return int(tot[0])
