"""Pins of the in-place scan oracle (CPU only).

The oracle (``oracle/scanc.c``) follows the up-sweep / down-sweep of
Algorithm 3 (Section 5.1).  It is pinned against the plain definition of the
exclusive prefix sum (numpy's cumulative sum, a library routine, shifted by
one), closed forms, the modular wrap-around of w-bit integers, and planted
mutations; the total is pinned as the sum of all elements.
"""
import ctypes
import os
import subprocess

import numpy as np
import pytest

import oracle
from tests.conftest import ROOT


def exclusive_by_definition(a: np.ndarray) -> np.ndarray:
    out = np.zeros_like(a)
    if a.shape[0] > 1:
        with np.errstate(over="ignore"):
            out[1:] = np.cumsum(a[:-1], dtype=a.dtype)
    return out


@pytest.mark.parametrize("dtype", [np.uint32, np.uint64])
@pytest.mark.parametrize("n", list(range(0, 34)) + [1000, 4097, 65536, 100003])
def test_matches_definition(dtype, n):
    rng = np.random.default_rng(n)
    a = rng.integers(0, np.iinfo(dtype).max, size=n, dtype=dtype, endpoint=True)
    want = exclusive_by_definition(a)
    with np.errstate(over="ignore"):
        total_want = int(np.sum(a, dtype=dtype)) if n else 0
    b = a.copy()
    total = oracle.scan_exclusive(b)
    assert np.array_equal(b, want)
    assert total == total_want


@pytest.mark.parametrize("n", [1, 2, 7, 1000, 12345])
def test_closed_forms(n):
    ones = np.ones(n, dtype=np.uint64)
    assert oracle.scan_exclusive(ones) == n
    assert np.array_equal(ones, np.arange(n, dtype=np.uint64))
    iota = np.arange(n, dtype=np.uint64)
    assert oracle.scan_exclusive(iota) == n * (n - 1) // 2
    i = np.arange(n, dtype=np.uint64)
    assert np.array_equal(iota, i * (i - np.uint64(1)) // np.uint64(2) if n else iota)


def test_wraps_modulo_word():
    a = np.full(5, 0xFFFFFFFF, dtype=np.uint32)
    assert oracle.scan_exclusive(a) == (5 * 0xFFFFFFFF) % (1 << 32)
    assert a.tolist() == [(k * 0xFFFFFFFF) % (1 << 32) for k in range(5)]
    b = np.full(3, 1 << 63, dtype=np.uint64)
    assert oracle.scan_exclusive(b) == (1 << 63)
    assert b.tolist() == [0, 1 << 63, 0]


MUTATIONS = {
    "up_adds_wrong_cell": ("    a[t] += a[k];\n}\n\nstatic void down64", "    a[t] += a[k + 1];\n}\n\nstatic void down64"),
    "down_reads_left_late": ("    const uint64_t left = a[k];\n    down64(a, s, k, p);",
                             "    down64(a, s, k, p);\n    const uint64_t left = a[k];"),
    "down_right_gets_p": ("    down64(a, k + 1, t, p + left);", "    down64(a, k + 1, t, p);"),
    "inclusive_leaf": ("    if (s == t) {\n        a[s] = p;\n        return;\n    }\n    const uint64_t k = (s + t) / 2;\n    const uint64_t left",
                       "    if (s == t) {\n        a[s] = p + a[s];\n        return;\n    }\n    const uint64_t k = (s + t) / 2;\n    const uint64_t left"),
    # the 32-bit path and the total
    "u32_up_adds_wrong_cell": ("    a[t] += a[k];\n}\n\nstatic void down32", "    a[t] += a[k + 1];\n}\n\nstatic void down32"),
    "u32_down_right_gets_p": ("    down32(a, k + 1, t, p + left);", "    down32(a, k + 1, t, p);"),
    "u32_left_gets_left_sum": ("    down32(a, s, k, p);", "    down32(a, s, k, p + left);"),
    "total_read_after_down": ("    *total = a[n - 1];\n    down64(a, 0, n - 1, 0);", "    down64(a, 0, n - 1, 0);\n    *total = a[n - 1];"),
}


def _scan_pins_pass(path):
    L = ctypes.CDLL(path)
    for fn, dtype in ((L.oracle_scan_u64, np.uint64), (L.oracle_scan_u32, np.uint32)):
        fn.argtypes = [ctypes.c_void_p, ctypes.c_uint64, ctypes.c_void_p]
        for n in (1, 2, 3, 5, 8, 13, 100):
            a = np.arange(1, n + 1, dtype=dtype) * dtype(3)
            want = exclusive_by_definition(a)
            tot = np.zeros(1, dtype=dtype)
            fn(a.ctypes.data, n, tot.ctypes.data)
            if not np.array_equal(a, want) or int(tot[0]) != 3 * n * (n + 1) // 2:
                return False
    return True


@pytest.mark.parametrize("name", sorted(MUTATIONS) + ["none"])
def test_planted_scan_mistake_is_caught(name, tmp_path):
    src = open(os.path.join(ROOT, "oracle", "scanc.c")).read()
    if name != "none":
        old, new = MUTATIONS[name]
        assert src.count(old) == 1, name
        src = src.replace(old, new)
    c = tmp_path / f"{name}.c"
    c.write_text(src)
    so = str(tmp_path / f"{name}.so")
    subprocess.check_call(["gcc", "-O1", "-std=c11", "-fPIC", "-shared", "-o", so, str(c)])
    assert _scan_pins_pass(so) == (name == "none")
