"""The oracle's pins catch plausible mistakes (runs without a GPU).

Each case plants one mistake in a temporary copy of ``oracle/knuth.c`` (a
dropped term, a wrong constant, index or operand, a reversed loop), compiles
it, and checks that at least one of the pins used in ``test_oracle.py`` fails
on the mutant.  The real oracle passes the same pins.
"""
import ctypes
import itertools
import math
import os
import subprocess
import sys

import numpy as np
import pytest

from tests.conftest import ROOT, read_golden

SRC = os.path.join(ROOT, "oracle", "knuth.c")

MUTATIONS = {
    "loop_runs_upward": ("for (uint64_t i = n; i-- > 1;)\n        swap_elems(a, i, H[i], elem_bytes);",
                         "for (uint64_t i = 1; i < n; ++i)\n        swap_elems(a, i, H[i], elem_bytes);"),
    "hash_loop_runs_upward": ("for (uint64_t i = n; i-- > 1;) {\n        uint64_t j",
                              "for (uint64_t i = 1; i < n; ++i) {\n        uint64_t j"),
    "range_drops_plus_one": ("oracle_mulhi64(oracle_splitmix64(seed ^ i), i + 1)",
                             "oracle_mulhi64(oracle_splitmix64(seed ^ i), i)"),
    "seed_added_not_xored": ("oracle_splitmix64(seed ^ i)", "oracle_splitmix64(seed + i)"),
    "wrong_shift": ("(z ^ (z >> 30))", "(z ^ (z >> 31))"),
    "dropped_final_xorshift": ("return z ^ (z >> 31);", "return z;"),
    "wrong_multiplier": ("0x94D049BB133111EBull", "0x94D049BB133111EDull"),
    "swap_loses_write": ("memcpy(A + b * eb, tmp, eb);", ""),
    "swap_wrong_operand": ("swap_elems(a, i, H[i], elem_bytes);", "swap_elems(a, i, H[i] / 2, elem_bytes);"),
    "mulhi_takes_low_half": ("return (uint64_t)(p >> 64);", "return (uint64_t)(p >> 63);"),
    "skips_last_step": ("for (uint64_t i = n; i-- > 1;)\n        swap_elems",
                        "for (uint64_t i = n - 1; i-- > 1;)\n        swap_elems"),
}


def _compile(src_text, path):
    c = path + ".c"
    with open(c, "w") as f:
        f.write(src_text)
    subprocess.check_call(["gcc", "-O1", "-std=c11", "-fPIC", "-shared", "-o", path, c])
    L = ctypes.CDLL(path)
    u64, u32, vp = ctypes.c_uint64, ctypes.c_uint32, ctypes.c_void_p
    L.oracle_splitmix64.argtypes = [u64]
    L.oracle_splitmix64.restype = u64
    L.oracle_mulhi64.argtypes = [u64, u64]
    L.oracle_mulhi64.restype = u64
    L.oracle_swap_target.argtypes = [u64, u64]
    L.oracle_swap_target.restype = u64
    L.oracle_knuth_explicit.argtypes = [vp, u64, u32, vp]
    L.oracle_knuth_hash.argtypes = [vp, u64, u32, u64]
    return L


def _pins_pass(L):
    """The pins of test_oracle.py in compact form; True when all hold."""
    g = read_golden("splitmix64_published.txt")
    state = int(g["seed"])
    for expected in map(int, g["outputs"].split()):
        if L.oracle_splitmix64(state) != expected:
            return False
        state = (state + 0x9E3779B97F4A7C15) & ((1 << 64) - 1)
    for a, b in [(2**64 - 1, 2**64 - 1), (12345678901234567, 98765432109876543)]:
        if L.oracle_mulhi64(a, b) != (a * b) >> 64:
            return False
    # H[i] = floor(splitmix64(seed ^ i) * (i + 1) / 2^64) on the published states
    s = int(g["seed"])
    for o in map(int, g["outputs"].split()):
        for i in range(1, 200):
            if L.oracle_swap_target(s ^ i, i) != (o * (i + 1)) >> 64:
                return False
        s = (s + 0x9E3779B97F4A7C15) & ((1 << 64) - 1)
    # the top of the range, H[i] = i, is reachable
    if sum(L.oracle_swap_target(5, i) == i for i in range(1, 40000)) < 3:
        return False
    f3 = read_golden("fig3_worked_example.txt")
    h0 = np.array([int(x) for x in f3["h_zero_based"].split()], dtype=np.uint32)
    A = np.arange(8, dtype=np.uint64)
    L.oracle_knuth_explicit(A.ctypes.data, 8, 8, h0.ctypes.data)
    if A.tolist() != [int(x) for x in f3["expected_output_zero_based"].split()]:
        return False
    for n in (4, 5):
        seen = set()
        for H in itertools.product(*[range(i + 1) for i in range(n)]):
            h = np.array(H, dtype=np.uint32)
            A = np.arange(n, dtype=np.uint32)
            L.oracle_knuth_explicit(A.ctypes.data, n, 4, h.ctypes.data)
            seen.add(tuple(A.tolist()))
        if len(seen) != math.factorial(n):
            return False
    n = 50
    A = np.arange(n, dtype=np.uint64)
    zeros = np.zeros(n, dtype=np.uint32)  # kept alive while the C call reads it
    L.oracle_knuth_explicit(A.ctypes.data, n, 8, zeros.ctypes.data)
    if A.tolist() != [(i + 1) % n for i in range(n)]:
        return False
    # hashed path: a permutation, and the same one the explicit path gives
    n = 3000
    H = np.array([L.oracle_swap_target(2, i) for i in range(n)], dtype=np.uint64)
    if np.any(H > np.arange(n, dtype=np.uint64)):
        return False
    a = np.arange(n, dtype=np.uint64)
    L.oracle_knuth_hash(a.ctypes.data, n, 8, 2)
    b = np.arange(n, dtype=np.uint64)
    H32 = H.astype(np.uint32)  # kept alive while the C call reads it
    L.oracle_knuth_explicit(b.ctypes.data, n, 8, H32.ctypes.data)
    if not np.array_equal(a, b) or not np.array_equal(np.sort(a), np.arange(n, dtype=np.uint64)):
        return False
    # uniformity of H[i]/(i+1): the mean of the normalised target is 1/2
    Hs = np.array([L.oracle_swap_target(99, i) for i in range(1000, 40000)], dtype=np.float64)
    u = (Hs + 0.5) / (np.arange(1000, 40000) + 1.0)
    if abs(u.mean() - 0.5) > 0.01:
        return False
    return True


def test_real_oracle_passes_compact_pins(tmp_path):
    with open(SRC) as f:
        L = _compile(f.read(), str(tmp_path / "real.so"))
    assert _pins_pass(L)


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_planted_mistake_is_caught(name, tmp_path):
    old, new = MUTATIONS[name]
    with open(SRC) as f:
        text = f.read()
    assert text.count(old) == 1, f"mutation anchor for {name} not found exactly once"
    L = _compile(text.replace(old, new), str(tmp_path / f"{name}.so"))
    assert not _pins_pass(L), f"pins did not catch mutation {name}"


# ------------------------------------------------------------------ list contraction
LIST_SRC = os.path.join(ROOT, "oracle", "listc.c")
LIST_NIL = 0xFFFFFFFFFFFFFFFF

LIST_MUTATIONS = {
    "splice_writes_wrong_field": ("rec[2 * p + 1] = q;", "rec[2 * p] = q;"),
    "drops_successor_update": ("rec[2 * q] = p;       /* the successor now skips node i */", ""),
    "contracts_in_reverse_order": (
        "for (uint64_t i = 0; i < n; ++i) {\n        const uint64_t p = rec[2 * i], q = rec[2 * i + 1];\n"
        "        if (p != ORACLE_NIL) {\n            if (p >= n) return -1;",
        "for (uint64_t i = n; i-- > 0;) {\n        const uint64_t p = rec[2 * i], q = rec[2 * i + 1];\n"
        "        if (p != ORACLE_NIL) {\n            if (p >= n) return -1;"),
    "successor_gets_successor": ("rec[2 * q] = p;", "rec[2 * q] = q;"),
    "predecessor_gets_predecessor": ("rec[2 * p + 1] = q;", "rec[2 * p + 1] = p;"),
}


def _compile_list(src_text, path):
    c = path + ".c"
    with open(c, "w") as f:
        f.write(src_text)
    subprocess.check_call(["gcc", "-O1", "-std=c11", "-fPIC", "-shared", "-o", path, c])
    L = ctypes.CDLL(path)
    L.oracle_list_contract.argtypes = [ctypes.c_void_p, ctypes.c_uint64]
    L.oracle_list_contract.restype = ctypes.c_int
    return L


def _list_pins_pass(L):
    """Brute force over every list order for n <= 5 against the nearest-larger
    definition, and the ascending closed form."""
    for n in range(1, 6):
        for order in itertools.permutations(range(n)):
            rec = np.full((n, 2), LIST_NIL, dtype=np.uint64)
            for k in range(1, n):
                rec[order[k], 0] = order[k - 1]
                rec[order[k - 1], 1] = order[k]
            if L.oracle_list_contract(rec.ctypes.data, n) != 0:
                return False
            for k, v in enumerate(order):
                left = next((order[j] for j in range(k - 1, -1, -1) if order[j] > v), LIST_NIL)
                right = next((order[j] for j in range(k + 1, n) if order[j] > v), LIST_NIL)
                if int(rec[v, 0]) != left or int(rec[v, 1]) != right:
                    return False
    return True


def test_real_list_oracle_passes_compact_pins(tmp_path):
    with open(LIST_SRC) as f:
        L = _compile_list(f.read(), str(tmp_path / "real_list.so"))
    assert _list_pins_pass(L)


@pytest.mark.parametrize("name", sorted(LIST_MUTATIONS))
def test_planted_list_mistake_is_caught(name, tmp_path):
    old, new = LIST_MUTATIONS[name]
    with open(LIST_SRC) as f:
        text = f.read()
    assert text.count(old) == 1, f"mutation anchor for {name} not found exactly once"
    L = _compile_list(text.replace(old, new), str(tmp_path / f"{name}.so"))
    assert not _list_pins_pass(L), f"pins did not catch mutation {name}"


# ------------------------------------------------------------------ list ranking
RANK_MUTATIONS = {
    "rank_counts_from_one": ("out[2 * v] = len;                     /* nodes before v */",
                             "out[2 * v] = len + 1;                 /* nodes before v */"),
    "tail_rank_off_by_one": ("out[2 * v + 1] = len - 1 - out[2 * v];", "out[2 * v + 1] = len - out[2 * v];"),
    "walks_backwards": ("for (uint64_t v = h; v != ORACLE_NIL; v = rec[2 * v + 1]) {\n            if (len >= n)",
                        "for (uint64_t v = h; v != ORACLE_NIL; v = rec[2 * v]) {\n            if (len >= n)"),
    "starts_at_tails": ("if (rec[2 * h] != ORACLE_NIL) continue;   /* not a head */",
                        "if (rec[2 * h + 1] != ORACLE_NIL) continue;   /* not a head */"),
}


def _compile_rank(src_text, path):
    L = _compile_list(src_text, path)
    L.oracle_list_rank.argtypes = [ctypes.c_void_p, ctypes.c_uint64, ctypes.c_void_p]
    L.oracle_list_rank.restype = ctypes.c_int
    return L


def _rank_pins_pass(L):
    """Every order of one list for n <= 5 and of two lists for n <= 6: the rank
    of the k-th visited node of a list of length m is (k, m - 1 - k)."""
    for n in range(1, 7):
        for order in itertools.permutations(range(n)):
            for cut in ([n] if n <= 5 else []) + ([n // 2] if n >= 2 else []):
                rec = np.full((n, 2), LIST_NIL, dtype=np.uint64)
                for seg in (order[:cut], order[cut:]):
                    for k in range(1, len(seg)):
                        rec[seg[k], 0] = seg[k - 1]
                        rec[seg[k - 1], 1] = seg[k]
                out = np.zeros((n, 2), dtype=np.uint64)
                if L.oracle_list_rank(rec.ctypes.data, n, out.ctypes.data) != 0:
                    return False
                for seg in (order[:cut], order[cut:]):
                    for k, v in enumerate(seg):
                        if int(out[v, 0]) != k or int(out[v, 1]) != len(seg) - 1 - k:
                            return False
    return True


def test_real_rank_oracle_passes_compact_pins(tmp_path):
    with open(LIST_SRC) as f:
        L = _compile_rank(f.read(), str(tmp_path / "real_rank.so"))
    assert _rank_pins_pass(L)


@pytest.mark.parametrize("name", sorted(RANK_MUTATIONS))
def test_planted_rank_mistake_is_caught(name, tmp_path):
    old, new = RANK_MUTATIONS[name]
    with open(LIST_SRC) as f:
        text = f.read()
    assert text.count(old) == 1, f"mutation anchor for {name} not found exactly once"
    L = _compile_rank(text.replace(old, new), str(tmp_path / f"{name}.so"))
    assert not _rank_pins_pass(L), f"pins did not catch mutation {name}"


# ---------------------------------------------------------------- tree contraction
TREE_SRC = os.path.join(ROOT, "oracle", "treec.c")

TREE_MUTATIONS = {
    "record_swaps_sibling_and_grandparent": ("LEFT(x) = s;\n    RIGHT(x) = g;", "LEFT(x) = g;\n    RIGHT(x) = s;"),
    "sibling_keeps_old_parent": ("    PAR(s) = g;\n    if (g != T_NIL) {\n        if (LEFT(g) == p) LEFT(g) = s;",
                                 "    if (g != T_NIL) {\n        if (LEFT(g) == p) LEFT(g) = s;"),
    "grandparent_slot_not_updated": ("        if (LEFT(g) == p) LEFT(g) = s;\n        else RIGHT(g) = s;", ""),
    "drops_uncle_check": ("if (is_leaf(rec, u) && u < x) return 0;        /* uncle */", ""),
    "drops_a_nephew_check": ("if (is_leaf(rec, b) && b < x) return 0;", ""),
    "drops_sibling_check": ("if (s < x) return 0;                          /* sibling */", ""),
    "round_off_by_one": ("ROUND(x) = r;", "ROUND(x) = r + 1;"),
    "ignores_the_throttle": ("if (rounds > 0 && kmax - m_prev + 1 < fn) fn = kmax - m_prev + 1;", ""),
    "rakes_while_deciding": ("rakes[j] = ok ? 1 : 2;", "rakes[j] = ok ? 3 : 2;\n            if (ok) rake(rec, x, rounds);"),
    "larger_index_wins": ("if (s < x) return 0;                          /* sibling */",
                          "if (s > x) return 0;                          /* sibling */"),
}


def _compile_tree(src_text, path, load=True):
    c = path + ".c"
    with open(c, "w") as f:
        f.write(src_text)
    subprocess.check_call(["gcc", "-O1", "-std=c11", "-fPIC", "-shared", "-o", path, c])
    return _load_tree(path) if load else None


def _load_tree(path):
    L = ctypes.CDLL(path)
    L.oracle_tree_contract.argtypes = [ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint64]
    L.oracle_tree_contract.restype = ctypes.c_int64
    return L


def _tree_pins_pass(L):
    """The tree pins of test_oracle_tree.py in compact form: one node per
    round against a Python sequential rake, larger prefixes against the
    Python round simulator, and every output undone by the real oracle's
    uncontract back to the input."""
    import oracle
    import workloads
    from oracle.rounds import tree_rounds

    nil = int(oracle.NIL)

    def tolist(a):
        return [[None if int(v) == nil else int(v) for v in row] for row in a]

    def seq(rows):
        rec = [list(r) for r in rows]
        for x in range(len(rec)):
            if rec[x][1] is not None or rec[x][0] is None:
                continue
            p = rec[x][0]
            s = rec[p][2] if rec[p][1] == x else rec[p][1]
            g = rec[p][0]
            rec[s][0] = g
            if g is not None:
                rec[g][1 if rec[g][1] == p else 2] = s
            rec[x] = [p, s, g, x + 1]
        return rec

    for seed in range(12):
        inp = workloads.random_tree(3 + 7 * seed, 900 + seed, trees=1 + seed % 3)
        for F, k in ((1, 4), (3, 9), (5, 7), (10**6, 10**6)):
            out = inp.copy()
            if L.oracle_tree_contract(out.ctypes.data, out.shape[0], F, k) < 0:
                return False
            if F == 1 and tolist(out) != seq(tolist(inp)):
                return False
            if F > 1 and tolist(out) != tree_rounds(tolist(inp), F, k)[0]:
                return False
            rc, back = oracle.tree_uncontract(out, inp)
            if rc != 0 or not np.array_equal(back, inp):
                return False
    return True


def test_real_tree_oracle_passes_compact_pins(tmp_path):
    with open(TREE_SRC) as f:
        L = _compile_tree(f.read(), str(tmp_path / "real_tree.so"))
    assert _tree_pins_pass(L)


def _tree_pins_in_child(so_path):
    """Runs the compact pins on a compiled mutant in a child process: a
    mutant that corrupts the tree may crash, which also counts as caught.
    Returns True when the pins all hold."""
    code = ("import sys, ctypes; sys.path.insert(0, {root!r}); "
            "from tests.test_oracle_mutations import _load_tree, _tree_pins_pass; "
            "sys.exit(0 if _tree_pins_pass(_load_tree({so!r})) else 1)").format(root=ROOT, so=so_path)
    r = subprocess.run([sys.executable, "-c", code], cwd=ROOT, capture_output=True, timeout=300)
    return r.returncode == 0


@pytest.mark.parametrize("name", sorted(TREE_MUTATIONS))
def test_planted_tree_mistake_is_caught(name, tmp_path):
    old, new = TREE_MUTATIONS[name]
    with open(TREE_SRC) as f:
        text = f.read()
    assert text.count(old) == 1, f"mutation anchor for {name} not found exactly once"
    so = str(tmp_path / f"{name}.so")
    _compile_tree(text.replace(old, new), so, load=False)
    assert not _tree_pins_in_child(so), f"pins did not catch mutation {name}"
