"""Pins of the tree-contraction oracle (Section 4.2, tree contraction under
the prefix schedule): runs without a GPU.

The oracle (``oracle/treec.c``) is checked against things it does not
compute itself:
  * a plain Python loop that rakes the leaves one at a time in index order
    (the schedule with one fresh node per round must give exactly that);
  * an independently written round simulator (``oracle/rounds.py``);
  * undoing the recorded rakes in decreasing round order (an independent
    consistency check: it must rebuild the input exactly, and it rejects a
    round whose rakes overlap);
  * two small trees worked by hand, and the caterpillar's closed form;
  * forest invariants (one leaf left per tree, each internal node removed
    once, with a leaf of its own).
"""
import numpy as np
import pytest

import oracle
import workloads
from oracle.rounds import tree_rounds

NIL = int(oracle.NIL)
N = None


def tolist(a):
    return [[None if int(v) == NIL else int(v) for v in row] for row in a]


def fromlist(rows):
    return np.array([[NIL if v is None else v for v in row] for row in rows], dtype=np.uint64)


def seq_rake_py(rows):
    """Rake every leaf in increasing index order (leaf i in round i + 1)."""
    rec = [list(r) for r in rows]
    for x in range(len(rec)):
        if rec[x][1] is not None or rec[x][0] is None:
            continue
        p = rec[x][0]
        s = rec[p][2] if rec[p][1] == x else rec[p][1]
        g = rec[p][0]
        rec[s][0] = g
        if g is not None:
            if rec[g][1] == p:
                rec[g][1] = s
            else:
                rec[g][2] = s
        rec[x] = [p, s, g, x + 1]
    return rec


def kmax_of(F):
    return F * 5 // 2 + 2


# the 5-node tree: root 4 -> (3, 2), 3 -> (0, 1)
FIVE = [[3, N, N, 0], [3, N, N, 0], [4, N, N, 0], [4, 0, 1, 0], [N, 3, 2, 0]]
FIVE_OUT = [[3, 1, 4, 1], [4, 2, N, 2], [N, N, N, 0], [4, 0, 1, 0], [N, 1, 2, 0]]

# the 7-node tree where the schedule matters: root 6 -> (2, 5), 5 -> (4, 3),
# 4 -> (0, 1); leaves z=0, x=1, l=2, w=3
SEVEN = [[4, N, N, 0], [4, N, N, 0], [6, N, N, 0], [5, N, N, 0], [5, 0, 1, 0], [6, 4, 3, 0], [N, 2, 5, 0]]
# all nodes active in round 1: leaves 0 and 2 are raked together (2's only
# leaf rival, its nephew 3, is larger), then 1 in round 2
SEVEN_ALL = [[4, 1, 5, 1], [5, 3, N, 2], [6, 5, N, 1], [N, N, N, 0], [5, 0, 1, 0], [N, 1, 3, 0], [N, 2, 5, 0]]
# one node per round: 0, then 1 (which removes 5, so 3 becomes 2's sibling),
# then 2
SEVEN_SEQ = [[4, 1, 5, 1], [5, 3, 6, 2], [6, 3, N, 3], [N, N, N, 0], [5, 0, 1, 0], [6, 1, 3, 0], [N, 2, 3, 0]]


def contract(rows, F, kmax=None):
    rec = fromlist(rows)
    r = oracle.tree_contract(rec, F, kmax if kmax is not None else kmax_of(F))
    return tolist(rec), r


def test_inputs_are_valid_forests():
    for rows in (FIVE, SEVEN):
        assert oracle.tree_check(fromlist(rows)) == 0
    for seed in range(20):
        assert oracle.tree_check(workloads.random_tree(1 + seed * 7, seed, trees=1 + seed % 3)) == 0
    assert oracle.tree_check(workloads.caterpillar_tree(9)) == 0


def test_check_rejects_broken_forests():
    bad = [r[:] for r in FIVE]
    bad[3][1] = N  # one child only
    assert oracle.tree_check(fromlist(bad)) != 0
    bad = [r[:] for r in FIVE]
    bad[0][0] = 4  # child does not point back
    assert oracle.tree_check(fromlist(bad)) != 0
    bad = [r[:] for r in FIVE]
    bad[4][0] = 3  # cycle
    bad[3][0] = 4
    assert oracle.tree_check(fromlist(bad)) != 0


def test_hand_worked_five_node_tree():
    for F in (1, 2, 5, 100):
        out, _ = contract(FIVE, F)
        assert out == FIVE_OUT, F


def test_hand_worked_seven_node_tree_both_schedules():
    out, rounds = contract(SEVEN, 7, 7)
    assert out == SEVEN_ALL and rounds == 3
    out, rounds = contract(SEVEN, 1)
    assert out == SEVEN_SEQ and rounds == 7
    assert seq_rake_py(SEVEN) == SEVEN_SEQ


@pytest.mark.parametrize("seed", range(12))
def test_one_node_per_round_is_the_sequential_rake(seed):
    rows = tolist(workloads.random_tree(1 + 5 * seed, seed, trees=1 + seed % 3))
    out, rounds = contract(rows, 1)
    assert out == seq_rake_py(rows)
    assert rounds == len(rows)
    rec = fromlist(rows)
    oracle.tree_contract_seq(rec)
    assert tolist(rec) == out


@pytest.mark.parametrize("F", [1, 2, 3, 8, 64, 10**6])
def test_c_matches_the_python_round_simulator(F):
    for seed in range(40):
        rows = tolist(workloads.random_tree(1 + seed % 31, 100 + seed, trees=1 + seed % 4))
        k = kmax_of(F) if F < 10**6 else F
        out, rounds = contract(rows, F, k)
        py, per_round = tree_rounds(rows, F, k)
        assert out == py and rounds == len(per_round), seed


@pytest.mark.parametrize("F", [1, 5, 40, 10**6])
def test_uncontract_rebuilds_the_input(F):
    for seed in range(25):
        inp = workloads.random_tree(1 + 13 * seed, 200 + seed, trees=1 + seed % 5, round_fill=7 + seed)
        out = inp.copy()
        oracle.tree_contract(out, F, kmax_of(F) if F < 10**6 else F)
        rc, back = oracle.tree_uncontract(out, inp)
        assert rc == 0 and np.array_equal(back, inp), (seed, rc)


def test_uncontract_rejects_an_overlapping_round():
    # raking siblings 0 and 1 in the same round cannot be undone
    bad = [[3, 1, 4, 1], [3, 0, 4, 1], [N, N, N, 0], [4, 0, 1, 0], [N, 1, 2, 0]]
    rc, _ = oracle.tree_uncontract(fromlist(bad), fromlist(FIVE))
    assert rc != 0
    # a wrong grandparent is caught too
    wrong = [r[:] for r in FIVE_OUT]
    wrong[0] = [3, 1, N, 1]
    rc, back = oracle.tree_uncontract(fromlist(wrong), fromlist(FIVE))
    assert rc != 0 or not np.array_equal(back, fromlist(FIVE))


def test_caterpillar_closed_form():
    # leaves numbered from the bottom of the spine up: every round rakes the
    # lowest leaf, which removes the lowest spine node
    L = 12
    rows = tolist(workloads.caterpillar_tree(L))
    for F in (1, 4, 10**6):
        out, rounds = contract(rows, F, kmax_of(F) if F < 10**6 else F)
        for j in range(L - 1):
            g = L + j + 1 if j + 1 <= L - 2 else None
            assert out[j] == [L + j, j + 1, g, j + 1], (F, j)
        assert out[L - 1][:3] == [None, None, None]


@pytest.mark.parametrize("seed", range(8))
def test_forest_invariants(seed):
    trees = 1 + seed % 4
    inp = workloads.random_tree(50 + 37 * seed, 300 + seed, trees=trees)
    n = inp.shape[0]
    out = inp.copy()
    rounds = oracle.tree_contract(out, 16, kmax_of(16))
    leaf = (inp[:, 1] == oracle.NIL)
    raked = leaf & (out[:, 3] > 0)
    kept = leaf & ~raked
    # one leaf left per tree, as a root
    assert int(kept.sum()) == trees
    assert np.all(out[kept, 0] == oracle.NIL)
    # each internal node removed exactly once, together with one of its leaves
    removed = out[raked, 0].astype(np.int64)
    assert sorted(removed.tolist()) == sorted(np.nonzero(~leaf)[0].tolist())
    assert np.all(out[raked, 3] <= rounds)
    # the removed parent's record lists the raked leaf and the recorded sibling
    for x in np.nonzero(raked)[0]:
        p, s = int(out[x, 0]), int(out[x, 1])
        assert {int(out[p, 1]), int(out[p, 2])} == {int(x), s}
    assert n == int(leaf.sum()) * 2 - trees


def test_degenerate_inputs():
    # a single leaf, a forest of single leaves, and an empty array
    out, r = contract([[N, N, N, 5]], 1)
    assert out == [[N, N, N, 5]] and r == 1
    out, r = contract([[N, N, N, 0]] * 4, 2)
    assert out == [[N, N, N, 0]] * 4 and r == 2
    rec = np.zeros((0, 4), dtype=np.uint64)
    assert oracle.tree_contract(rec, 1, 4) == 0


def test_out_of_range_pointer_is_reported():
    bad = [r[:] for r in FIVE]
    bad[0][0] = 99
    with pytest.raises(ValueError):
        contract(bad, 5)
