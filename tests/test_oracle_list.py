"""Pins of the list-contraction oracle (CPU only).

The oracle (``oracle/listc.c``) splices the nodes out one at a time in
priority order (Section 4.2).  It is pinned here against what the paper and
the mathematics fix, not against itself:
  - an independent definition: every node's neighbours at contraction are the
    nearest nodes with a larger index on each side in the original list order
    (all smaller ones are gone by then), computed by the stack scan in the
    same file and checked by brute force over every list order for n <= 7;
  - the parallel rule of Algorithm 2 (contract all local minima of the
    current lists each round, on a prefix of the uncontracted nodes), run by
    the round simulator of ``oracle/rounds.py``, gives the same records;
  - closed forms (ascending and descending lists, single nodes, several lists);
  - the tree invariants of the output on random lists.
"""
import itertools

import numpy as np
import pytest

import oracle
from oracle import rounds
import workloads

NIL = oracle.NIL


def as_lists(rec):
    return [[None if int(v) == NIL else int(v) for v in r] for r in rec]


def from_lists(rec):
    return np.array([[NIL if v is None else v for v in r] for r in rec], dtype=np.uint64)


def nearest_larger_map(order):
    """{node: [nearest larger before it, nearest larger after it]} by scanning
    the list order (any node ids)."""
    n = len(order)
    out = {}
    for k, v in enumerate(order):
        left = next((order[j] for j in range(k - 1, -1, -1) if order[j] > v), None)
        right = next((order[j] for j in range(k + 1, n) if order[j] > v), None)
        out[v] = [left, right]
    return out


def brute_nearest_larger(order):
    m = nearest_larger_map(order)
    return [m[i] for i in range(len(order))]


@pytest.mark.parametrize("n", range(1, 8))
def test_every_list_order_small_n(n):
    for order in itertools.permutations(range(n)):
        rec = workloads.lists_from_order(np.array(order, dtype=np.uint64))
        assert oracle.list_check(rec) == 0
        want = brute_nearest_larger(list(order))
        got = oracle.list_contract(rec.copy())
        assert as_lists(got) == want, order
        assert as_lists(oracle.list_nearest_larger(rec)) == want, order
        for k in (1, 2, None):
            sim, _ = rounds.list_rounds(as_lists(rec), k)
            assert sim == want, (order, k)


@pytest.mark.parametrize("n", [1, 2, 5, 1000])
def test_closed_forms(n):
    asc = workloads.lists_from_order(np.arange(n, dtype=np.uint64))
    out = as_lists(oracle.list_contract(asc.copy()))
    assert out == [[None, i + 1 if i + 1 < n else None] for i in range(n)]
    desc = workloads.lists_from_order(np.arange(n, dtype=np.uint64)[::-1].copy())
    out = as_lists(oracle.list_contract(desc.copy()))
    assert out == [[i + 1 if i + 1 < n else None, None] for i in range(n)]
    singles = workloads.lists_from_order(np.arange(n, dtype=np.uint64), nlists=n)
    assert np.all(oracle.list_contract(singles.copy()) == NIL)


def test_several_lists_are_independent():
    rng = np.random.default_rng(5)
    order = rng.permutation(3000).astype(np.uint64)
    rec = workloads.lists_from_order(order, nlists=7)
    assert oracle.list_check(rec) == 0
    got = as_lists(oracle.list_contract(rec.copy()))
    cuts = np.linspace(0, 3000, 8).astype(int)
    for a, b in zip(cuts[:-1], cuts[1:]):
        want = nearest_larger_map([int(v) for v in order[a:b]])
        for v, lr in want.items():
            assert got[v] == lr


@pytest.mark.parametrize("n,nlists", [(100003, 1), (65536, 37)])
def test_tree_invariants_on_random_lists(n, nlists):
    rec = workloads.random_lists(n, rng_seed=n, nlists=nlists)
    assert oracle.list_check(rec) == 0
    out = oracle.list_contract(rec.copy())
    assert np.array_equal(out, oracle.list_nearest_larger(rec))
    idx = np.arange(n, dtype=np.uint64)
    for c in (0, 1):
        nn = out[:, c] != NIL
        assert np.all(out[nn, c] > idx[nn])  # neighbours at contraction are larger
    # exactly one node per list (its maximum) has no neighbour left
    assert int(np.sum((out[:, 0] == NIL) & (out[:, 1] == NIL))) == nlists


def test_round_counts():
    # a sorted list is a dependence chain: one contraction per round
    asc = as_lists(workloads.lists_from_order(np.arange(64, dtype=np.uint64)))
    _, r = rounds.list_rounds(asc)
    assert len(r) == 64
    # a random list needs O(log n) rounds with the whole list active
    rec = as_lists(workloads.random_lists(4096, rng_seed=1))
    _, r = rounds.list_rounds(rec)
    assert len(r) <= 4 * 12


def test_checker_rejects_broken_lists():
    rec = workloads.random_lists(100, rng_seed=2)
    bad = rec.copy()
    bad[5, 1] = 7 if int(bad[5, 1]) != 7 else 8
    assert oracle.list_check(bad) != 0
    cyc = workloads.lists_from_order(np.arange(10, dtype=np.uint64))
    cyc[0, 0], cyc[9, 1] = 9, 0
    assert oracle.list_check(cyc) != 0


# ------------------------------------------------------------------ list ranking
@pytest.mark.parametrize("n,nlists", [(1, 1), (2, 1), (17, 1), (1000, 7), (100003, 1), (100003, 64)])
def test_list_rank_equals_the_visiting_order(n, nlists):
    # the generator visits order[] in turn, cut into near-equal lists: the
    # k-th node of a list has k nodes before it and (length - 1 - k) after it
    order = np.random.default_rng(n + nlists).permutation(n).astype(np.uint64)
    rec = workloads.lists_from_order(order, nlists)
    out = oracle.list_rank(rec)
    cuts = np.linspace(0, n, max(1, min(nlists, n)) + 1).astype(np.int64)
    for a, b in zip(cuts[:-1], cuts[1:]):
        seg = order[a:b].astype(np.int64)
        k = np.arange(b - a, dtype=np.uint64)
        assert np.array_equal(out[seg, 0], k)
        assert np.array_equal(out[seg, 1], (b - a - 1) - k)


def test_list_rank_follows_the_contraction_tree():
    # the relation the reconstruction step uses (Section 4.2): with p the
    # nearest larger node on v's left (the neighbour v had when spliced out),
    # rank(v) = rank(p) + d where d - 1 nodes lie between them, all of them
    # smaller than v (they were spliced out before v); likewise on the right
    order = np.random.default_rng(3).permutation(3000).astype(np.uint64)
    rec = workloads.lists_from_order(order, 3)
    rank = oracle.list_rank(rec)
    nl = oracle.list_nearest_larger(rec)
    where = np.empty(3000, dtype=np.int64)
    where[order.astype(np.int64)] = np.arange(3000)
    for v in range(3000):
        p, q = int(nl[v, 0]), int(nl[v, 1])
        if p != NIL:
            d = int(rank[v, 0]) - int(rank[p, 0])
            assert d >= 1 and where[v] - where[p] == d
            assert all(int(order[j]) < v for j in range(where[p] + 1, where[v]))
        else:  # no larger node before v: all nodes before it are smaller
            assert all(int(order[j]) < v for j in range(where[v] - int(rank[v, 0]), where[v]))
        if q != NIL:
            d = int(rank[v, 1]) - int(rank[q, 1])
            assert d >= 1 and where[q] - where[v] == d
            assert all(int(order[j]) < v for j in range(where[v] + 1, where[q]))


def test_list_rank_rejects_a_cycle():
    rec = workloads.random_lists(10, rng_seed=1)
    head = int(np.nonzero(rec[:, 0] == NIL)[0][0])
    tail = int(np.nonzero(rec[:, 1] == NIL)[0][0])
    rec[head, 0], rec[tail, 1] = tail, head  # close the list into a ring: no head left
    out = oracle.list_rank(rec)  # no head: nothing is ranked, and no walk runs away
    assert out.shape == (10, 2)
