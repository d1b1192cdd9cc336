"""Round-by-round simulators of the parallel Knuth shuffle and of parallel
list and tree contraction (debugging aids and cross-checks).

TEST INFRASTRUCTURE ONLY (same rule as the rest of ``oracle/``).

This is a plain restatement of Algorithm 1 (Section 4.1) run under the
deterministic-reservations framework of Section 7.2 / Appendix A.1: each round
works on the first ``k`` unfinished swaps in sequential order (the Decomposable
Property's prefix of n^(1-eps) swaps, Section 4.1), every one of them reserves,
then the ones whose reservations all hold commit, and the rest are packed and
retried.  Two reservation rules are offered:

* ``"two"`` -- Algorithm 1 as printed: swap s writes max(R[s], s) and
  max(R[H[s]], s); it commits when R[s] = s and R[H[s]] = s.
* ``"oneres"`` -- the RP-OneRes rule of Appendix A.2: only R[H[s]] is written;
  swap s commits when (R[s] is unset or R[s] = s) and R[H[s]] = s.

Self-loops (H[s] = s) are removed, as the text under Algorithm 1 says, when
``skip_self_loops`` is true: they never reserve and finish in their first
round.  Indices are 0-based: the paper's step p is step p-1 here, and a larger
index is an earlier sequential step, so ``max`` picks the earliest.

The per-round winner sets are returned so that tests can compare them with the
worked example of Figure 3.  The final array is also returned; it equals the
sequential Knuth shuffle whenever the rule is correct, which is what makes this
a useful cross-check of ``knuth.c`` (and vice versa).  Round counts are not a
parity target for the GPU path (its prefix, rule variant and self-loop handling
may differ).
"""
from __future__ import annotations


def simulate(A, H, k: int | None = None, rule: str = "oneres", skip_self_loops: bool = True):
    """Run the round simulator.

    A: list of elements (copied, not modified); H: list of 0-based targets with
    H[i] <= i; k: prefix size (None = all unfinished swaps each round).
    Returns (final list, list of per-round winner sets).
    """
    n = len(A)
    if len(H) != n:
        raise ValueError("H must have one entry per element")
    for i in range(1, n):
        if not (0 <= H[i] <= i):
            raise ValueError(f"H[{i}]={H[i]} is outside [0, {i}]")
    if rule not in ("two", "oneres"):
        raise ValueError("rule must be 'two' or 'oneres'")
    A = list(A)
    unfinished = list(range(n - 1, 0, -1))  # sequential order: n-1 first; step 0 is a no-op
    rounds = []
    while unfinished:
        prefix = unfinished if k is None else unfinished[:k]
        rest = [] if k is None else unfinished[k:]
        R = {}  # reservation map: location -> max step index written there

        def reserve(loc, s):
            R[loc] = max(R.get(loc, -1), s)

        # reserve phase
        for s in prefix:
            if skip_self_loops and H[s] == s:
                continue
            if rule == "two":
                reserve(s, s)
            reserve(H[s], s)
        # commit phase: decide every swap against the full R, then apply
        winners = []
        for s in prefix:
            if skip_self_loops and H[s] == s:
                winners.append(s)
                continue
            own = R.get(s, -1)
            if rule == "two":
                ok = own == s and R.get(H[s], -1) == s
            else:
                ok = (own == -1 or own == s) and R.get(H[s], -1) == s
            if ok:
                winners.append(s)
        won = set(winners)
        # the committed swaps touch disjoint locations, so any order gives the same array
        for s in winners:
            t = H[s]
            A[s], A[t] = A[t], A[s]
        rounds.append(won)
        # pack the leftovers, keeping sequential order, ahead of the untouched rest
        unfinished = [s for s in prefix if s not in won] + rest
    return A, rounds


def list_rounds(rec, k: int | None = None):
    """Algorithm 2 (Section 4.2) under deterministic reservations.

    rec: list of [prev, next] pairs over nodes 0..n-1 (None marks a list end);
    node i has priority i.  Each round works on the first ``k`` uncontracted
    nodes in priority order (None = all of them); every one that is a local
    minimum of the remaining lists (both current neighbours absent or larger)
    is marked, then all marked nodes are spliced out together.  A contracted
    node keeps the neighbours it had when spliced out.  Returns (records,
    list of per-round contracted sets).
    """
    rec = [list(r) for r in rec]
    n = len(rec)
    todo = list(range(n))
    rounds = []
    while todo:
        active = todo if k is None else todo[:k]
        marked = [i for i in active
                  if (rec[i][0] is None or rec[i][0] > i) and (rec[i][1] is None or rec[i][1] > i)]
        if not marked:
            raise RuntimeError("no local minimum among the active nodes (a cycle?)")
        for i in marked:
            p, q = rec[i]
            if p is not None:
                rec[p][1] = q
            if q is not None:
                rec[q][0] = p
        done = set(marked)
        todo = [i for i in todo if i not in done]
        rounds.append(done)
    return rec, rounds


def tree_rounds(rec, F: int, kmax: int):
    """Tree contraction under the prefix schedule (Section 4.2), written
    independently of ``treec.c`` as a cross-check on small forests.

    rec: list of [parent, left, right, round] over nodes 0..n-1, None for a
    missing pointer.  Round r (from 1) works on the carried leaves plus the
    next fn = min(F, unadmitted, kmax - m + 1) node ids (m the previous
    active count; fn = min(F, n) in round 1).  An active leaf with a parent
    is raked when no leaf among its sibling, its nephews (children of the
    sibling) and its uncle (the other child of the grandparent) has a smaller
    id, else carried (both decided on the state at the start of the round,
    so a carried leaf may have become a root meanwhile).  Raking x with
    parent p, sibling s, grandparent g splices p out (s takes its place) and
    sets x's record to [p, s, g, r].  Returns (records, per-round raked sets).
    """
    rec = [list(r) for r in rec]
    n = len(rec)

    def leaf(v):
        return rec[v][1] is None and rec[v][2] is None

    def kids(v):
        return [rec[v][1], rec[v][2]]

    admitted, carried, m_prev, rounds = 0, [], 0, []
    while True:
        fn = min(F, n - admitted)
        if rounds:
            fn = min(fn, kmax - m_prev + 1)
        active = carried + list(range(admitted, admitted + fn))
        admitted += fn
        if not active:
            break
        r = len(rounds) + 1
        plan, carried = {}, []
        for x in active:
            if not leaf(x) or rec[x][0] is None:
                continue
            p = rec[x][0]
            s = [c for c in kids(p) if c != x][0]
            g = rec[p][0]
            rivals = [s] if leaf(s) else kids(s)
            if g is not None:
                rivals += [c for c in kids(g) if c != p]
            if all(not leaf(y) or y > x for y in rivals):
                plan[x] = (p, s, g)
            else:
                carried.append(x)
        for x, (p, s, g) in plan.items():
            rec[s][0] = g
            if g is not None:
                rec[g][1 if rec[g][1] == p else 2] = s
            rec[x] = [p, s, g, r]
        if carried and not plan:
            raise RuntimeError("no leaf raked in a round")
        rounds.append(set(plan))
        m_prev = len(active)
    return rec, rounds
