/*
 * Tree contraction by rounds over a prefix of the nodes: the oracle the GPU
 * tree-contraction path is checked against.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may link, load or
 * call this file; only the tests, the smoke check and the benchmark's CPU
 * baseline do.  It shares no code, header or constant with the CUDA library.
 *
 * What it computes (Section 4.2, the tree contraction paragraph, read with
 * the Decomposable Property of Section 3).  The input is a forest of rooted
 * binary trees in which every internal node has exactly two children: node
 * i holds the record (parent, left, right, round) at rec[4i .. 4i+3], NIL =
 * 2^64 - 1 for a missing pointer; a leaf has left = right = NIL, a root has
 * parent = NIL; the round word is not read.
 *
 * Raking a leaf l whose parent is p removes l together with p: the other
 * child s of p (its sibling) takes p's place under p's parent g (or becomes
 * a root when p was one).  Two rakes may run in the same round only when
 * neither removes a node the other reads or writes; that is the case unless
 * one leaf is the other's sibling, uncle (the other child of its
 * grandparent) or nephew (a child of its sibling), which also keeps a
 * parent-child pair from being contracted in one round, the condition the
 * paper states.
 *
 * The rounds follow the prefix schedule of deterministic reservations.  Node
 * i has priority i.  Round r works on the active set: the leaves carried from
 * round r-1 and a fresh block of the next fn node indices (internal nodes and
 * leaves without a parent in it need no work and leave at once), with
 *     fn = min(F, nodes not yet admitted, kmax - m + 1),
 * m the size of the previous active set (for round 1, fn = min(F, n)).  In a
 * round every active leaf with a parent is raked exactly when its index is
 * below those of all its sibling, uncle and nephew leaves (all decided on the
 * state at the start of the round); the rest are carried.  The smallest
 * active leaf is always raked, so every round makes progress.  A raked leaf's
 * record becomes (p, s, g, r): the parent removed with it, the sibling that
 * took the parent's place, the grandparent (NIL if none) and the round,
 * counted from 1.  A removed internal node keeps the record it had when it
 * was removed; a leaf that is never raked (the last leaf of its tree) keeps
 * its round word.
 *
 * With F = 1 every round admits one node, which is then the smallest leaf
 * not yet raked, so the rounds rake the leaves one at a time in index order:
 * oracle_tree_contract_seq writes that sequential process out on its own
 * (round = index + 1) as a check of the round schedule.  The output of any
 * schedule can be checked by oracle_tree_uncontract, which undoes the rakes
 * in decreasing round order and must give back the input.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORACLE_API __attribute__((visibility("default")))
#define T_NIL 0xFFFFFFFFFFFFFFFFull
#define PAR(i) rec[4 * (i) + 0]
#define LEFT(i) rec[4 * (i) + 1]
#define RIGHT(i) rec[4 * (i) + 2]
#define ROUND(i) rec[4 * (i) + 3]

static int is_leaf(const uint64_t *rec, uint64_t i) { return LEFT(i) == T_NIL && RIGHT(i) == T_NIL; }

/* The other child of p (the one that is not c), or T_NIL if c is not a child. */
static uint64_t other_child(const uint64_t *rec, uint64_t p, uint64_t c)
{
    if (LEFT(p) == c) return RIGHT(p);
    if (RIGHT(p) == c) return LEFT(p);
    return T_NIL;
}

/* 1 if the leaf x (a leaf with a parent) may be raked in a round that starts
 * from the current state: its index is below that of every sibling, uncle and
 * nephew that is a leaf.  -1 on inconsistent input. */
static int may_rake(const uint64_t *rec, uint64_t n, uint64_t x)
{
    const uint64_t p = PAR(x);
    const uint64_t s = other_child(rec, p, x);
    if (s == T_NIL || s >= n) return -1;
    if (is_leaf(rec, s)) {
        if (s < x) return 0;                          /* sibling */
    } else {
        const uint64_t a = LEFT(s), b = RIGHT(s);
        if (a >= n || b >= n) return -1;
        if (is_leaf(rec, a) && a < x) return 0;        /* nephews */
        if (is_leaf(rec, b) && b < x) return 0;
    }
    const uint64_t g = PAR(p);
    if (g != T_NIL) {
        if (g >= n) return -1;
        const uint64_t u = other_child(rec, g, p);
        if (u == T_NIL || u >= n) return -1;
        if (is_leaf(rec, u) && u < x) return 0;        /* uncle */
    }
    return 1;
}

/* Rake the leaf x in round r (see the header). */
static void rake(uint64_t *rec, uint64_t x, uint64_t r)
{
    const uint64_t p = PAR(x);
    const uint64_t s = other_child(rec, p, x);
    const uint64_t g = PAR(p);
    PAR(s) = g;
    if (g != T_NIL) {
        if (LEFT(g) == p) LEFT(g) = s;
        else RIGHT(g) = s;
    }
    LEFT(x) = s;
    RIGHT(x) = g;
    ROUND(x) = r;
}

/* The round schedule of the header with fresh block F and active-set cap
 * kmax (kmax >= F).  Returns the number of rounds, or -1 on a pointer out of
 * range or inconsistent input, -2 when out of memory, -3 when a round makes
 * no progress. */
ORACLE_API int64_t oracle_tree_contract(uint64_t *rec, uint64_t n, uint64_t F, uint64_t kmax)
{
    if (n == 0) return 0;
    if (F < 1 || kmax < F) return -1;
    uint64_t *active = (uint64_t *)malloc((kmax + 1) * sizeof(uint64_t));
    uint64_t *carried = (uint64_t *)malloc((kmax + 1) * sizeof(uint64_t));
    unsigned char *rakes = (unsigned char *)malloc(kmax + 1);
    if (active == NULL || carried == NULL || rakes == NULL) {
        free(active); free(carried); free(rakes);
        return -2;
    }
    uint64_t U = 0, ncarried = 0, m_prev = 0, rounds = 0;
    int64_t ret = 0;
    for (;;) {
        uint64_t fn = F < n - U ? F : n - U;
        if (rounds > 0 && kmax - m_prev + 1 < fn) fn = kmax - m_prev + 1;
        uint64_t m = 0;
        for (uint64_t j = 0; j < ncarried; ++j) active[m++] = carried[j];
        for (uint64_t i = U; i < U + fn; ++i) active[m++] = i;
        U += fn;
        if (m == 0) break;
        ++rounds;
        /* decide on the state at the start of the round */
        uint64_t nr = 0;
        for (uint64_t j = 0; j < m; ++j) {
            const uint64_t x = active[j];
            rakes[j] = 0;
            if (PAR(x) != T_NIL && PAR(x) >= n) { ret = -1; goto out; }
            if (LEFT(x) != T_NIL && LEFT(x) >= n) { ret = -1; goto out; }
            if (RIGHT(x) != T_NIL && RIGHT(x) >= n) { ret = -1; goto out; }
            if (!is_leaf(rec, x) || PAR(x) == T_NIL) continue;   /* no work */
            const int ok = may_rake(rec, n, x);
            if (ok < 0) { ret = -1; goto out; }
            rakes[j] = ok ? 1 : 2;
            nr += ok ? 1 : 0;
        }
        /* then apply the round's rakes (they touch disjoint words) */
        ncarried = 0;
        for (uint64_t j = 0; j < m; ++j) {
            if (rakes[j] == 1) rake(rec, active[j], rounds);
            else if (rakes[j] == 2) carried[ncarried++] = active[j];
        }
        if (nr == 0 && ncarried > 0) { ret = -3; goto out; }
        m_prev = m;
    }
    ret = (int64_t)rounds;
out:
    free(active); free(carried); free(rakes);
    return ret;
}

/* Sequential tree contraction: every leaf in increasing index order is
 * raked (if it still has a parent), leaf i in "round" i + 1.  Returns 0, or
 * -1 on a pointer out of range or inconsistent input. */
ORACLE_API int oracle_tree_contract_seq(uint64_t *rec, uint64_t n)
{
    for (uint64_t x = 0; x < n; ++x) {
        if (!is_leaf(rec, x) || PAR(x) == T_NIL) continue;
        const uint64_t p = PAR(x);
        if (p >= n) return -1;
        const uint64_t s = other_child(rec, p, x);
        if (s == T_NIL || s >= n) return -1;
        if (PAR(p) != T_NIL && PAR(p) >= n) return -1;
        rake(rec, x, x + 1);
    }
    return 0;
}

/* 0 when rec holds a forest of rooted binary trees over 0..n-1 in which every
 * internal node has two children: pointers in range or NIL, a node is a leaf
 * exactly when both child pointers are NIL, every child's parent points
 * back, and every node is reached from a root.  Otherwise a negative code. */
ORACLE_API int oracle_tree_check(const uint64_t *rec, uint64_t n)
{
    for (uint64_t i = 0; i < n; ++i) {
        const uint64_t p = PAR(i), a = LEFT(i), b = RIGHT(i);
        if ((a == T_NIL) != (b == T_NIL)) return -1;
        if (a != T_NIL && (a >= n || b >= n || a == b || PAR(a) != i || PAR(b) != i)) return -2;
        if (p != T_NIL && (p >= n || (LEFT(p) != i && RIGHT(p) != i))) return -3;
    }
    /* every node must reach a root by parent pointers within n steps */
    for (uint64_t i = 0; i < n; ++i) {
        uint64_t v = i, steps = 0;
        while (PAR(v) != T_NIL) {
            v = PAR(v);
            if (++steps > n) return -4;
        }
    }
    return 0;
}

/* Undo a contraction.  out is the record array after contraction; raked
 * leaves (round word in [1, max_round], given by the caller as the list of
 * raked leaves in rk[0..nr)) are put back in decreasing round order: for a
 * leaf x with record (p, s, g, r), p returns between g and s with its two
 * children as they were when it was removed, and x becomes a leaf under p
 * again.  The round words of raked leaves are restored to orig_round[x].
 * Returns 0 if every step finds the state it expects, else a negative code:
 * within a round the removed nodes (raked leaves and their parents) must be
 * distinct and none may be the sibling or grandparent of another rake of the
 * round (rakes of one round may share a grandparent, or one's sibling may be
 * another's grandparent: they then write different words); s must be a
 * child of g (a root when g is NIL) and p's recorded children x and s.  The
 * caller compares the result with the input. */
ORACLE_API int oracle_tree_uncontract(uint64_t *rec, uint64_t n, const uint64_t *rk, uint64_t nr,
                                      const uint64_t *orig_round)
{
    /* sort the raked leaves by round (counting sort) */
    uint64_t maxr = 0;
    for (uint64_t j = 0; j < nr; ++j) {
        const uint64_t x = rk[j];
        if (x >= n || ROUND(x) == 0) return -1;
        if (ROUND(x) > maxr) maxr = ROUND(x);
    }
    uint64_t *start = (uint64_t *)calloc(maxr + 2, sizeof(uint64_t));
    uint64_t *ord = (uint64_t *)malloc((nr ? nr : 1) * sizeof(uint64_t));
    uint64_t *stamp = (uint64_t *)calloc(n ? n : 1, sizeof(uint64_t));
    if (start == NULL || ord == NULL || stamp == NULL) { free(start); free(ord); free(stamp); return -2; }
    for (uint64_t j = 0; j < nr; ++j) start[ROUND(rk[j]) + 1]++;
    for (uint64_t r = 1; r <= maxr + 1; ++r) start[r] += start[r - 1];
    {
        uint64_t *fill = (uint64_t *)malloc((maxr + 2) * sizeof(uint64_t));
        if (fill == NULL) { free(start); free(ord); free(stamp); return -2; }
        memcpy(fill, start, (maxr + 2) * sizeof(uint64_t));
        for (uint64_t j = 0; j < nr; ++j) ord[fill[ROUND(rk[j])]++] = rk[j];
        free(fill);
    }
    int ret = 0;
    for (uint64_t r = maxr; r >= 1 && ret == 0; --r) {
        const uint64_t a = start[r], b = start[r + 1];
        /* the removed nodes of round r are distinct ... */
        for (uint64_t j = a; j < b; ++j) {
            const uint64_t x = ord[j], p = PAR(x);
            if (p >= n) { ret = -3; break; }
            if (stamp[x] == r || stamp[p] == r) { ret = -4; break; }
            stamp[x] = r;
            stamp[p] = r;
        }
        /* ... and no rake of the round has one as its sibling or grandparent */
        for (uint64_t j = a; j < b && ret == 0; ++j) {
            const uint64_t x = ord[j], s = LEFT(x), g = RIGHT(x);
            if (s >= n || (g != T_NIL && g >= n)) { ret = -3; break; }
            if (stamp[s] == r || (g != T_NIL && stamp[g] == r)) { ret = -4; break; }
        }
        for (uint64_t j = a; j < b && ret == 0; ++j) {
            const uint64_t x = ord[j];
            const uint64_t p = PAR(x), s = LEFT(x), g = RIGHT(x);
            if (PAR(s) != g) { ret = -5; break; }
            if (g != T_NIL && LEFT(g) != s && RIGHT(g) != s) { ret = -6; break; }
            if (!((LEFT(p) == x && RIGHT(p) == s) || (LEFT(p) == s && RIGHT(p) == x))) { ret = -7; break; }
            if (PAR(p) != g) { ret = -8; break; }
            if (g != T_NIL) {
                if (LEFT(g) == s) LEFT(g) = p;
                else RIGHT(g) = p;
            }
            PAR(s) = p;
            LEFT(x) = T_NIL;
            RIGHT(x) = T_NIL;
            ROUND(x) = orig_round[x];
        }
    }
    free(start); free(ord); free(stamp);
    return ret;
}
