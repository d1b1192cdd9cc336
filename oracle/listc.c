/*
 * Sequential list contraction: the oracle the GPU list-contraction path is
 * checked against.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may link, load or
 * call this file; only the tests, the smoke check and the benchmark's CPU
 * baseline do.  It shares no code, header or constant with the CUDA library.
 *
 * What it computes (Section 4.2, Algorithm 2 and the text around it).  The
 * input is a set of doubly-linked lists over the nodes 0..n-1: node i holds
 * the record (prev, next) at rec[2i], rec[2i+1], with NIL = 2^64 - 1 at the
 * ends of a list.  Node i has priority i: a node may be contracted (spliced
 * out of its list, so that its predecessor's next becomes its successor and
 * its successor's prev becomes its predecessor) once both its current
 * neighbours have larger priority.  Algorithm 2 contracts all such local
 * minima of the remaining lists in parallel, round after round; because a
 * node is contracted only after every smaller neighbour is gone, each node
 * sees the same neighbours at its contraction as when the nodes are spliced
 * out one at a time in priority order, which is what the oracle does.  In the
 * in-place form the record of a contracted node keeps the two neighbours it
 * had when it was spliced out (the tree edges that the reconstruction step
 * of list ranking walks), so the output is the record array after every node
 * has been contracted.
 *
 * A second, independent definition of the same output serves as a check:
 * the neighbours at contraction are the nearest nodes with a larger index on
 * each side in the original list order (all smaller nodes are gone by then),
 * computed with the classic stack scan for nearest larger values.
 *
 * List ranking (Section 4.2: list contraction followed by the reconstruction
 * step that distributes the values back down the contraction tree) returns
 * for each node its position in its list.  Its output is unique, so the
 * oracle is the plain definition: walk every list from its head and count,
 * from the head and from the tail.
 */
#include <stdint.h>
#include <stdlib.h>

#define ORACLE_API __attribute__((visibility("default")))
#define ORACLE_NIL 0xFFFFFFFFFFFFFFFFull

/* Contract every node of the lists in rec (n records of two uint64), in place,
 * one node at a time in priority order.  Returns 0, or -1 if a pointer is out
 * of range. */
ORACLE_API int oracle_list_contract(uint64_t *rec, uint64_t n)
{
    for (uint64_t i = 0; i < n; ++i) {
        const uint64_t p = rec[2 * i], q = rec[2 * i + 1];
        if (p != ORACLE_NIL) {
            if (p >= n) return -1;
            rec[2 * p + 1] = q;   /* the predecessor now skips node i */
        }
        if (q != ORACLE_NIL) {
            if (q >= n) return -1;
            rec[2 * q] = p;       /* the successor now skips node i */
        }
    }
    return 0;
}

/* 0 when rec holds valid acyclic doubly-linked lists over 0..n-1 (every
 * pointer in range or NIL, prev and next consistent, every node on exactly
 * one list that starts at a node with prev = NIL); otherwise a negative code. */
ORACLE_API int oracle_list_check(const uint64_t *rec, uint64_t n)
{
    uint64_t seen = 0;
    for (uint64_t i = 0; i < n; ++i) {
        const uint64_t p = rec[2 * i], q = rec[2 * i + 1];
        if (p != ORACLE_NIL && (p >= n || rec[2 * p + 1] != i)) return -1;
        if (q != ORACLE_NIL && (q >= n || rec[2 * q] != i)) return -2;
    }
    for (uint64_t h = 0; h < n; ++h) {
        if (rec[2 * h] != ORACLE_NIL) continue;
        for (uint64_t v = h, steps = 0; v != ORACLE_NIL; v = rec[2 * v + 1]) {
            if (++steps > n) return -3;
            ++seen;
        }
    }
    return seen == n ? 0 : -4;   /* nodes not reached from a head lie on cycles */
}

/* The nearest larger node on each side of every node, in list order:
 * out[2i] = the closest node before i in its list with an index above i (or
 * NIL), out[2i+1] = the closest such node after i.  rec must pass
 * oracle_list_check.  Returns 0, or -1 when out of memory. */
ORACLE_API int oracle_list_nearest_larger(const uint64_t *rec, uint64_t n, uint64_t *out)
{
    uint64_t *stack = (uint64_t *)malloc((n ? n : 1) * sizeof(uint64_t));
    if (stack == NULL) return -1;
    for (uint64_t h = 0; h < n; ++h) {
        if (rec[2 * h] != ORACLE_NIL) continue;
        /* forward pass: nearest larger to the left */
        uint64_t top = 0, tail = h;
        for (uint64_t v = h; v != ORACLE_NIL; v = rec[2 * v + 1]) {
            while (top > 0 && stack[top - 1] < v) --top;
            out[2 * v] = top > 0 ? stack[top - 1] : ORACLE_NIL;
            stack[top++] = v;
            tail = v;
        }
        /* backward pass: nearest larger to the right */
        top = 0;
        for (uint64_t v = tail; v != ORACLE_NIL; v = rec[2 * v]) {
            while (top > 0 && stack[top - 1] < v) --top;
            out[2 * v + 1] = top > 0 ? stack[top - 1] : ORACLE_NIL;
            stack[top++] = v;
        }
    }
    free(stack);
    return 0;
}

/* List ranking by its definition: out[2i] = the number of nodes before node
 * i in its list, out[2i+1] = the number of nodes after it.  rec must pass
 * oracle_list_check (the walk stops at n steps otherwise).  Returns 0, or -1
 * when a list is longer than n (a cycle). */
ORACLE_API int oracle_list_rank(const uint64_t *rec, uint64_t n, uint64_t *out)
{
    for (uint64_t h = 0; h < n; ++h) {
        if (rec[2 * h] != ORACLE_NIL) continue;   /* not a head */
        uint64_t len = 0;
        for (uint64_t v = h; v != ORACLE_NIL; v = rec[2 * v + 1]) {
            if (len >= n) return -1;
            out[2 * v] = len;                     /* nodes before v */
            ++len;
        }
        for (uint64_t v = h; v != ORACLE_NIL; v = rec[2 * v + 1])
            out[2 * v + 1] = len - 1 - out[2 * v];  /* nodes after v */
    }
    return 0;
}
