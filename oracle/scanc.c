/*
 * In-place exclusive scan: the oracle for the GPU scan path.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may link, load or
 * call this file; only the tests, the smoke check and the benchmark's CPU
 * baseline do.  It shares no code, header or constant with the CUDA library.
 *
 * What it computes (Section 5.1, Algorithm 3, In-Place-Scan): the exclusive
 * prefix sums of A under + (here: integer addition modulo 2^w for w = 32 or
 * 64, which is associative, so every evaluation order gives the same result)
 * and the total sigma, in place, with only the recursion stack as auxiliary
 * space.  The steps follow the algorithm as written, 0-based:
 *   up-sweep(s, t): if s < t, with k = floor((s + t) / 2), up-sweep the two
 *     halves [s, k] and [k+1, t], then add A[k] (the left half's sum) into
 *     A[t]; afterwards A[t] holds the sum of [s, t] and A[k] the left sum;
 *   sigma = A[n-1];
 *   down-sweep(s, t, p): if s = t, A[s] = p; otherwise take LeftSum = A[k]
 *     first, then down-sweep [s, k] with p and [k+1, t] with p + LeftSum.
 * The recursion here runs the two halves one after the other (the paper runs
 * them in parallel; the result is the same).
 */
#include <stdint.h>

#define ORACLE_API __attribute__((visibility("default")))

static void up32(uint32_t *a, uint64_t s, uint64_t t)
{
    if (s >= t) return;
    const uint64_t k = (s + t) / 2;
    up32(a, s, k);
    up32(a, k + 1, t);
    a[t] += a[k];
}

static void down32(uint32_t *a, uint64_t s, uint64_t t, uint32_t p)
{
    if (s == t) {
        a[s] = p;
        return;
    }
    const uint64_t k = (s + t) / 2;
    const uint32_t left = a[k];
    down32(a, s, k, p);
    down32(a, k + 1, t, p + left);
}

static void up64(uint64_t *a, uint64_t s, uint64_t t)
{
    if (s >= t) return;
    const uint64_t k = (s + t) / 2;
    up64(a, s, k);
    up64(a, k + 1, t);
    a[t] += a[k];
}

static void down64(uint64_t *a, uint64_t s, uint64_t t, uint64_t p)
{
    if (s == t) {
        a[s] = p;
        return;
    }
    const uint64_t k = (s + t) / 2;
    const uint64_t left = a[k];
    down64(a, s, k, p);
    down64(a, k + 1, t, p + left);
}

/* Exclusive scan of n 4-byte unsigned integers in place; *total = sigma. */
ORACLE_API void oracle_scan_u32(uint32_t *a, uint64_t n, uint32_t *total)
{
    if (n == 0) {
        *total = 0;
        return;
    }
    up32(a, 0, n - 1);
    *total = a[n - 1];
    down32(a, 0, n - 1, 0);
}

/* Exclusive scan of n 8-byte unsigned integers in place; *total = sigma. */
ORACLE_API void oracle_scan_u64(uint64_t *a, uint64_t n, uint64_t *total)
{
    if (n == 0) {
        *total = 0;
        return;
    }
    up64(a, 0, n - 1);
    *total = a[n - 1];
    down64(a, 0, n - 1, 0);
}
