/*
 * Sequential Knuth shuffle: the oracle the GPU path is checked against.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may link, load or
 * call this file; only the tests, the smoke check and the benchmark's CPU
 * baseline do.  It shares no code, header or constant table with the CUDA
 * library: every definition below is written out here from the paper and
 * from the published definition of SplitMix64.
 *
 * What it computes (Section 4.1, the Knuth-Shuffle pseudocode): for
 * i = n..1 (1-based), swap(A[i], A[H[i]]) with H[i] uniform in [1..i].
 * In 0-based form, used throughout: for i = n-1 down to 1, swap A[i] with
 * A[H[i]], 0 <= H[i] <= i.  Step i = 0 always swaps A[0] with itself and is
 * skipped.  The parallel method of Algorithm 1 (made in-place by Theorem 4.1
 * and Theorem 4.2) yields exactly this permutation, so the oracle is this
 * plain definition, one swap at a time.
 *
 * Swap targets come from one of two sources:
 *   - explicit: a caller-supplied array H[0..n) (H[0] is ignored);
 *   - hashed:   H[i] = mulhi64(splitmix64(seed XOR i), i + 1), where
 *     splitmix64 is one output step of the SplitMix64 generator
 *     (Steele, Lea and Flood, OOPSLA 2014) taken from state x, and mulhi64
 *     is the high 64 bits of the 128-bit product (Lemire's multiply-shift
 *     range reduction without rejection).  The paper fixes only that H[i]
 *     is uniform on [0, i]; this generator is the reading the library
 *     adopts, and its bias of at most (i+1)/2^64 is far below anything a
 *     test can see.
 *
 * Elements are opaque byte strings of 4, 8 or 16 bytes; a swap moves the
 * whole element.
 */
#include <stdint.h>
#include <stddef.h>
#include <string.h>

#define ORACLE_API __attribute__((visibility("default")))

/* SplitMix64 output step from state x: advance the state by the golden-ratio
 * increment, then apply the two xor-shift-multiply rounds and a final
 * xor-shift.  All arithmetic is modulo 2^64. */
ORACLE_API uint64_t oracle_splitmix64(uint64_t x)
{
    uint64_t z = x + 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

/* floor(a * b / 2^64), exact, through the compiler's 128-bit integers. */
ORACLE_API uint64_t oracle_mulhi64(uint64_t a, uint64_t b)
{
    unsigned __int128 p = (unsigned __int128)a * (unsigned __int128)b;
    return (uint64_t)(p >> 64);
}

/* The hashed swap target of step i (0-based): an integer in [0, i]. */
ORACLE_API uint64_t oracle_swap_target(uint64_t seed, uint64_t i)
{
    return oracle_mulhi64(oracle_splitmix64(seed ^ i), i + 1);
}

/* Writes H[i] for i in [0, n) into out (H[0] is always 0). */
ORACLE_API void oracle_fill_targets(uint64_t seed, uint64_t n, uint64_t *out)
{
    for (uint64_t i = 0; i < n; ++i)
        out[i] = oracle_swap_target(seed, i);
}

static void swap_elems(unsigned char *A, uint64_t a, uint64_t b, uint32_t eb)
{
    unsigned char tmp[16];
    memcpy(tmp, A + a * eb, eb);
    memcpy(A + a * eb, A + b * eb, eb);
    memcpy(A + b * eb, tmp, eb);
}

static int valid_elem_bytes(uint32_t eb)
{
    return eb == 4 || eb == 8 || eb == 16;
}

/* Knuth shuffle with hashed targets.  Returns 0, or -1 on a bad element
 * size. */
ORACLE_API int oracle_knuth_hash(void *A, uint64_t n, uint32_t elem_bytes,
                                 uint64_t seed)
{
    if (!valid_elem_bytes(elem_bytes)) return -1;
    unsigned char *a = (unsigned char *)A;
    for (uint64_t i = n; i-- > 1;) {
        uint64_t j = oracle_swap_target(seed, i);
        swap_elems(a, i, j, elem_bytes);
    }
    return 0;
}

/* Knuth shuffle with explicit targets H[0..n) (H[0] ignored).  Returns 0,
 * -1 on a bad element size, or -2 if some H[i] > i (checked before any
 * element moves). */
ORACLE_API int oracle_knuth_explicit(void *A, uint64_t n, uint32_t elem_bytes,
                                     const uint32_t *H)
{
    if (!valid_elem_bytes(elem_bytes)) return -1;
    for (uint64_t i = 1; i < n; ++i)
        if ((uint64_t)H[i] > i) return -2;
    unsigned char *a = (unsigned char *)A;
    for (uint64_t i = n; i-- > 1;)
        swap_elems(a, i, H[i], elem_bytes);
    return 0;
}

/*
 * Uniformity check support: for seeds s_t = t * seed_stride (t = 0..count-1)
 * shuffles A = [0, 1, ..., n-1] with hashed targets and counts how often
 * each of the n! permutations appears.  The permutation's rank is its
 * Lehmer code in the factorial number system.  n must be at most 10.
 * counts must hold n! zero-initialised entries.  Returns 0 or -1.
 */
ORACLE_API int oracle_perm_histogram(uint32_t n, uint64_t count,
                                     uint64_t seed_stride, uint64_t *counts)
{
    if (n == 0 || n > 10) return -1;
    uint64_t perm[10];
    for (uint64_t t = 0; t < count; ++t) {
        for (uint32_t i = 0; i < n; ++i) perm[i] = i;
        oracle_knuth_hash(perm, n, 8, t * seed_stride);
        uint64_t rank = 0;
        for (uint32_t i = 0; i < n; ++i) {
            uint64_t smaller = 0;
            for (uint32_t j = i + 1; j < n; ++j)
                if (perm[j] < perm[i]) ++smaller;
            rank = rank * (n - i) + smaller;
        }
        counts[rank] += 1;
    }
    return 0;
}
