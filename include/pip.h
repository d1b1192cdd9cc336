/*
 * pip.h -- C ABI of the GB300 parallel in-place random permutation library.
 *
 * The library permutes an array A of n elements in place on one GPU and
 * produces exactly the result of the sequential Knuth shuffle (Section 4.1):
 *
 *     for i = n-1 down to 1:  swap(A[i], A[H[i]]),   0 <= H[i] <= i
 *
 * (0-based; the paper is 1-based, its step p is step p-1 here, and step 0 is a
 * no-op).  Swap targets are either hashed,
 *
 *     H[i] = mulhi64(splitmix64(seed XOR i), i + 1)
 *
 * (splitmix64 = one SplitMix64 output step from state x; mulhi64 = high 64 bits
 * of the 128-bit product), or supplied explicitly.  The work runs as rounds of
 * deterministic reservations (Algorithm 1, Section 7.2, Appendix A.1) over a
 * prefix of about C * n^(1-eps) unfinished swaps, so that the auxiliary device
 * memory is O(n^(1-eps)) (the relaxed PIP model, Section 3.2; Theorem 4.2).
 *
 * Conventions for every entry point:
 *  - Pointers named *_dev are device pointers (cudaMalloc'd or any memory the
 *    GPU can address); the caller owns them and must keep them alive until the
 *    work queued on `stream` has finished.  Other pointers are host pointers.
 *  - `stream` is a cudaStream_t passed as void*; NULL means the legacy default
 *    stream.  Calls are asynchronous with respect to the host unless stated.
 *  - Every function returns a pip_status.  No C++ exception crosses the ABI.
 *    Argument errors are detected before anything is queued.  Errors detected
 *    on the device (a barrier wait that ran out, an invalid explicit target)
 *    are latched in a per-device word and reported by pip_check().
 *  - The library keeps no state between calls other than that per-device
 *    error word and the per-device launch attributes it caches; it is safe to
 *    call from several host threads on different streams.
 */
#ifndef PIP_H
#define PIP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Element type.  Elements are opaque and move whole. */
typedef enum {
    PIP_U32 = 0,    /* 4-byte elements,  A 4-byte aligned  */
    PIP_U64 = 1,    /* 8-byte elements,  A 8-byte aligned  */
    PIP_REC128 = 2  /* 16-byte records,  A 16-byte aligned */
} pip_dtype;

typedef enum {
    PIP_OK = 0,
    PIP_EINVAL = 1,    /* bad argument (null pointer, eps outside (0,1), n >= 2^32, misaligned A, H[i] > i) */
    PIP_ENOMEM = 2,    /* device or host allocation failed */
    PIP_ECUDA = 3,     /* a CUDA runtime call failed */
    PIP_ETIMEOUT = 4,  /* a bounded device-side wait ran out; the array content is unspecified */
    PIP_EAGAIN = 5,    /* serve poll: the request has not finished yet */
    PIP_EBUSY = 6,     /* serve: the request is queued behind the memory budget */
    PIP_EINTERNAL = 7, /* a device-side consistency check failed (round cap exceeded) */
    PIP_ETOOLARGE = 8  /* pip_shuffle_noalloc: the plan needs more scratch than the fixed area */
} pip_status;

/* Planned execution of one shuffle (filled by pip_plan). */
typedef struct {
    uint64_t n;
    uint32_t elem_bytes;
    double eps;
    uint32_t fresh_per_round;  /* F: fresh swaps added to the prefix each round, ~C*n^(1-eps) */
    uint32_t max_active;       /* k: cap on the swaps active in one round (F plus carried losers) */
    uint32_t slots;            /* reservation slots per round table (tree plans: phase-B cache bytes per thread) */
    uint32_t grid_blocks;      /* persistent blocks launched (0 = decided at launch) */
    uint32_t block_threads;
    uint64_t aux_bytes;        /* exact device scratch bytes this plan allocates */
    uint64_t aux_bound_bytes;  /* c*n^(1-eps) + 4096 with c = PIP_AUX_C: the bound aux_bytes obeys */
    uint64_t min_rounds;       /* ceil((n-1)/F): a lower bound on the rounds */
    uint32_t driver;           /* 0 = persistent grid, 1 = one block, 2 = one cluster (shared-memory tables), 3 = list contraction, 4 = tree contraction */
    uint32_t flags;            /* PIP_FLAG_* bits the plan runs with: the caller's plus the planner's choices */
    uint64_t smem_bytes;       /* on-chip scratch of the one-block driver (counted in the bound) */
} pip_plan_info;

/* Aux constant c (bytes per unit of n^(1-eps)) that every plan obeys. */
#define PIP_AUX_C 128.0

/* Tuning overrides; zero fields keep the planner's choice. */
typedef struct {
    double prefix_c;           /* C in F = C * n^(1-eps) (default 4 for one array, 1 for a batch;
                                  clamped so aux stays within the bound) */
    uint32_t fresh_per_round;  /* explicit F (overrides prefix_c; still clamped by the bound) */
    uint32_t slot_factor;      /* reservation slots per active swap (2..16, default 4) */
    uint32_t grid_blocks;      /* persistent blocks (clamped to what can be co-resident) */
    uint32_t block_threads;    /* multiple of 32: 128..512 for the grid driver, up to 1024 for the others */
    uint64_t wait_timeout_ns;  /* limit of each device-side barrier wait (default 2e9 ns) */
    uint32_t flags;            /* PIP_FLAG_* */
} pip_options;

/* Test hook: block 0 never arrives at its first barrier, so every other block's
 * bounded wait runs out and the call reports PIP_ETIMEOUT.  The array is left
 * untouched (the hook fires before any swap). */
#define PIP_FLAG_TEST_SKIP_BARRIER 1u
/* Prefetch into L2, one round ahead, the array lines the next fresh block
 * will swap. */
#define PIP_FLAG_PREFETCH 2u
/* Grid driver: how a winning swap moves its two elements.  Exchange commit:
 * the own element is loaded with the reservation checks, one atomic exchange
 * at L2 puts it into A[H[i]] and returns the target's element, which is
 * stored at A[i] -- one random L2 transaction per swap instead of a load and
 * a store.  Load-store commit: both elements are loaded (after the decision,
 * or with the checks under PIP_FLAG_SPECULATE) and both are stored.  By
 * default the planner takes the exchange commit for large prefixes (the
 * random-access-bound regime) and the speculative load-store commit for
 * small ones (the latency-bound regime, where the exchange would add a
 * memory round trip per round); these flags force one.  Performance only;
 * results are identical. */
#define PIP_FLAG_SWAP_LOADSTORE 4u
#define PIP_FLAG_SWAP_EXCHANGE 8u
/* Grid driver: keep the normal L2 eviction priority for the array stores
 * (by default they are marked evict-first).  Performance only; results are
 * identical. */
#define PIP_FLAG_STORE_EVICT_NORMAL 16u
/* Driver selection: by default arrays whose prefix fits in one block's shared
 * memory run on one block, larger prefixes on the persistent grid. */
#define PIP_FLAG_FORCE_GRID 32u
#define PIP_FLAG_FORCE_CTA 64u
/* One thread-block cluster (up to 16 CTAs) with the tables in distributed
 * shared memory: the default for prefixes too large for one block. */
#define PIP_FLAG_FORCE_CLUSTER 128u
/* Grid driver: issue a swap's array loads together with its reservation
 * checks instead of after them (one memory round trip less per round, extra
 * loads for the swaps that lose).  Performance only; results are identical. */
#define PIP_FLAG_SPECULATE 256u
/* The reservation rule of Algorithm 1 as printed: each step reserves both its
 * own location and its target, and commits iff it holds the maximum on both.
 * The default is the one-reservation rule of Appendix A.2 (RP-OneRes: only
 * the target is reserved, the own location is checked).  Both give the same
 * winners in every round and the same result; this one costs one more
 * reservation per step.  Honoured by the grid and one-block drivers (the
 * planner does not choose the cluster driver under it). */
#define PIP_FLAG_TWO_RES 512u
/* pip_list_contract_ex: check the whole input (every pointer in range or NIL,
 * prev and next consistent) before anything is modified, and reject it
 * untouched with PIP_EINVAL.  Without it only the range of each pointer is
 * checked, as the contraction reads it (an error then leaves the records
 * unspecified); the full check costs two random reads per node. */
#define PIP_FLAG_VALIDATE_INPUT 1024u
/* Grid driver: in each round, the next round's fresh block reserves and the
 * tables of two rounds back are cleaned before the commit instead of after
 * it, so that their latency overlaps the commit's loads rather than adding
 * to the round's end.  The planner sets it for small prefixes (the
 * latency-bound regime: measured 1.7-1.9 % faster at F ~ 70K, 3.4 % slower
 * at F ~ 706K); a caller may set it for any prefix.  Performance only;
 * results are identical. */
#define PIP_FLAG_EARLY_RESERVE 4096u
/* Test hook: run the grid driver the way a serving lane does -- launched
 * without the cooperative attribute, its blocks first meeting at a start
 * gate that gives up after wait_timeout_ns -- with errors reported in the
 * stats record (status) rather than the per-device latch.  With
 * PIP_FLAG_TEST_SKIP_BARRIER as well, block 0 never checks in, so the gate
 * gives up: every block leaves before touching the array or the tables and
 * the stats record PIP_EBUSY. */
#define PIP_FLAG_TEST_GATED 8192u

/* Per-call statistics written by the device at the end of a shuffle. */
typedef struct {
    uint32_t status;          /* pip_status of the device-side run */
    uint32_t rounds;          /* rounds executed */
    uint64_t attempts;        /* sum over rounds of the active swaps (F per round plus losers) */
    uint64_t losers;          /* sum over rounds of the swaps carried to the next round */
    uint32_t max_active;      /* largest active set seen */
    uint32_t grid_blocks;     /* blocks that ran */
    uint64_t reserved[4];
} pip_stats;

/* Per-array statistics of a batched run. */
typedef struct {
    uint32_t status;
    uint32_t rounds;
    uint64_t attempts;
    uint64_t losers;
    uint32_t max_active;
    uint32_t pad;
} pip_job_stats;

/* One array of a batch. */
typedef struct {
    void *A_dev;              /* device array of n elements (caller-owned) */
    const uint32_t *H_dev;    /* explicit targets, or NULL for hashed targets */
    uint64_t n;               /* < 2^32 */
    uint64_t seed;            /* hashed-target seed */
} pip_batch_item;

/* Launch plan of a batch (host struct, filled by pip_batch_plan_make). */
typedef struct {
    uint32_t count;
    uint32_t elem_bytes;
    uint32_t fmax;            /* largest per-array fresh block */
    uint32_t slot_factor;
    uint32_t block_threads;
    uint32_t max_blocks;      /* 0 = as many as fit */
    uint32_t any_explicit;
    uint32_t pad;
    uint64_t jobs_bytes;      /* device bytes of the job list (pip_batch_prepare) */
    uint64_t smem_bytes;      /* shared memory per block */
    uint64_t total_elems;
    double eps;
} pip_batch_plan;

/*
 * pip_shuffle -- in-place Knuth shuffle of A_dev[0..n) with hashed targets
 * H[i] = mulhi64(splitmix64(seed ^ i), i + 1) (Section 4.1, Theorem 4.2).
 *   A_dev : device array of n elements of `dtype`, aligned to the element size.
 *   n     : element count, n < 2^32.  n <= 1 is a no-op returning PIP_OK.
 *   eps   : 0 < eps < 1; the prefix is about n^(1-eps) swaps, the device
 *           scratch at most pip_aux_bytes(n, dtype, eps) bytes.
 *   stream: cudaStream_t (void*), NULL = default stream.
 * Allocates its scratch with cudaMallocAsync on `stream` and frees it the same
 * way.  Deterministic: equal arguments give equal output.
 */
pip_status pip_shuffle(void *A_dev, uint64_t n, pip_dtype dtype, uint64_t seed,
                       double eps, void *stream);

/*
 * pip_shuffle_explicit_h -- the same with caller-supplied targets
 * H_dev[0..n) (uint32, device, H_dev[0] ignored, 0 <= H_dev[i] <= i).  The
 * targets are validated on the device first; a violation leaves A untouched
 * and is reported as PIP_EINVAL by pip_check().  Used by the tests to drive
 * the kernels through every target sequence of small n and through the
 * closed-form worst cases (H = 0, H[i] = i-1).
 */
pip_status pip_shuffle_explicit_h(void *A_dev, uint64_t n, pip_dtype dtype,
                                  const uint32_t *H_dev, double eps, void *stream);

/*
 * pip_shuffle_ex -- full-control form of the two calls above.
 *   H_dev    : NULL for hashed targets (seed used), else explicit targets.
 *   opt      : host pointer to overrides, or NULL.
 *   aux_dev  : caller-provided device scratch of aux_bytes bytes (at least the
 *              plan's aux_bytes, 256-byte aligned), or NULL to allocate.
 *   stats_dev: device pointer to a pip_stats the kernel fills, or NULL.
 */
pip_status pip_shuffle_ex(void *A_dev, uint64_t n, pip_dtype dtype, uint64_t seed,
                          const uint32_t *H_dev, double eps, const pip_options *opt,
                          void *aux_dev, uint64_t aux_bytes, pip_stats *stats_dev,
                          void *stream);

/*
 * pip_shuffle_batch -- shuffles `count` independent arrays in one persistent
 * launch (spec batching pattern; each array is the method of Section
 * 4.1 with its own targets H_j[i] = mulhi64(splitmix64(seeds[j] ^ i), i+1)).
 *   A_devs, ns, seeds: host arrays of length count; A_devs[j] is a device
 *                      array of ns[j] elements of `dtype`.
 * Every array gets the same result as pip_shuffle(A_devs[j], ns[j], dtype,
 * seeds[j], eps).  Builds the job list on the host (synchronous copy), then
 * queues the launch on `stream`; the job list is freed stream-ordered.
 */
pip_status pip_shuffle_batch(void *const *A_devs, const uint64_t *ns, const uint64_t *seeds,
                             uint32_t count, pip_dtype dtype, double eps, void *stream);

/*
 * Graph-capturable batch in three calls:
 *   pip_batch_plan_make -- host-only planning of `items` (host array).
 *   pip_batch_prepare   -- writes the job list (largest array first) into
 *                          jobs_dev (plan->jobs_bytes device bytes, 256-byte
 *                          aligned); synchronous.
 *   pip_batch_run       -- queues the run on `stream`: a memset of the job
 *                          list's counters and one kernel launch (plus a
 *                          validation kernel when explicit targets are
 *                          present).  May be captured into a CUDA graph and
 *                          replayed; each replay shuffles every array again.
 *   stats_dev: NULL or a device array of plan->count pip_job_stats, indexed
 *              like `items`.
 */
pip_status pip_batch_plan_make(const pip_batch_item *items, uint32_t count, pip_dtype dtype, double eps,
                               const pip_options *opt, pip_batch_plan *out);
pip_status pip_batch_prepare(const pip_batch_item *items, const pip_batch_plan *plan,
                             const pip_options *opt, void *jobs_dev);
pip_status pip_batch_run(const pip_batch_plan *plan, void *jobs_dev, pip_job_stats *stats_dev,
                         void *stream);

/* ------------------------------------------------------------------ serving */

/* A request server (opaque). */
typedef struct pip_server pip_server;

/* Server tuning; zero fields keep the defaults. */
typedef struct {
    uint32_t max_resident;     /* requests on the device at once (default: one per tick block) */
    uint32_t rounds_per_tick;  /* cap on the rounds a request advances per tick (default: no cap) */
    uint32_t fresh_cap;        /* cap on a request's fresh block F (default 1024; one block each) */
    uint32_t slot_factor;      /* reservation slots per fresh swap (default 4) */
    uint32_t block_threads;    /* threads per block of the tick kernel (default 512) */
    uint32_t tick_us;          /* GPU time budget of one tick, shared by the resident requests (default 1000) */
    double prefix_c;           /* C in F = C * n^(1-eps) of tick requests (default 1) */
    uint32_t lanes;            /* large requests running at once on lanes, each on a stream of its own
                                  (default: CUDA_DEVICE_MAX_CONNECTIONS - 3, at most 16, i.e. 5 unless that
                                  variable raises the device's work queues above 8; PIP_SERVE_NO_LANES: none) */
    uint32_t lane_min_log2;    /* requests of at least 2^lane_min_log2 elements take a lane (default 22) */
    uint32_t lane_blocks;      /* cap on the grid blocks all lanes hold together (default: half of what the
                                  persistent grid can keep resident) */
    uint32_t pad;
} pip_serve_options;
#define PIP_SERVE_NO_LANES 0xFFFFFFFFu

/* Per-request record.  Times are host steady-clock nanoseconds. */
typedef struct {
    uint32_t status;
    uint32_t rounds;
    uint64_t attempts;
    uint64_t losers;
    uint64_t n;
    uint64_t charged_bytes;    /* array + scratch charged against the budget */
    int64_t submit_ns;
    int64_t admit_ns;
    int64_t done_ns;
    uint32_t ticks;            /* ticks the request was resident for */
    uint32_t fresh_per_round;
    uint32_t lane_launches;    /* 0: served by tick blocks; else launches on a lane (more than one when
                                  its blocks did not all meet at the start gate in time) */
    uint32_t pad;
} pip_req_stats;

/* Server-wide counters. */
typedef struct {
    uint64_t budget_bytes;
    uint64_t used_bytes;
    uint64_t peak_used_bytes;  /* never above budget_bytes */
    uint64_t submitted;
    uint64_t admitted;
    uint64_t completed;
    uint64_t ticks;
    uint32_t resident;
    uint32_t waiting;
    uint32_t tick_blocks;
    uint32_t fresh_cap;
    uint32_t status;           /* PIP_ECUDA once a tick failed */
    uint32_t lane_requests;    /* requests served on a lane so far */
    uint64_t tick_kernels;     /* tick launches (loop passes with resident tick requests) */
    uint64_t tick_wait_ns;     /* host time the loop spent waiting for tick launches to finish */
    uint64_t lane_launches;    /* lane launches, including relaunches after a start gate timed out */
    uint64_t lane_setup_ns;    /* host time the loop spent queueing lane launches */
} pip_serve_info;

/*
 * pip_serve_create -- starts a server on `device` with a device-memory budget.
 * A background thread repeats ticks: it admits waiting requests in arrival
 * order while budget_bytes allows, charging each request its array
 * (n * element bytes) plus its O(n^(1-eps)) scratch; it then advances every
 * resident request, most remaining work first, for a slice of the tick's
 * time budget in one launch (each request on one block, round state kept in
 * device memory between ticks), and retires finished ones.  Requests arriving meanwhile join at the next
 * tick, so their work overlaps on the device with the requests already
 * running (continuous batching).
 * Large requests (at least 2^lane_min_log2 elements, when their prefix is
 * large enough for several blocks) take a lane instead: the persistent grid
 * driver on a slice of the GPU -- about one block per thousand fresh swaps,
 * within the lanes' block budget -- launched on a low-priority stream next
 * to the ticks, so that such a request finishes in about the time the whole
 * grid would take instead of one block's.  A large request waiting for a
 * lane does not hold back smaller requests behind it.
 * The result of every request equals pip_shuffle on the same array, seed
 * and eps.
 */
pip_status pip_serve_create(pip_server **out, uint64_t device_budget_bytes, int device,
                            const pip_serve_options *opt);

/*
 * pip_serve_submit -- queues a request; never blocks on the GPU.
 *   A_dev: the caller's device array (caller-owned, must stay valid until the
 *          request is released), or NULL: the server allocates the array when
 *          the request is admitted and fills it with A[i] = i (16-byte
 *          records: {i, splitmix64(i)}).
 *   ticket: filled with the request's handle.
 * PIP_EINVAL if the request alone exceeds the budget.
 */
pip_status pip_serve_submit(pip_server *srv, void *A_dev, uint64_t n, pip_dtype dtype, uint64_t seed,
                            double eps, uint64_t *ticket);

/* pip_serve_poll -- PIP_EAGAIN while the request runs; once done, its status
 * (PIP_OK on success), the array pointer and the stats (both optional). */
pip_status pip_serve_poll(pip_server *srv, uint64_t ticket, void **A_out, pip_req_stats *st);

/* pip_serve_wait -- pip_serve_poll that blocks up to timeout_ms. */
pip_status pip_serve_wait(pip_server *srv, uint64_t ticket, uint32_t timeout_ms, void **A_out,
                          pip_req_stats *st);

/* pip_serve_next_done -- the ticket of a finished request not yet returned by
 * this call, in completion order; blocks up to timeout_ms (PIP_EAGAIN when
 * none finished in time).  Lets a client release each request as soon as it
 * is done, whatever the submission order. */
pip_status pip_serve_next_done(pip_server *srv, uint32_t timeout_ms, uint64_t *ticket);

/* pip_serve_release -- forgets a finished request, frees its array if the
 * server allocated it, and returns its charge to the budget. PIP_EAGAIN if
 * the request has not finished. */
pip_status pip_serve_release(pip_server *srv, uint64_t ticket);

/* pip_serve_info_get -- server counters. */
pip_status pip_serve_info_get(pip_server *srv, pip_serve_info *out);

/* pip_serve_destroy -- drops never-admitted requests, lets resident ones
 * finish, frees everything the server owns. */
pip_status pip_serve_destroy(pip_server *srv);

/*
 * pip_plan -- the plan pip_shuffle_ex would use for these arguments on the
 * current device (host only; queries device attributes, launches nothing).
 *   out : host pointer, filled on PIP_OK.
 */
pip_status pip_plan(uint64_t n, pip_dtype dtype, double eps, const pip_options *opt,
                    pip_plan_info *out);

/* pip_aux_bytes -- exact device scratch bytes pip_shuffle allocates for these
 * arguments with default options; 0 when n <= 1 or the arguments are invalid. */
uint64_t pip_aux_bytes(uint64_t n, pip_dtype dtype, double eps);

/*
 * pip_check -- synchronizes `stream`, then returns and clears the error latched
 * by device-side work on the current device (PIP_OK if none), or PIP_ECUDA if
 * the stream reported a CUDA error.
 */
pip_status pip_check(void *stream);

/*
 * pip_shuffle_noalloc -- pip_shuffle for callers that cannot allocate device
 * memory at call time (an application that reserved the whole GPU for its
 * own pool, a latency-critical path that must not enter the CUDA allocator,
 * code holding a lock the allocator may need).  The paper has no counterpart:
 * it is an interface for such callers, not part of the method.
 *   Same arguments, same result as pip_shuffle (hashed targets, persistent
 *   grid driver), but the scratch comes from a fixed 16 MiB device area
 *   compiled into the library, which a device holds from the first call on
 *   it until the process exits.  Nothing is allocated or freed.
 *   Requests whose plan needs more than 16 MiB of scratch (pip_plan with
 *   PIP_FLAG_FORCE_GRID reports the need as aux_bytes) return PIP_ETOOLARGE
 *   before anything is queued.
 *   A_dev must be device (or managed) memory of the current device: host
 *   memory, registered or not, returns PIP_EINVAL before anything is queued.
 *   Set-up: the first call on a device looks up the area's device address.
 *   Under CUDA's lazy module loading (the default) that lookup is also when
 *   the driver reserves the 16 MiB, so make the first call -- a call with
 *   n = 0 does only the set-up and returns -- before the application
 *   reserves the rest of the GPU's memory for itself, and before any stream
 *   capture.  If the area cannot be reserved then, the call returns
 *   PIP_ENOMEM (and the next call tries again).
 *   Each call clears the part of the area it uses; the area keeps the last
 *   call's contents.  All calls on a device share the area, so calls whose
 *   work overlaps on the GPU race and corrupt each other: order them on one
 *   stream.
 */
pip_status pip_shuffle_noalloc(void *A_dev, uint64_t n, pip_dtype dtype, uint64_t seed,
                               double eps, void *stream);

/*
 * pip_calibrate_swap_floor -- BENCHMARK-ONLY PROBE THAT DESTROYS ITS INPUT; not
 * a shuffle.  The paper has no counterpart; it is a tool for reading the round
 * drivers' speed and has no use in a program that wants its data.
 *   Performs the n-1 swaps A[i] <-> A[H[i]] (hashed targets of `seed`) all at
 *   once with no conflict resolution, so A ends up with unspecified content
 *   (its elements may be duplicated or lost).  Times taken around it give the
 *   cost of the bare data movement of a shuffle on this GPU: coalesced i-side
 *   accesses plus one random element access per swap, done as the round
 *   drivers' commit modes do it: mode PIP_FLOOR_EXCHANGE (0) exchanges A[i]
 *   into A[H[i]] with one atomic at L2 and stores the returned element at
 *   A[i]; mode PIP_FLOOR_LOADSTORE (1) loads both elements and stores both.
 *   Other modes return PIP_EINVAL.
 */
#define PIP_FLOOR_EXCHANGE 0
#define PIP_FLOOR_LOADSTORE 1
pip_status pip_calibrate_swap_floor(void *A_dev, uint64_t n, pip_dtype dtype, uint64_t seed, int mode,
                                    void *stream);

/*
 * pip_shuffle_host_stream -- shuffles `count` arrays held in host memory, in
 * order: array j (n elements of dtype at in_hosts[j]) is copied to the
 * device, shuffled as pip_shuffle(..., seeds[j], eps) would, and copied back
 * to out_hosts[j] (which may be in_hosts[j]).  A shuffle touches its whole
 * array, so its own copies cannot overlap it; array j's copies overlap the
 * shuffles of arrays j-1 and j+1 instead (device buffers used in turn,
 * separate streams for copies in, shuffles and copies out, ordered by
 * events; the shuffles run one at a time).  A buffer passes through copy
 * in, shuffle and copy out before it takes its next array, so four buffers
 * are used where there is room for them (three hold the pace only while
 * copy in + shuffle + copy out stays under three shuffles).
 *   in_hosts, out_hosts, seeds: host arrays of length count.  The arrays
 *              are independent: an input must not be another array's output
 *              (a copy in may run before an earlier array's copy out).  The copies
 *              are asynchronous and overlap only for page-locked host memory
 *              (cudaHostAlloc / cudaHostRegister); pageable memory works
 *              but serialises.  The host buffers must stay valid until
 *              `stream` reaches the end of the call.
 *   dev_buf  : NULL (min(count, 4) buffers allocated with cudaMallocAsync
 *              on `stream` and freed the same way), or caller device memory
 *              of at least min(count, 3) * round_up(n * elem, 256) bytes,
 *              256-byte aligned, of which min(count, 4) buffers are used
 *              when dev_bytes holds them.
 *   stream   : the caller's stream; the work starts after what is queued on
 *              it and `stream` waits for the last copy back, so pip_check(stream)
 *              reports completion and any device-side error.
 * Returns PIP_EINVAL for bad arguments (nothing queued), else the first
 * failure while queueing (after waiting for whatever was queued).
 */
pip_status pip_shuffle_host_stream(const void *const *in_hosts, void *const *out_hosts, const uint64_t *seeds,
                                   uint32_t count, uint64_t n, pip_dtype dtype, double eps, void *dev_buf,
                                   uint64_t dev_bytes, void *stream);

/* ------------------------------------------------------------ list contraction */

/* One node of a doubly-linked list (16 bytes): the indices of its neighbours,
 * PIP_LIST_NIL at the ends of a list. */
typedef struct {
    uint64_t prev;
    uint64_t next;
} pip_list_node;
#define PIP_LIST_NIL 0xFFFFFFFFFFFFFFFFull

/*
 * pip_list_contract -- in-place list contraction (Section 4.2, Algorithm 2),
 * made relaxed-PIP by the Decomposable Property: every round works on about
 * C * n^(1-eps) nodes, so the device scratch stays within
 * PIP_AUX_C * n^(1-eps) + 4096 bytes (no array indexed by node).
 *   nodes_dev: device array of n records (16-byte aligned) describing any
 *              number of acyclic doubly-linked lists over the nodes 0..n-1.
 *   n        : node count, n < 2^32 - 1.  n <= 1 is a no-op.
 * Node i has priority i.  Every node is spliced out of its list once both of
 * its current neighbours are NIL or larger (all local minima of a round at
 * once), and keeps in its record the two neighbours it had at that moment:
 * on return, record i holds the nearest nodes with a larger index before and
 * after i in its original list (PIP_LIST_NIL where there is none) -- the tree
 * edges of the contraction.  The result equals splicing the nodes out one at
 * a time in index order.
 * Errors (reported by pip_check()): a pointer out of range stops the run
 * with PIP_EINVAL before any access outside the array; a cycle is detected
 * when a round contracts nothing, PIP_EINTERNAL; in both cases the records
 * are then unspecified.  Other inconsistent input (prev and next not
 * matching) gives unspecified records.  With PIP_FLAG_VALIDATE_INPUT in
 * pip_list_contract_ex the whole input is checked first and rejected
 * untouched (PIP_EINVAL).
 * Scratch is allocated with cudaMallocAsync on `stream` and freed the same way.
 */
pip_status pip_list_contract(pip_list_node *nodes_dev, uint64_t n, double eps, void *stream);

/* pip_list_contract_ex -- the same with overrides (opt: prefix_c,
 * fresh_per_round, grid_blocks, block_threads up to 512, wait_timeout_ns),
 * caller-provided scratch (aux_dev of at least pip_list_plan's aux_bytes,
 * 256-byte aligned, or NULL) and a device pip_stats the kernel fills (or
 * NULL; attempts counts active nodes over all rounds, losers the nodes
 * carried to a next round). */
pip_status pip_list_contract_ex(pip_list_node *nodes_dev, uint64_t n, double eps, const pip_options *opt,
                                void *aux_dev, uint64_t aux_bytes, pip_stats *stats_dev, void *stream);

/*
 * pip_list_rank -- list ranking (Section 4.2): list contraction followed by
 * the reconstruction step, which distributes the values back down the tree
 * the contraction leaves, both on the relaxed-PIP round engine (about
 * C * n^(1-eps) nodes a round, the scratch of pip_list_plan).
 *   nodes_dev: as for pip_list_contract -- n records (prev, next), 16-byte
 *              aligned, any number of acyclic doubly-linked lists over
 *              0..n-1 -- overwritten with the result.
 *   n        : node count, n < 2^31 (distances travel in 32 bits).
 * On return (stream-ordered) record i holds (nodes before i in its list,
 * nodes after i in its list), two uint64; a list's length is their sum plus
 * one.  The contraction keeps, in each node's two words, its nearest larger
 * node on each side and the distance to it (the node index in the low 32
 * bits, the distance in the high 32 bits, while it runs); the reconstruction
 * then takes the nodes from the largest index down: nodes before i = nodes
 * before its nearest larger node on the left + the distance between them
 * (the distance minus one when there is none), and likewise after i.  The
 * result is unique, so it is bit-exact whatever the schedule.
 * Errors (pip_check): a pointer out of range gives PIP_EINVAL before any
 * access outside the array, a cycle PIP_EINTERNAL; the records are then
 * unspecified.  PIP_FLAG_VALIDATE_INPUT in pip_list_rank_ex checks the whole
 * input first and rejects it untouched (PIP_EINVAL).
 * Scratch is allocated with cudaMallocAsync on `stream` and freed the same way.
 */
pip_status pip_list_rank(pip_list_node *nodes_dev, uint64_t n, double eps, void *stream);

/* pip_list_rank_ex -- the same with the overrides, caller scratch (at least
 * pip_list_plan's aux_bytes, 256-byte aligned, or NULL) and device stats of
 * pip_list_contract_ex (rounds, attempts and losers are the contraction's;
 * status is the whole call's). */
pip_status pip_list_rank_ex(pip_list_node *nodes_dev, uint64_t n, double eps, const pip_options *opt,
                            void *aux_dev, uint64_t aux_bytes, pip_stats *stats_dev, void *stream);

/* pip_list_plan -- the plan pip_list_contract_ex would use (host only):
 * elem_bytes = 16, fresh_per_round, max_active, grid_blocks, block_threads,
 * aux_bytes, smem_bytes, aux_bound_bytes, min_rounds; driver = 3. */
pip_status pip_list_plan(uint64_t n, double eps, const pip_options *opt, pip_plan_info *out);

/* ------------------------------------------------------------ tree contraction */

/* One node of a forest of rooted binary trees (32 bytes): its parent and its
 * two children, PIP_TREE_NIL where there is none (a leaf has no children, a
 * root no parent, and every other node exactly two children); `round` is
 * written for raked leaves only (see pip_tree_contract). */
typedef struct {
    uint64_t parent;
    uint64_t left;
    uint64_t right;
    uint64_t round;
} pip_tree_node;
#define PIP_TREE_NIL 0xFFFFFFFFFFFFFFFFull

/*
 * pip_tree_contract -- in-place tree contraction (Section 4.2, the tree
 * contraction paragraph), relaxed-PIP by the Decomposable Property: every
 * round works on a prefix of about C * n^(1-eps) nodes in index order, so the
 * device scratch stays within PIP_AUX_C * n^(1-eps) + 4096 bytes.
 *   nodes_dev: device array of n records (32-byte aligned) describing a
 *              forest of rooted binary trees over the nodes 0..n-1 in which
 *              every internal node has two children.
 *   n        : node count, n < 2^32 - 1.  n <= 1 is a no-op.
 * Raking a leaf l with parent p removes l and p: the other child s of p takes
 * p's place under p's parent g (or becomes a root).  Node i has priority i.
 * Round r (from 1) works on the leaves carried from round r-1 plus the next
 * fn = min(F, nodes not yet admitted, kmax - m + 1) node indices, F and kmax
 * those of pip_tree_plan (fresh_per_round, max_active) and m the previous
 * round's active count; internal nodes and parentless leaves in it need no
 * work.  An active leaf with a parent is raked in the round exactly when no
 * leaf among its sibling, its nephews (the sibling's children) and its uncle
 * (the other child of its grandparent) has a smaller index, decided on the
 * state at the start of the round; so no two rakes of a round touch the same
 * word and no parent-child pair is contracted in one round.  On return every
 * tree has one leaf left, as a root; a raked leaf's record holds
 * (parent = p, left = s, right = g, round = r) as they were at its rake; a
 * removed internal node keeps the record it had when it was removed.  The
 * rounds (and so the result) depend on F and kmax only, never on the launch.
 * Errors (reported by pip_check()): a pointer out of range, or a parent that
 * does not list the node as a child, stops the run with PIP_EINVAL before
 * any access outside the array (the records are then unspecified).  Other
 * inconsistent input gives unspecified records.  With
 * PIP_FLAG_VALIDATE_INPUT in pip_tree_contract_ex the whole input is checked
 * first and rejected untouched (PIP_EINVAL).
 * Scratch is allocated with cudaMallocAsync on `stream` and freed the same way.
 */
pip_status pip_tree_contract(pip_tree_node *nodes_dev, uint64_t n, double eps, void *stream);

/* pip_tree_contract_ex -- the same with overrides (opt: prefix_c,
 * fresh_per_round, grid_blocks, block_threads up to 512, wait_timeout_ns,
 * flags), caller-provided scratch (aux_dev of at least pip_tree_plan's
 * aux_bytes, 256-byte aligned, or NULL) and a device pip_stats the kernel
 * fills (or NULL; attempts counts active nodes over all rounds, losers the
 * leaves carried to a next round). */
pip_status pip_tree_contract_ex(pip_tree_node *nodes_dev, uint64_t n, double eps, const pip_options *opt,
                                void *aux_dev, uint64_t aux_bytes, pip_stats *stats_dev, void *stream);

/* pip_tree_plan -- the plan pip_tree_contract_ex would use (host only):
 * elem_bytes = 32, fresh_per_round (F), max_active (kmax), grid_blocks,
 * block_threads, aux_bytes, smem_bytes, aux_bound_bytes, min_rounds;
 * driver = 4.  `slots` holds the on-chip phase-B cache per thread in bytes
 * (counted in smem_bytes): 12 per cached leaf when the leaf's parent, sibling
 * and grandparent are kept, 8 when only the last two are, 0 for no cache.
 * The results never depend on it. */
pip_status pip_tree_plan(uint64_t n, double eps, const pip_options *opt, pip_plan_info *out);

/* ------------------------------------------------------------ scan */

/*
 * pip_scan -- in-place exclusive prefix sum (Section 5.1, Algorithm 3): on
 * return A[i] = A[0] + ... + A[i-1] (A[0] = 0) with the addition of w-bit
 * unsigned integers modulo 2^w, and *total_dev (if not NULL) holds the sum of
 * all n inputs.
 *   A_dev    : device array of n elements, 16-byte aligned.
 *   dtype    : PIP_U32 or PIP_U64.
 *   total_dev: NULL or a device pointer to one element of dtype.
 * The auxiliary device memory is a constant pip_scan_aux_bytes() (64 KB),
 * whatever n (the space bound of the paper's strong PIP algorithm): a
 * control block and a ring of tile descriptors.  Allocated with
 * cudaMallocAsync on `stream` and freed the same way.  A bounded device-side
 * wait that runs out is reported as PIP_ETIMEOUT by pip_check() (A is then
 * unspecified).
 */
pip_status pip_scan(void *A_dev, uint64_t n, pip_dtype dtype, void *total_dev, void *stream);

/* pip_scan_ex -- the same with caller-provided scratch (aux_dev: at least
 * pip_scan_aux_bytes() device bytes, 256-byte aligned), or NULL to allocate. */
pip_status pip_scan_ex(void *A_dev, uint64_t n, pip_dtype dtype, void *total_dev, void *aux_dev,
                       uint64_t aux_bytes, void *stream);

/* pip_scan_aux_bytes -- the fixed scratch size of pip_scan_ex. */
uint64_t pip_scan_aux_bytes(void);

/* pip_status_string -- static English description of a status code. */
const char *pip_status_string(pip_status s);

/* pip_version -- library version string. */
const char *pip_version(void);

#ifdef __cplusplus
}
#endif

#endif /* PIP_H */
