// Host-side internals shared by the library's translation units.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "pip.h"

namespace pip {

// Byte layout of one shuffle's device scratch ("aux").  All offsets are
// 256-byte aligned.  Ctrl words come first so a single memset clears them
// together with the reservation tables.
struct Ctrl {
  uint32_t cnt[3];              // loser-queue allocators, rotating by round
  uint32_t status;              // first device-side error of this call
  unsigned long long barrier;   // monotone arrival counter (cluster driver)
  // Per-round barrier words of the grid driver, rotating by round: arriving
  // blocks, blocks that recorded an error, and the sums of the blocks' losers
  // and of the losers they could not keep on chip (field layout in
  // device.cuh).
  unsigned long long bw[3];
  // Start gate of a grid-driver launch that is not cooperative (a serving
  // lane): arriving blocks, and the decision (kGateGo / kGateAbort) taken by
  // the first block that sees all arrivals or runs out of time.
  uint32_t gate_count;
  uint32_t gate_decision;
  uint32_t lane_status;  // error latch of a lane launch (instead of the per-device one)
  uint32_t pad[49];
};
static_assert(sizeof(Ctrl) == 256, "ctrl block is one 256-byte line pair");

enum Driver : uint32_t { kDriverGrid = 0, kDriverCta = 1, kDriverCluster = 2 };

struct Plan {
  uint32_t driver = kDriverGrid;
  uint32_t sigma = 4;
  uint64_t smem_bytes = 0;  // on-chip scratch of the block-resident driver
  uint32_t n = 0;
  uint32_t elem_bytes = 0;
  double eps = 0.5;
  uint32_t F = 0;          // fresh swaps per round
  uint32_t kmax = 0;       // cap on active swaps per round
  uint32_t nslots = 0;     // reservation slots per table
  uint32_t blocks = 0;     // persistent grid blocks
  uint32_t threads = 0;    // threads per block
  uint32_t kloc = 0;       // grid driver: on-chip loser list capacity per block and round
  uint64_t timeout_ns = 0;
  uint64_t deadline_ns = 0;
  uint32_t flags = 0;
  // aux layout
  uint64_t off_S[3] = {0, 0, 0};
  uint64_t off_D[3] = {0, 0, 0};
  uint64_t off_Q[2] = {0, 0};
  uint64_t aux_bytes = 0;
  uint64_t aux_bound = 0;
};

// Kernel arguments of the persistent round driver.
struct GridArgs {
  void* A;
  const uint32_t* H;   // explicit targets, or nullptr for hashed targets
  uint64_t seed;
  uint32_t n;
  uint32_t F;
  uint32_t kmax;
  uint32_t nslots;
  uint32_t* S[3];
  uint32_t* D[3];      // window bitmaps: bit d set when an active swap targets location wlo + d
  uint32_t* Q[2];      // overflow queues: losers that did not fit their block's on-chip list
  uint32_t kloc;       // capacity of a block's on-chip loser list (shared memory holds two)
  Ctrl* ctrl;
  pip_stats* stats;    // may be nullptr
  uint64_t timeout_ns;
  uint32_t max_rounds;
  uint32_t flags;
  uint32_t* latch;     // per-device error latch
  uint64_t deadline_ns;  // whole-kernel time limit
  uint64_t gate_timeout_ns;  // > 0: blocks meet at a start gate first (non-cooperative launch)
};

// One array of a block-resident (batched) run.  40 bytes.
struct BatchJob {
  void* A;
  const uint32_t* H;   // explicit targets or nullptr
  uint64_t seed;
  uint32_t n;
  uint32_t F;          // fresh swaps per round for this array
  uint32_t slot;       // index of the array in the caller's list (stats)
  uint32_t pad;
};
static_assert(sizeof(BatchJob) == 40, "job layout");

// Device-resident header in front of the job list.  `next` and `status` are
// reset before every run (a 256-byte memset of the header's first line).
struct BatchHeader {
  uint32_t next;        // work counter: next job to take
  uint32_t status;      // first error of the run
  uint32_t count;
  uint32_t fmax;
  uint32_t sigma;
  uint32_t flags;       // PIP_FLAG_PREFETCH: one-round-ahead loads in every block
  uint64_t deadline_ns;
  uint32_t* latch;
  uint32_t pad[54];
};
static_assert(sizeof(BatchHeader) == 256, "header is 256 bytes");

// Round state of a request run in slices (serving), in device memory.  The
// frontier and the carried losers describe the next round completely.
struct ResumeState {
  uint32_t started;
  uint32_t done;
  uint32_t status;
  uint32_t rounds;
  uint32_t L;          // lowest activated step
  uint32_t Lprev;      // end of the current fresh block
  uint32_t nl;         // carried losers (in Q)
  uint32_t m;          // active swaps of the next round
  uint64_t attempts;
  uint64_t losers;
  uint32_t max_active;
  uint32_t pad;
  uint32_t* Q;         // carried-loser queue, at least cta_kmax(F) words
};

struct BatchLaunch {
  BatchHeader* hdr;
  BatchJob* jobs;
  pip_job_stats* stats;
  uint32_t count;
  uint32_t elem_bytes;
  uint32_t fmax;
  uint32_t sigma;
  uint32_t threads;
  uint32_t max_blocks;
  bool any_explicit;
};

// Block-resident driver (cta_driver.cu).  A run with fresh block F keeps at
// most cta_kmax(F) swaps active: the next fresh block is sized once the
// round's losers are known, so the cap only leaves F/4 of room for them
// before the fresh block shrinks.
__host__ __device__ __forceinline__ uint32_t cta_kmax(uint32_t F) { return F + F / 4u + 2u; }
__host__ __device__ __forceinline__ uint32_t cta_window_words(uint32_t F) { return (((F + 31u) >> 5) + 3u) & ~3u; }
// Words of the slot table for fresh blocks up to fmax, a multiple of 4 so
// that the window bitmap after it stays 16-byte aligned.
__host__ __device__ __forceinline__ uint32_t cta_table_words(uint32_t fmax, uint32_t sigma) {
  return (sigma * fmax + 32u + 3u) & ~3u;
}
uint64_t cta_smem_bytes(uint32_t fmax, uint32_t sigma);
uint32_t cta_max_fmax(uint32_t sigma);
pip_status launch_cta_driver(const BatchLaunch& bl, cudaStream_t stream);
// One array on one block (small prefixes): validation (explicit targets) and
// the kernel, on `stream`; `aux` holds the 256-byte Ctrl block.
pip_status launch_cta_single(const Plan& plan, void* A, const uint32_t* H, uint64_t seed, void* aux,
                             pip_stats* stats, cudaStream_t stream);

// Cluster driver (cluster_driver.cu): shared memory per CTA for a cluster of
// `cs` CTAs and fresh block F; whether such a launch fits on this device;
// the launch itself (plan.blocks = cluster size).
uint64_t cluster_cta_smem(uint32_t F, uint32_t sigma, uint32_t cs);
bool cluster_supported(uint32_t elem_bytes, uint32_t cs, uint32_t threads, uint64_t smem);
pip_status launch_cluster_driver(const Plan& plan, void* A, const uint32_t* H, uint64_t seed, void* aux,
                                 pip_stats* stats, cudaStream_t stream);

// List contraction (list_driver.cu): plan and launch.
struct ListPlan {
  uint32_t n = 0;
  uint32_t F = 0;        // fresh nodes per round
  uint32_t kmax = 0;     // cap on active nodes per round
  uint32_t kloc = 0;     // on-chip carried-node list per block
  uint32_t blocks = 0;
  uint32_t threads = 0;
  uint32_t flags = 0;
  uint64_t timeout_ns = 0;
  uint64_t deadline_ns = 0;
  uint64_t off_Q[2] = {0, 0};
  uint64_t aux_bytes = 0;
  uint64_t smem_bytes = 0;  // all blocks' on-chip lists and caches (counted in the bound)
  uint64_t aux_bound = 0;
  uint32_t cache_per_thread = 0;  // bytes of on-chip cache per thread (tree contraction)
  uint32_t cache_slot_bytes = 0;  // bytes per cached slot (tree contraction: 8 or 12)
  uint64_t block_smem() const { return 8ull * kloc + (uint64_t)cache_per_thread * threads; }
};
// The shape of a round-engine plan depends on its kernel's occupancy:
// blocks_per_sm(threads, dynamic shared bytes) gives it (the list kernel's
// when null); cache_per_thread adds on-chip bytes per thread to each block.
pip_status make_list_plan(uint64_t n, double eps, const pip_options* opt, ListPlan* out,
                          int (*blocks_per_sm)(uint32_t threads, uint64_t smem) = nullptr,
                          uint32_t cache_per_thread = 0);
pip_status launch_list_driver(const ListPlan& plan, void* rec, void* aux, pip_stats* stats, cudaStream_t stream);

// Tree contraction (tree_driver.cu): the plan is a ListPlan made with the
// tree kernel's occupancy.
pip_status make_tree_plan(uint64_t n, double eps, const pip_options* opt, ListPlan* out);
pip_status launch_tree_driver(const ListPlan& plan, void* rec, void* aux, pip_stats* stats, cudaStream_t stream);

// Scan (scan.cu): bytes of the fixed scratch (control block and descriptor ring).
uint64_t scan_aux_bytes();

// Device facts cached per device.
struct DeviceInfo {
  int sms = 0;
  int max_threads_per_sm = 0;
  size_t l2_bytes = 0;
};
pip_status device_info(DeviceInfo* out);

// Planner (planner.cpp).
pip_status make_plan(uint64_t n, pip_dtype dtype, double eps, const pip_options* opt, Plan* out);
// Fresh-per-round F of one array run by the block-resident driver, within the
// aux bound and the shared-memory cap.
uint32_t cta_fresh(uint64_t n, double eps, const pip_options* opt, uint32_t sigma, uint32_t fcap);
// Bytes the block-resident driver holds for one array with fresh block F.
uint64_t cta_job_bytes(uint32_t F, uint32_t sigma);
uint32_t elem_bytes_of(pip_dtype dtype);

// Round driver launch (grid_driver.cu).  Queues the explicit-target
// validation (if H is given), then the persistent kernel, on `stream`.
pip_status launch_grid_driver(const Plan& plan, void* A, const uint32_t* H, uint64_t seed,
                              void* aux, pip_stats* stats, cudaStream_t stream);
// The same persistent grid driver launched without the cooperative attribute,
// for a serving lane that runs next to other kernels: `plan.blocks` blocks
// first meet at a start gate, and if they are not all resident within
// `gate_timeout_ns` every block leaves before touching the array or the
// tables, and the run reports PIP_EBUSY (it can simply be launched again).
// Errors go to the launch's own status word in the Ctrl block (and to
// `stats`), not to the per-device latch.
pip_status launch_grid_lane(const Plan& plan, void* A, uint64_t seed, void* aux, pip_stats* stats,
                            uint64_t gate_timeout_ns, cudaStream_t stream);
// Device address of the per-device error latch (current device), or nullptr.
uint32_t* error_latch_ptr();
// Reads and clears the latch of the current device (synchronous).
pip_status take_error_latch(uint32_t* value);

// Largest co-resident block count for the driver with this element size and
// block size (cached per device).
uint32_t grid_driver_max_blocks(uint32_t elem_bytes, bool explicit_h, uint32_t threads, uint32_t kloc);
// Shared memory of one grid-driver block: two on-chip loser lists of kloc words.
inline uint64_t grid_block_smem(uint32_t kloc) { return 8ull * kloc; }

}  // namespace pip
