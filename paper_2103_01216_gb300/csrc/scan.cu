// In-place exclusive scan (Section 5.1, Algorithm 3: the output of
// In-Place-Scan, exclusive prefix sums and the total, computed in place with
// only a bounded amount of auxiliary space).
//
// The GPU design is a single pass over the array in tiles with decoupled
// look-back: block b of a grid of G resident blocks takes tiles b, b + G,
// ..., each moved into shared memory by a bulk asynchronous copy
// (cp.async.bulk completing on an mbarrier), two or three copies ahead.  The
// block is warp-specialised:
//   - the scanning warps read tile i into registers (which frees its
//     buffer), scan it, publish its sum in a descriptor and hand the sum to
//     the look-back warp through an mbarrier; kDefer tiles later they add
//     the prefix the look-back warp handed back, write the tile to a staging
//     buffer and send it out with a bulk copy;
//   - the look-back warp derives each tile's exclusive prefix from its
//     predecessors' descriptors (32 per L2 round trip) and publishes the
//     inclusive prefix.
// The two roles meet only at the mbarriers of one tile, so a look-back can
// take kDefer tiles' time before the scanning warps wait for it, and each
// element is read once and written once: the pass is bound by HBM bandwidth.
//
// The descriptors form a ring of kRing entries reused modulo kRing, tagged
// with the tile index.  A block publishes the sum of its local tile i only
// after the look-back of its tile i - 1 - kDefer has ended, and a look-back
// never reads further back than its block's previous tile (whose prefix was
// published before it started).  While one look-back waits, no block can get
// more than (kDefer + 1) G tiles past its first missing sum, so the indices
// read or written at one time span fewer than (2 kDefer + 3) G; a ring of
// (2 kDefer + 4) G or more is never overwritten while it is read.  The
// auxiliary space is therefore a constant (the ring and a control block,
// 64 KB), whatever n -- the space bound of the paper's strong PIP algorithm.
//
// Addition is modulo 2^w (w = 32 or 64), which is associative, so the result
// does not depend on the order in which partial sums are combined: the
// output is bit-identical to the sequential definition.
#include <algorithm>
#include <cstdint>
#include <map>
#include <mutex>

#include "device.cuh"
#include "internal.h"

namespace pip {
namespace {

// Shape (one block per SM): PIP_SCAN_THREADS scanning threads plus the
// look-back warp; per element size a tile size and a number of tile buffers
// (all but one for loads, one staging tile for the stores), and the
// deferral: tiles between a tile's scan and its finish.  Measured on GB300
// at 10^9 elements (fraction of the HBM copy bandwidth, u64 / u32):
//   40 KB x 5, deferral 2: 86 / 87 %   48 KB x 4, deferral 2: 82 / 89 %
//   56 KB x 4, deferral 1: 85 / 84 %   56 KB x 4, deferral 2: 81 / 85 %
//   48 KB x 4, deferral 1: 78 / 81 %   32 KB x 6, deferral 2: 62 / 66 %
// (two deferred tiles of 56 KB spill registers at u64; 512 scanning threads
// keep a thread's 16-byte shared-memory accesses free of bank conflicts).
#ifndef PIP_SCAN_THREADS
#define PIP_SCAN_THREADS 512
#endif
#ifdef PIP_SCAN_TILE_KB
#define PIP_SCAN_TILE_KB_4 PIP_SCAN_TILE_KB
#define PIP_SCAN_TILE_KB_8 PIP_SCAN_TILE_KB
#endif
#ifdef PIP_SCAN_STAGES
#define PIP_SCAN_STAGES_4 PIP_SCAN_STAGES
#define PIP_SCAN_STAGES_8 PIP_SCAN_STAGES
#endif
#ifndef PIP_SCAN_TILE_KB_4
#define PIP_SCAN_TILE_KB_4 48
#endif
#ifndef PIP_SCAN_STAGES_4
#define PIP_SCAN_STAGES_4 4
#endif
#ifndef PIP_SCAN_TILE_KB_8
#define PIP_SCAN_TILE_KB_8 40
#endif
#ifndef PIP_SCAN_STAGES_8
#define PIP_SCAN_STAGES_8 5
#endif
#ifndef PIP_SCAN_LB_PER_LANE
#define PIP_SCAN_LB_PER_LANE 1
#endif
#ifndef PIP_SCAN_POLL_NS
#define PIP_SCAN_POLL_NS 64
#endif
constexpr uint32_t kScanThreads = PIP_SCAN_THREADS;     // scanning threads
constexpr uint32_t kBlockThreads = kScanThreads + 32u;  // and the look-back warp
#ifndef PIP_SCAN_DEFER
#define PIP_SCAN_DEFER 2
#endif
constexpr uint32_t kDefer = PIP_SCAN_DEFER;  // tiles between a tile's scan and its finish
constexpr uint32_t kSlots = 4;               // hand-over slots between the two warp roles
constexpr uint32_t kLbPerLane = PIP_SCAN_LB_PER_LANE;

// The tile shape of one element type.
template <typename T>
struct ScanShape {
  static constexpr uint32_t kTileBytes = (sizeof(T) == 4 ? PIP_SCAN_TILE_KB_4 : PIP_SCAN_TILE_KB_8) * 1024u;
  static constexpr uint32_t kStages = sizeof(T) == 4 ? PIP_SCAN_STAGES_4 : PIP_SCAN_STAGES_8;  // tile buffers
  static constexpr uint32_t kLoadBufs = kStages - 1u;  // tiles loading or being read
  static constexpr uint32_t kAhead = kLoadBufs - 1u;   // copies in flight ahead
  static constexpr uint32_t kSmemBytes = kStages * kTileBytes;
  static_assert(kStages >= 3, "at least one copy ahead");
};
constexpr uint32_t kRing = 4096;  // descriptors, a power of two
constexpr uint64_t kFlagAgg = 1, kFlagPrefix = 2;
constexpr uint32_t kBarScan = 1;  // named barrier of the scanning threads
static_assert(kScanThreads % 32u == 0 && kBlockThreads <= 1024u, "scan shape");
static_assert(kDefer >= 1 && kSlots >= kDefer + 2, "hand-over slots outlast the deferral");

struct ScanCtrl {
  unsigned long long unused;
  uint32_t status;  // first error of this call
  uint32_t pad[61];
};
static_assert(sizeof(ScanCtrl) == 256, "scan control block is 256 bytes");

// A tile's descriptor is two 64-bit words, one per 32-bit half of the value,
// each holding [tile tag : 24][flag : 2][unused : 6][half : 32].  A word is
// written and read as one 64-bit access, so a reader that finds the expected
// tag and the same flag in both words has a consistent value without any
// fence; a torn pair (one word updated from "aggregate" to "prefix" before
// the other) simply fails the check and is read again.  The tag is the tile
// index modulo 2^24, enough to tell apart the tiles that share a ring slot
// while any of them is in flight.
constexpr uint32_t kTagBits = 24;
constexpr uint64_t kTagMask = (1ull << kTagBits) - 1ull;

struct __align__(16) ScanDesc {
  unsigned long long w[2];
};

__device__ __forceinline__ unsigned long long desc_word(uint64_t tile, uint64_t flag, uint32_t half) {
  return ((tile & kTagMask) << 40) | (flag << 38) | (unsigned long long)half;
}

// Descriptor words are written and read with relaxed gpu-scope accesses: a
// tile's sum and its prefix are written by two threads of one block ordered
// by a barrier, and such strong accesses keep that order in every reader's
// view of the word.
__device__ __forceinline__ void st_relaxed_u64(unsigned long long* p, unsigned long long v) {
  asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

template <typename T>
__device__ __forceinline__ void desc_publish(ScanDesc* d, uint64_t tile, uint64_t flag, T value) {
  const unsigned long long v = (unsigned long long)value;
  st_relaxed_u64(&d->w[1], desc_word(tile, flag, (uint32_t)(v >> 32)));
  st_relaxed_u64(&d->w[0], desc_word(tile, flag, (uint32_t)v));
}

// 0 when the descriptor does not (yet) describe `tile`; else its flag, with
// the value in *value.
// A window read takes each descriptor with one 16-byte load at L2
// (kStrong = false): it may tear between the two words or return an older
// state of a word, but a torn pair fails the tag / flag check and is read
// again, and an older state is the tile's sum where its prefix is already
// out -- still a correct value, the walk just goes further back.  The
// single-lane poll of one descriptor (kStrong = true) uses relaxed loads,
// which the compiler may not hoist out of the polling loop.
template <typename T, bool kStrong = false>
__device__ __forceinline__ uint64_t desc_read(const ScanDesc* d, uint64_t tile, T* value) {
  unsigned long long a, b;
  if (!kStrong) {
    const ulonglong2 ab = __ldcg(reinterpret_cast<const ulonglong2*>(d));
    a = ab.x;
    b = ab.y;
  } else {
    a = ld_relaxed_u64(&d->w[0]);
    b = ld_relaxed_u64(&d->w[1]);
  }
  const uint64_t tag = tile & kTagMask;
  if ((a >> 40) != tag || (b >> 40) != tag) return 0;
  const uint64_t fa = (a >> 38) & 3ull, fb = (b >> 38) & 3ull;
  if (fa != fb) return 0;
  *value = (T)(((unsigned long long)(uint32_t)b << 32) | (uint32_t)a);
  return fa;
}

// ---- bulk asynchronous copies and the mbarrier they complete on
__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
               : "memory");
}
// Waits for the given phase of the mbarrier, bounded: false when it gave up.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t phase, uint64_t timeout_ns) {
  uint64_t t0 = 0;
  for (uint32_t k = 0;; ++k) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
        : "=r"(done)
        : "r"(smem_addr(bar)), "r"(phase)
        : "memory");
    if (done) return true;
    if ((k & 63u) == 63u) {
      const uint64_t now = globaltimer_ns();
      if (t0 == 0) t0 = now;
      else if (now - t0 > timeout_ns) return false;
    }
  }
}
__device__ __forceinline__ void bulk_load(void* dst_smem, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_addr(dst_smem)),
               "l"(src), "r"(bytes), "r"(smem_addr(bar))
               : "memory");
}
__device__ __forceinline__ void bulk_store(void* dst, const void* src_smem, uint32_t bytes) {
  asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(dst), "r"(smem_addr(src_smem)),
               "r"(bytes)
               : "memory");
  asm volatile("cp.async.bulk.commit_group;" ::: "memory");
}
// Until the shared-memory source of every committed bulk store has been read.
__device__ __forceinline__ void bulk_wait_read() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }
// Orders this thread's ordinary shared-memory writes before later bulk-copy
// reads of that memory.
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

template <typename T>
__device__ __forceinline__ T warp_incl_scan(T v, uint32_t lane) {
#pragma unroll
  for (uint32_t d = 1; d < 32; d <<= 1) {
    const T u = __shfl_up_sync(0xffffffffu, v, d);
    if (lane >= d) v += u;
  }
  return v;
}

// The look-back warp's part of a tile: the decoupled look-back.  Lane k reads
// the descriptors of tiles top-kQ-q (q < kLbPerLane), 32 * kLbPerLane
// predecessors per window (their loads are independent, so a window costs
// one L2 latency), and the warp adds them from the top down to the nearest
// published inclusive prefix.  A window that is ready only in part still
// counts: its ready run from the top is added, and then lane 0 alone polls
// the first descriptor that was not ready (with a short sleep between
// polls, so that spinning warps do not crowd the L2 lines their
// predecessors are publishing to) before the next window starts there.
// Returns the exclusive prefix of tile t (in every lane), or sets *fail.
template <typename T>
__device__ __forceinline__ T look_back(const ScanDesc* ring, uint64_t t, uint32_t lane, ScanCtrl* ctrl,
                                       uint64_t timeout_ns, uint32_t* fail) {
  T prefix = 0;
  int64_t top = (int64_t)t - 1;  // highest predecessor not yet accounted for
  uint64_t t0 = 0;
  while (top >= 0) {
    uint64_t flag[kLbPerLane];
    T val[kLbPerLane];
#pragma unroll
    for (uint32_t q = 0; q < kLbPerLane; ++q) {
      const int64_t j = top - (int64_t)(lane * kLbPerLane + q);
      flag[q] = kFlagAgg;  // below tile 0: ready aggregates of 0
      val[q] = 0;
      if (j >= 0) flag[q] = desc_read<T>(ring + (j & (kRing - 1)), (uint64_t)j, &val[q]);
    }
    // this lane's ready run from its top: cnt descriptors, ending at a
    // prefix when found
    uint32_t cnt = kLbPerLane;
    bool found = false;
#pragma unroll
    for (int q = (int)kLbPerLane - 1; q >= 0; --q) {
      if (flag[q] == 0) {
        cnt = (uint32_t)q;
        found = false;
      } else if (flag[q] == kFlagPrefix) {
        cnt = (uint32_t)q + 1u;
        found = true;
      }
    }
    // the first lane that stops the run (a gap or a prefix) bounds the
    // window: lanes before it contribute everything, it contributes cnt
    const unsigned full = __ballot_sync(0xffffffffu, cnt == kLbPerLane && !found);
    const uint32_t last = full == 0xffffffffu ? 32u : (uint32_t)(__ffs(~full) - 1);
    const uint32_t last_cnt = last < 32u ? __shfl_sync(0xffffffffu, cnt, last) : 0u;
    const bool done = last < 32u && __shfl_sync(0xffffffffu, (uint32_t)found, last) != 0u;
    T v = 0;
    const uint32_t take = lane < last ? kLbPerLane : (lane == last ? last_cnt : 0u);
#pragma unroll
    for (uint32_t q = 0; q < kLbPerLane; ++q)
      if (q < take) v += val[q];
#pragma unroll
    for (uint32_t d = 16; d >= 1; d >>= 1) v += __shfl_xor_sync(0xffffffffu, v, d);
    prefix += v;
    if (done) break;
    top -= (int64_t)(last * kLbPerLane + last_cnt);
    if (last == 32u || top < 0) continue;  // the whole window was ready
    // lane 0 waits for descriptor `top` (bounded), then the warp goes on
    uint32_t bad = 0;
    if (lane == 0) {
      T unused;
      for (uint32_t k = 0; desc_read<T, true>(ring + (top & (kRing - 1)), (uint64_t)top, &unused) == 0; ++k) {
        if (PIP_SCAN_POLL_NS > 0) __nanosleep(PIP_SCAN_POLL_NS);
        if ((k & 15u) == 15u) {
          if (ld_relaxed_u32(&ctrl->status) != 0u) {
            bad = 1;
            break;
          }
          const uint64_t now = globaltimer_ns();
          if (t0 == 0) t0 = now;
          else if (now - t0 > timeout_ns) {
            set_status(&ctrl->status, PIP_ETIMEOUT);
            bad = 1;
            break;
          }
        }
      }
    }
    if (__shfl_sync(0xffffffffu, bad, 0)) {
      *fail = 1u;
      return 0;
    }
  }
  return prefix;
}

__device__ __forceinline__ void named_sync(uint32_t id, uint32_t count) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(count) : "memory");
}

// mbarrier arrive (one arrival; the phase completes with it).
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}

// One pass over tiles of kItems elements, kPer consecutive elements per
// scanning thread.  Block b takes its m tiles b, b + G, ... (G = grid size,
// every block resident).  Local tile i arrives in load buffer i % kLoadBufs
// (kAhead copies ahead); the scanning threads read it into registers (which
// frees the buffer), scan it, publish its sum and hand the sum to the
// look-back warp (mbarrier agg[i % kSlots]).  Tile i is finished kDefer tiles
// later, once the look-back warp has handed back its prefix (mbarrier
// pre[i % kSlots]): the prefix is added to the values still held in
// registers, written to the staging buffer and stored with a bulk copy.  So a
// tile's look-back may take up to kDefer tiles' time before the scanning
// threads wait for it.  Every wait is bounded; a failed one changes no
// arrival and no copy (the output is then unspecified), so no wait on the
// other side runs into its own limit because of it.
template <typename T>
__global__ void __launch_bounds__(kBlockThreads, 1)
    scan_kernel(T* A, uint64_t n, T* total_out, ScanCtrl* ctrl, ScanDesc* ring, uint64_t timeout_ns,
                uint32_t* latch) {
  constexpr uint32_t kTileBytes = ScanShape<T>::kTileBytes;
  constexpr uint32_t kLoadBufs = ScanShape<T>::kLoadBufs;
  constexpr uint32_t kAhead = ScanShape<T>::kAhead;
  constexpr uint32_t kItems = kTileBytes / sizeof(T);
  constexpr uint32_t kPer = kItems / kScanThreads;
  constexpr uint32_t kVec = 16u / sizeof(T);  // elements per 16-byte access
  static_assert(kPer * kScanThreads == kItems && kPer % kVec == 0, "tile shape");
  extern __shared__ __align__(128) unsigned char s_raw[];
  T* const s_load = reinterpret_cast<T*>(s_raw);   // kLoadBufs tiles
  T* const s_stage = s_load + kLoadBufs * kItems;  // one tile, source of the bulk stores
  __shared__ __align__(8) uint64_t s_bar_load[kLoadBufs];
  __shared__ __align__(8) uint64_t s_bar_agg[kSlots];
  __shared__ __align__(8) uint64_t s_bar_pre[kSlots];
  __shared__ T s_warp[kScanThreads / 32u];
  __shared__ T s_agg[kSlots];  // tile sums, scanning threads -> look-back warp
  __shared__ T s_pre[kSlots];  // tile prefixes, look-back warp -> scanning threads
  const uint32_t tid = threadIdx.x, lane = tid & 31u, warp = tid >> 5;
  const uint64_t ntiles = (n + kItems - 1) / kItems;
  const uint64_t G = gridDim.x, blk = blockIdx.x;
  const uint64_t m = blk < ntiles ? (ntiles - 1 - blk) / G + 1 : 0;  // this block's tiles
  if (tid == 0) {
    for (uint32_t q = 0; q < kLoadBufs; ++q) mbar_init(&s_bar_load[q], 1);
    for (uint32_t q = 0; q < kSlots; ++q) {
      mbar_init(&s_bar_agg[q], 1);
      mbar_init(&s_bar_pre[q], 1);
    }
  }
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  __syncthreads();

  if (warp == kScanThreads / 32u) {
    // ---- the look-back warp: tile i's sum in, tile i's prefix out
    bool failed = false;
    for (uint64_t i = 0; i < m; ++i) {
      const uint32_t slot = (uint32_t)(i % kSlots), par = (uint32_t)((i / kSlots) & 1u);
      // lane 0 waits for the sum (the arrive releases it, the wait acquires
      // it) and hands it to the other lanes
      uint32_t ok = 1;
      T agg = 0;
      if (lane == 0) {
        ok = mbar_wait(&s_bar_agg[slot], par, timeout_ns) ? 1u : 0u;
        agg = s_agg[slot];
      }
      ok = __shfl_sync(0xffffffffu, ok, 0);
      agg = __shfl_sync(0xffffffffu, agg, 0);
      if (!ok) {
        if (lane == 0) set_status(&ctrl->status, PIP_ETIMEOUT);
        failed = true;
      }
      const uint64_t t = blk + i * G;
      T prefix = 0;
      if (t > 0 && !failed) {
        uint32_t fail = 0;
        prefix = look_back<T>(ring, t, lane, ctrl, timeout_ns, &fail);
        failed = fail != 0u;
        if (!failed && lane == 0) desc_publish<T>(ring + (t & (kRing - 1)), t, kFlagPrefix, (T)(prefix + agg));
      }
      if (lane == 0) {
        s_pre[slot] = prefix;
        if (t == ntiles - 1 && total_out != nullptr) stcg(total_out, (T)(prefix + agg));
        mbar_arrive(&s_bar_pre[slot]);
      }
      __syncwarp();
    }
    return;
  }

  // ---- the scanning threads
  auto full_tile = [&](uint64_t u) { return (u + 1) * kItems <= n; };
  // thread 0 issues every copy (bulk groups are per thread)
  auto start_load = [&](uint64_t i) {
    const uint64_t u = blk + i * G;
    if (i < m && full_tile(u)) {
      uint64_t* bar = &s_bar_load[i % kLoadBufs];
      mbar_expect_tx(bar, kTileBytes);
      bulk_load(s_load + (i % kLoadBufs) * kItems, A + u * kItems, kTileBytes, bar);
    }
  };
  if (tid == 0)
    for (uint32_t i = 0; i < kAhead; ++i) start_load(i);
  // values of the tiles waiting for their prefix: vd[0] the newest
  T vd[kDefer + 1][kPer];
  T offd[kDefer + 1];
  uint64_t td[kDefer + 1];
#pragma unroll
  for (uint32_t d = 0; d <= kDefer; ++d) {
    offd[d] = 0;
    td[d] = 0;
  }
  for (uint64_t i = 0; i < m + kDefer; ++i) {
    // the staging buffer's last bulk store has read it (it is written below,
    // after a barrier of the scanning threads)
    if (tid == 0) bulk_wait_read();
    // shift the pending tiles: slot 0 takes tile i, slot kDefer is finished now
#pragma unroll
    for (uint32_t d = kDefer; d >= 1; --d) {
#pragma unroll
      for (uint32_t k = 0; k < kPer; ++k) vd[d][k] = vd[d - 1][k];
      offd[d] = offd[d - 1];
      td[d] = td[d - 1];
    }
    if (i < m) {
      const uint64_t t = blk + i * G;
      const uint64_t base = t * kItems;
      // the buffer of tile i + kAhead last held tile i - 1, whose reads all
      // ended before the barrier of the previous step
      if (tid == 0) start_load(i + kAhead);
      T run = 0;
      if (full_tile(t)) {
        if (!mbar_wait(&s_bar_load[i % kLoadBufs], (uint32_t)((i / kLoadBufs) & 1u), timeout_ns))
          set_status(&ctrl->status, PIP_ETIMEOUT);
        const uint4* src = reinterpret_cast<const uint4*>(s_load + (i % kLoadBufs) * kItems + tid * kPer);
#pragma unroll
        for (uint32_t q = 0; q < kPer / kVec; ++q) {
          const uint4 w = src[q];
          const T* e = reinterpret_cast<const T*>(&w);
#pragma unroll
          for (uint32_t k = 0; k < kVec; ++k) {
            vd[0][q * kVec + k] = run;
            run += e[k];
          }
        }
      } else {  // the ragged last tile, read with plain loads
#pragma unroll
        for (uint32_t k = 0; k < kPer; ++k) {
          const uint64_t g = base + tid * kPer + k;
          vd[0][k] = run;
          if (g < n) run += ldcg(A + g);
        }
      }
      const T incl = warp_incl_scan(run, lane);
      if (lane == 31u) s_warp[warp] = incl;
      named_sync(kBarScan, kScanThreads);
      T woff = 0, agg = 0;
#pragma unroll
      for (uint32_t w = 0; w < kScanThreads / 32u; ++w) {
        const T x = s_warp[w];
        agg += x;
        if (w < warp) woff += x;
      }
      offd[0] = woff + (incl - run);
      td[0] = t;
      if (tid == 0) {
        desc_publish<T>(ring + (t & (kRing - 1)), t, t == 0 ? kFlagPrefix : kFlagAgg, agg);
        s_agg[i % kSlots] = agg;
        mbar_arrive(&s_bar_agg[i % kSlots]);
      }
      // s_warp is read by every scanning thread before it is written again
      named_sync(kBarScan, kScanThreads);
    } else {
      named_sync(kBarScan, kScanThreads);  // the staging buffer is free (thread 0 waited)
    }
    if (i >= kDefer) {
      // finish tile j = i - kDefer with the prefix the look-back warp found
      const uint64_t j = i - kDefer;
      const uint32_t slot = (uint32_t)(j % kSlots);
      if (!mbar_wait(&s_bar_pre[slot], (uint32_t)((j / kSlots) & 1u), timeout_ns))
        set_status(&ctrl->status, PIP_ETIMEOUT);
      const T add = s_pre[slot] + offd[kDefer];
      const uint64_t tj = td[kDefer];
      const uint64_t base = tj * kItems;
      if (full_tile(tj)) {
        uint4* dst = reinterpret_cast<uint4*>(s_stage + tid * kPer);
#pragma unroll
        for (uint32_t q = 0; q < kPer / kVec; ++q) {
          uint4 w;
          T* e = reinterpret_cast<T*>(&w);
#pragma unroll
          for (uint32_t k = 0; k < kVec; ++k) e[k] = vd[kDefer][q * kVec + k] + add;
          dst[q] = w;
        }
        fence_proxy_async();
        named_sync(kBarScan, kScanThreads);
        if (tid == 0) bulk_store(A + base, s_stage, kTileBytes);
      } else {
#pragma unroll
        for (uint32_t k = 0; k < kPer; ++k) {
          const uint64_t g = base + tid * kPer + k;
          if (g < n) stcg(A + g, (T)(vd[kDefer][k] + add));
        }
      }
    }
  }
  if (tid == 0) {
    bulk_wait_all();
    const uint32_t st = ld_relaxed_u32(&ctrl->status);
    if (st != 0u) atomicCAS(latch, 0u, st);
  }
}

template <typename T>
int scan_blocks_per_sm() {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  static std::mutex mu;
  static std::map<int, int> cache;
  std::lock_guard<std::mutex> lk(mu);
  auto it = cache.find(dev);
  if (it == cache.end()) {
    int per_sm = 0;
    constexpr uint32_t kSmemBytes = ScanShape<T>::kSmemBytes;
    if (cudaFuncSetAttribute(scan_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemBytes) !=
            cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, scan_kernel<T>, (int)kBlockThreads, kSmemBytes) !=
            cudaSuccess) {
      cudaGetLastError();
      return 0;
    }
    it = cache.emplace(dev, per_sm).first;
  }
  return it->second;
}

template <typename T>
pip_status launch_scan(T* A, uint64_t n, T* total, void* aux, uint64_t timeout_ns, cudaStream_t s) {
  DeviceInfo di;
  if (device_info(&di) != PIP_OK) return PIP_ECUDA;
  const int per_sm = scan_blocks_per_sm<T>();
  if (per_sm < 1) return PIP_ECUDA;
  uint32_t* latch = error_latch_ptr();
  if (latch == nullptr) return PIP_ECUDA;
  // at most kRing / (2 kDefer + 4) blocks, so that the ring outlasts every
  // look-back (the indices in use span fewer than (2 kDefer + 3) G);
  // the tags hold 24 bits of the tile index, far more than the tiles in
  // flight
  constexpr uint64_t kItems = ScanShape<T>::kTileBytes / sizeof(T);
  const uint64_t ntiles = (n + kItems - 1) / kItems;
  const uint32_t blocks = (uint32_t)std::max<uint64_t>(
      1, std::min<uint64_t>({(uint64_t)per_sm * di.sms, (uint64_t)kRing / (2u * kDefer + 4u), ntiles}));
  if (cudaMemsetAsync(aux, 0, scan_aux_bytes(), s) != cudaSuccess) return PIP_ECUDA;
  ScanCtrl* ctrl = static_cast<ScanCtrl*>(aux);
  ScanDesc* ring = reinterpret_cast<ScanDesc*>(static_cast<char*>(aux) + sizeof(ScanCtrl));
  // every block must be resident (a tile's look-back waits on the tiles of
  // other blocks), which the cooperative launch guarantees
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = dim3(blocks);
  cfg.blockDim = dim3(kBlockThreads);
  cfg.dynamicSmemBytes = ScanShape<T>::kSmemBytes;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  void* args[] = {&A, &n, &total, &ctrl, &ring, &timeout_ns, &latch};
  if (cudaLaunchKernelExC(&cfg, reinterpret_cast<const void*>(&scan_kernel<T>), args) != cudaSuccess) {
    cudaGetLastError();
    return PIP_ECUDA;
  }
  return PIP_OK;
}

}  // namespace

uint64_t scan_aux_bytes() { return sizeof(ScanCtrl) + (uint64_t)kRing * sizeof(ScanDesc); }

}  // namespace pip

using namespace pip;

extern "C" {

uint64_t pip_scan_aux_bytes(void) { return scan_aux_bytes(); }

pip_status pip_scan_ex(void* A_dev, uint64_t n, pip_dtype dtype, void* total_dev, void* aux_dev, uint64_t aux_bytes,
                       void* stream) {
  if (dtype != PIP_U32 && dtype != PIP_U64) return PIP_EINVAL;
  const uint32_t eb = dtype == PIP_U32 ? 4u : 8u;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (n == 0) {
    if (total_dev != nullptr) {
      if (reinterpret_cast<uintptr_t>(total_dev) % eb != 0) return PIP_EINVAL;
      if (cudaMemsetAsync(total_dev, 0, eb, s) != cudaSuccess) return PIP_ECUDA;
    }
    return PIP_OK;
  }
  if (A_dev == nullptr || reinterpret_cast<uintptr_t>(A_dev) % 16 != 0) return PIP_EINVAL;
  if (total_dev != nullptr && reinterpret_cast<uintptr_t>(total_dev) % eb != 0) return PIP_EINVAL;
  if (n >= (1ull << 40)) return PIP_EINVAL;
  void* aux = aux_dev;
  bool owned = false;
  if (aux != nullptr) {
    if (aux_bytes < scan_aux_bytes() || reinterpret_cast<uintptr_t>(aux) % 256 != 0) return PIP_EINVAL;
  } else {
    if (cudaMallocAsync(&aux, scan_aux_bytes(), s) != cudaSuccess) {
      cudaGetLastError();
      return PIP_ENOMEM;
    }
    owned = true;
  }
  const uint64_t timeout = 2000000000ull;
  pip_status st;
  if (dtype == PIP_U32)
    st = launch_scan(static_cast<uint32_t*>(A_dev), n, static_cast<uint32_t*>(total_dev), aux, timeout, s);
  else
    st = launch_scan(static_cast<unsigned long long*>(A_dev), n, static_cast<unsigned long long*>(total_dev), aux,
                     timeout, s);
  if (owned && cudaFreeAsync(aux, s) != cudaSuccess && st == PIP_OK) st = PIP_ECUDA;
  return st;
}

pip_status pip_scan(void* A_dev, uint64_t n, pip_dtype dtype, void* total_dev, void* stream) {
  return pip_scan_ex(A_dev, n, dtype, total_dev, nullptr, 0, stream);
}

}  // extern "C"
