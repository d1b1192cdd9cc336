// In-place list contraction (Section 4.2, Algorithm 2) on the
// deterministic-reservation round engine: one cooperative launch contracts
// every node of a set of doubly-linked lists with no host round trip.
//
// Input: n records (prev, next) of 64-bit node indices, PIP_LIST_NIL at the
// ends of a list.  Node i has priority i.  Round r works on the active set:
// every uncontracted node below the frontier U_r (the invariant that makes a
// contraction safe), i.e. the nodes carried from round r-1 plus the fresh
// block [U_{r-1}, U_r) of about n^(1-eps) nodes (the Decomposable Property:
// the order of contraction does not matter, so a prefix of the nodes can be
// processed round after round).  A round has two phases:
//   A. every active node reads its record and is marked when it is a local
//      minimum (both current neighbours NIL or larger); unmarked nodes are
//      kept for the next round;
//   B. (after a grid barrier) every marked node splices itself out: its
//      predecessor's next becomes its successor and vice versa.
// Two adjacent nodes are never both marked, and a marked node's own record
// is written by nobody in phase B, so the splices of a round never collide.
// A contracted node keeps the two neighbours it had when spliced out (the
// tree edges of the contraction), which is the output: the same records as
// contracting the nodes one at a time in priority order.  The smallest
// uncontracted node is always a local minimum, so every round contracts at
// least one node; a round that contracts none means the input has a cycle
// and the call reports PIP_EINTERNAL.
//
// As the paper notes for its in-place implementation, no array indexed by
// node (its R array) is needed: the marks live in a register bit mask of the
// thread that owns the node for the round, and the only scratch is the loser
// lists, on chip per block with an overflow queue in device memory.
//
// Input checks: phase A checks the range of both pointers of every record it
// reads, and the first bad one stops the run at the next barrier with
// PIP_EINVAL before phase B could follow it (every pointer a splice writes
// was itself checked in that round), so no access leaves the array; the
// records are then unspecified.  PIP_FLAG_VALIDATE_INPUT adds a full check of
// the lists (range and prev / next consistency) before anything is modified.
#include <algorithm>
#include <cstddef>
#include <cmath>
#include <cstdint>
#include <map>
#include <mutex>
#include <tuple>

#include "device.cuh"
#include "internal.h"

namespace pip {
namespace {

constexpr uint64_t kNil = PIP_LIST_NIL;
constexpr unsigned kFullL = 0xffffffffu;
constexpr uint32_t kMaxSlots = 32;  // items per thread and round (one mark bit each)
constexpr uint32_t kListThreads = 512;
#ifndef PIP_LIST_MIN_BLOCKS
#define PIP_LIST_MIN_BLOCKS 2
#endif

struct ListArgs {
  ulonglong2* rec;
  uint32_t n;
  uint32_t F;
  uint32_t kmax;
  uint32_t kloc;
  uint32_t* Q[2];  // overflow queues of carried nodes
  Ctrl* ctrl;
  pip_stats* stats;
  uint32_t* latch;
  uint64_t timeout_ns;
  uint64_t deadline_ns;
  uint32_t max_rounds;
  uint32_t flags;
};

__device__ __forceinline__ ulonglong2 ld_rec(const ulonglong2* p) { return __ldcg(p); }

// A block's contiguous slice [off, off + cnt) of a fresh block of f nodes.
__device__ __forceinline__ void list_slice(uint32_t f, uint32_t* off, uint32_t* cnt) {
  const uint32_t kf = (f + gridDim.x - 1u) / gridDim.x;
  const uint32_t f0 = min(f, blockIdx.x * kf);
  *off = f0;
  *cnt = min(f, f0 + kf) - f0;
}

// Link words of list ranking (kRank): the low 32 bits hold the neighbour's
// index (kNil32 at a list's end), the high 32 bits the weight of the link,
// i.e. the distance to that neighbour in the original list.
constexpr uint32_t kNil32 = 0xFFFFFFFFu;
__device__ __forceinline__ uint32_t link_node(unsigned long long w) { return (uint32_t)w; }
__device__ __forceinline__ unsigned long long link_weight(unsigned long long w) { return w >> 32; }
__device__ __forceinline__ unsigned long long make_link(unsigned long long weight, uint32_t node) {
  return (weight << 32) | node;
}

template <bool kRank>
__global__ void __launch_bounds__(kListThreads, PIP_LIST_MIN_BLOCKS) list_rounds_kernel(const ListArgs a) {
  extern __shared__ uint32_t s_loc[];  // two on-chip lists of a.kloc carried nodes
  __shared__ uint32_t s_nloc[2];
  __shared__ uint32_t s_lcount, s_err;
  __shared__ uint32_t s_U, s_f, s_g, s_m, s_stop;
  __shared__ unsigned long long s_attempts, s_losers, s_deadline;
  __shared__ uint32_t s_max_active, s_rounds, s_start_status;

  Ctrl* ctrl = a.ctrl;
  ulonglong2* rec = a.rec;
  const uint32_t NT = blockDim.x, lane = threadIdx.x & 31u;
  auto fail = [&](uint32_t code) {
    set_status(&ctrl->status, code);
    s_err = 1u;
  };

  if (threadIdx.x == 0) {
    s_nloc[0] = s_nloc[1] = 0;
    s_lcount = 0;
    s_err = 0;
    s_attempts = s_losers = 0;
    s_max_active = s_rounds = 0;
    s_deadline = globaltimer_ns() + a.deadline_ns;
    s_f = min(a.F, a.n);  // round 0: fresh block [0, f)
    s_U = s_f;
    s_g = 0;
    s_m = s_f;
    s_stop = 0;
    // invalid input found by the validation pass (read once for the block,
    // so that the whole block leaves together)
    s_start_status = ld_relaxed_u32(&ctrl->status);
  }
  __syncthreads();
  if (s_start_status != 0u) goto done;

  for (uint32_t r = 0;; ++r) {
    // barrier numbering: phase A of round r ends at barrier 2r+1, phase B at
    // 2r+2; barrier e uses word bw[e % 3]
    const uint32_t U = s_U, f = s_f, m = s_m, g = s_g;
    const uint32_t eA = 2u * r + 1u, eB = 2u * r + 2u;
    const uint32_t* const loc_in = s_loc + (r & 1u) * a.kloc;
    uint32_t* const loc_out = s_loc + ((r + 1u) & 1u) * a.kloc;
    uint32_t* const Qout = a.Q[(r + 1u) & 1u];
    uint32_t* const cnt_out = &ctrl->cnt[(r + 1u) % 3u];
    // this block's items: a slice of the fresh block [U - f, U), then its
    // carried nodes (on-chip list, then a slice of the overflow queue)
    uint32_t f0, nf;
    list_slice(f, &f0, &nf);
    const uint32_t nloc = s_nloc[r & 1u];
    const uint32_t kg = (g + gridDim.x - 1u) / gridDim.x;
    const uint32_t g0 = min(g, blockIdx.x * kg);
    const uint32_t nlg = nloc + (min(g, g0 + kg) - g0);
    const uint32_t* const Qg = a.Q[r & 1u] + g0 - nloc;
    const uint32_t nfs = (nf + NT - 1u) / NT;
    const uint32_t nslot = nfs + (nlg + NT - 1u) / NT;
    const uint32_t fbase = U - f + f0;

    if (blockIdx.x == 0 && threadIdx.x == 0) {
      // the word of barrier eA+1 = eB (last used at barrier eA-2) and the
      // overflow allocator of round r+2 (last used in round r-1)
      stcg(&ctrl->bw[eB % 3u], 0ull);
      stcg(&ctrl->cnt[(r + 2u) % 3u], 0u);
      if (globaltimer_ns() > s_deadline) fail(PIP_ETIMEOUT);
    }
    if (nslot > kMaxSlots && threadIdx.x == 0) fail(PIP_EINTERNAL);  // the planner keeps this from happening

    // ---- phase A: mark the local minima, keep the others
    uint32_t marks = 0;
    for (uint32_t q = 0; q < nslot && q < kMaxSlots; ++q) {
      uint32_t i = 0;
      bool act;
      if (q < nfs) {
        const uint32_t o = q * NT + threadIdx.x;
        act = o < nf;
        i = fbase + o;
      } else {
        const uint32_t p = (q - nfs) * NT + threadIdx.x;
        act = p < nlg;
        if (act) i = (p < nloc) ? loc_in[p] : ldcg(Qg + p);
      }
      bool lm = false;
      if (act) {
        const ulonglong2 v = ld_rec(rec + i);
        // a pointer out of range stops the run before phase B can use it;
        // every pointer a splice writes comes from a record checked here
        if constexpr (kRank) {
          const uint32_t p = link_node(v.x), q = link_node(v.y);
          if ((p != kNil32 && p >= a.n) || (q != kNil32 && q >= a.n)) fail(PIP_EINVAL);
          lm = (p == kNil32 || p > i) && (q == kNil32 || q > i);
        } else {
          if ((v.x != kNil && v.x >= a.n) || (v.y != kNil && v.y >= a.n)) fail(PIP_EINVAL);
          lm = (v.x == kNil || v.x > i) && (v.y == kNil || v.y > i);
        }
      }
      if (lm) marks |= 1u << q;
      const bool keep = act && !lm;
      const unsigned mask = __ballot_sync(kFullL, keep);
      if (mask) {
        const int leader = __ffs(mask) - 1;
        uint32_t wbase = 0;
        if ((int)lane == leader) wbase = atomicAdd(&s_lcount, (uint32_t)__popc(mask));
        wbase = __shfl_sync(kFullL, wbase, leader);
        const uint32_t idx = wbase + __popc(mask & ((1u << lane) - 1u));
        const bool spill = keep && idx >= a.kloc;
        if (keep && !spill) loc_out[idx] = i;
        const unsigned smask = __ballot_sync(kFullL, spill);
        if (smask) {
          const int sl = __ffs(smask) - 1;
          uint32_t qbase = 0;
          if ((int)lane == sl) qbase = atomicAdd(cnt_out, (uint32_t)__popc(smask));
          qbase = __shfl_sync(kFullL, qbase, sl);
          if (spill) {
            const uint32_t qq = qbase + __popc(smask & ((1u << lane) - 1u));
            if (qq < a.kmax) stcg(Qout + qq, i);
            else fail(PIP_EINTERNAL);  // cannot happen: the throttle bounds the carried nodes by kmax
          }
        }
      }
    }
    __syncthreads();  // s_lcount is final
    {
      const uint32_t lc = s_lcount;
      const uint32_t spilled = lc > a.kloc ? lc - a.kloc : 0u;
      // barrier A carries the block's carried and spilled counts; thread 0
      // derives the next round's state from the sums
      round_barrier(&ctrl->bw[eA % 3u], gridDim.x, lc, spilled, s_err != 0u, &ctrl->status, a.timeout_ns, true,
                    [&](bool ok, const RoundSum& sum) {
                      if (!ok) {
                        s_stop = 2u;
                        return;
                      }
                      if (sum.errors != 0u) {
                        s_stop = 1u;
                        return;
                      }
                      const uint32_t m0 = s_m, U0 = s_U, kept = sum.count0;
                      if (kept >= m0) {  // nothing contracted: only possible on a cycle
                        set_status(&ctrl->status, PIP_EINTERNAL);
                        s_stop = 1u;
                        return;
                      }
                      // next fresh block, throttled so that m_{r+1} <= (m_r - 1) + fn <= kmax
                      const uint32_t fn = min(min(a.F, a.n - U0), a.kmax - m0 + 1u);
                      const uint32_t rr = s_rounds + 1u;
                      s_rounds = rr;
                      s_attempts += m0;
                      s_losers += kept;
                      s_max_active = max(s_max_active, m0);
                      s_U = U0 + fn;
                      s_f = fn;
                      s_g = sum.count1;
                      s_m = kept + fn;
                      s_nloc[rr & 1u] = min(s_lcount, a.kloc);
                      s_lcount = 0;
                      s_stop = (kept + fn == 0u) ? 3u : 0u;  // 3: last round, finish phase B first
                      if (rr >= a.max_rounds) {
                        set_status(&ctrl->status, PIP_EINTERNAL);
                        s_stop = 1u;
                      }
                    });
    }
    if (s_stop == 1u || s_stop == 2u) break;

    // ---- phase B: the marked nodes splice themselves out (their own records
    // are not written by anyone in this phase, so they are read again here)
    for (uint32_t q = 0; q < nslot && q < kMaxSlots; ++q) {
      if (!((marks >> q) & 1u)) continue;
      uint32_t i;
      if (q < nfs) {
        i = fbase + q * NT + threadIdx.x;
      } else {
        const uint32_t p = (q - nfs) * NT + threadIdx.x;
        i = (p < nloc) ? loc_in[p] : ldcg(Qg + p);
      }
      const ulonglong2 v = ld_rec(rec + i);
      if constexpr (kRank) {
        // the new link between the two neighbours spans both of i's links
        const unsigned long long w = link_weight(v.x) + link_weight(v.y);
        const uint32_t p = link_node(v.x), q = link_node(v.y);
        if (p != kNil32) stcg(&rec[p].y, make_link(w, q));
        if (q != kNil32) stcg(&rec[q].x, make_link(w, p));
      } else {
        if (v.x != kNil) stcg(&rec[v.x].y, v.y);
        if (v.y != kNil) stcg(&rec[v.y].x, v.x);
      }
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) stcg(&ctrl->bw[(eB + 1u) % 3u], 0ull);  // word of barrier eB+1
    round_barrier(&ctrl->bw[eB % 3u], gridDim.x, 0u, 0u, s_err != 0u, &ctrl->status, a.timeout_ns, true,
                  [&](bool ok, const RoundSum& sum) {
                    if (!ok) s_stop = 2u;
                    else if (sum.errors != 0u) s_stop = 1u;
                  });
    if (s_stop != 0u) break;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0 && a.stats != nullptr && s_stop != 2u) {
    a.stats->rounds = s_rounds;
    a.stats->attempts = s_attempts;
    a.stats->losers = s_losers;
    a.stats->max_active = s_max_active;
    a.stats->grid_blocks = gridDim.x;
  }
done:
  if (threadIdx.x == 0) {
    const uint32_t st = ld_relaxed_u32(&ctrl->status);
    if (st != 0u) atomicCAS(a.latch, 0u, st);
    if (blockIdx.x == 0 && a.stats != nullptr) a.stats->status = st;
  }
}

// ---------------------------------------------------------------- list ranking
// List ranking = the contraction above with link weights (kRank), then the
// reconstruction step (Section 4.2: the values are distributed back down the
// contraction tree).  After the weighted contraction, node v's record holds
// its nearest larger node on each side, p and q, with the distance to each in
// the original list.  Every node between p and v is smaller than v, so
// before(v) = before(p) + distance(p, v), with before(v) = distance - 1 when
// p is the list's start (NIL); likewise after(v) from q.  p and q have larger
// indices than v, so the reconstruction runs the round engine downward: the
// active set is every unfinished node at or above the frontier D (nodes
// carried from the last round plus the fresh block [D_r, D_{r-1})), and a
// node finishes a side once that neighbour's value is final.  The largest
// active node always finishes (its neighbours are larger, hence finished),
// so every round makes progress.  A finished side's word is written as
// kDone | value, once, by the node's own thread, and read by the smaller
// nodes that name it; a read that races with that write returns the old
// word or the final one (single 64-bit accesses), so it only ever delays a
// node.  A last pass clears kDone, leaving (before, after) in every record.
constexpr unsigned long long kDone = 1ull << 63;

__device__ __forceinline__ unsigned long long ld_word(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_word(unsigned long long* p, unsigned long long v) {
  asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

// Input records (prev, next) -> link words of weight 1; a pointer out of
// range records PIP_EINVAL (the contraction then does not start).
__global__ void rank_pack_kernel(ulonglong2* rec, uint32_t n, Ctrl* ctrl) {
  if (block_status(&ctrl->status) != 0u) return;  // the full input check refused the lists: leave them as they are
  bool bad = false;
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const ulonglong2 v = rec[i];
    bad |= (v.x != kNil && v.x >= n) || (v.y != kNil && v.y >= n);
    rec[i] = make_ulonglong2(make_link(1, v.x == kNil ? kNil32 : (uint32_t)v.x),
                             make_link(1, v.y == kNil ? kNil32 : (uint32_t)v.y));
  }
  if (__syncthreads_or(bad) && threadIdx.x == 0) set_status(&ctrl->status, PIP_EINVAL);
}

// Drops the finished marks: record i = (nodes before i, nodes after i).
__global__ void rank_unmark_kernel(ulonglong2* rec, uint32_t n, Ctrl* ctrl) {
  if (block_status(&ctrl->status) != 0u) return;  // a failed run leaves its records as they are
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const ulonglong2 v = rec[i];
    rec[i] = make_ulonglong2(v.x & ~kDone, v.y & ~kDone);
  }
}

__global__ void __launch_bounds__(kListThreads, PIP_LIST_MIN_BLOCKS) rank_rounds_kernel(const ListArgs a) {
  extern __shared__ uint32_t s_loc[];  // two on-chip lists of a.kloc carried nodes
  __shared__ uint32_t s_nloc[2];
  __shared__ uint32_t s_lcount, s_err;
  __shared__ uint32_t s_D, s_f, s_g, s_m, s_stop;
  __shared__ unsigned long long s_deadline;
  __shared__ uint32_t s_rounds, s_start_status;

  Ctrl* ctrl = a.ctrl;
  unsigned long long* words = reinterpret_cast<unsigned long long*>(a.rec);  // word 2i: before side, 2i+1: after side
  const uint32_t NT = blockDim.x, lane = threadIdx.x & 31u;
  auto fail = [&](uint32_t code) {
    set_status(&ctrl->status, code);
    s_err = 1u;
  };
  if (threadIdx.x == 0) {
    s_nloc[0] = s_nloc[1] = 0;
    s_lcount = 0;
    s_err = 0;
    s_rounds = 0;
    s_deadline = globaltimer_ns() + a.deadline_ns;
    s_f = min(a.F, a.n);  // round 0: fresh block [n - f, n)
    s_D = a.n - s_f;
    s_g = 0;
    s_m = s_f;
    s_stop = 0;
    s_start_status = ld_relaxed_u32(&ctrl->status);  // the contraction's outcome, read once for the block
  }
  __syncthreads();
  if (s_start_status != 0u) goto done;

  for (uint32_t r = 0;; ++r) {
    const uint32_t D = s_D, f = s_f, g = s_g;
    const uint32_t* const loc_in = s_loc + (r & 1u) * a.kloc;
    uint32_t* const loc_out = s_loc + ((r + 1u) & 1u) * a.kloc;
    uint32_t* const Qout = a.Q[(r + 1u) & 1u];
    uint32_t* const cnt_out = &ctrl->cnt[(r + 1u) % 3u];
    uint32_t f0, nf;
    list_slice(f, &f0, &nf);
    const uint32_t nloc = s_nloc[r & 1u];
    const uint32_t kg = (g + gridDim.x - 1u) / gridDim.x;
    const uint32_t g0 = min(g, blockIdx.x * kg);
    const uint32_t nlg = nloc + (min(g, g0 + kg) - g0);
    const uint32_t* const Qg = a.Q[r & 1u] + g0 - nloc;
    const uint32_t nfs = (nf + NT - 1u) / NT;
    const uint32_t nslot = nfs + (nlg + NT - 1u) / NT;
    const uint32_t fbase = D + f0;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
      // the barrier word of round r+1 (last used at round r-2) and the
      // overflow allocator of round r+2 (last used in round r-1)
      stcg(&ctrl->bw[(r + 1u) % 3u], 0ull);
      stcg(&ctrl->cnt[(r + 2u) % 3u], 0u);
      if (globaltimer_ns() > s_deadline) fail(PIP_ETIMEOUT);
    }
    if (nslot > kMaxSlots && threadIdx.x == 0) fail(PIP_EINTERNAL);  // the planner keeps this from happening
    for (uint32_t q = 0; q < nslot && q < kMaxSlots; ++q) {
      uint32_t v = 0;
      bool act;
      if (q < nfs) {
        const uint32_t o = q * NT + threadIdx.x;
        act = o < nf;
        v = fbase + o;
      } else {
        const uint32_t p = (q - nfs) * NT + threadIdx.x;
        act = p < nlg;
        if (act) v = (p < nloc) ? loc_in[p] : ldcg(Qg + p);
      }
      bool keep = false;
      if (act) {
        unsigned long long x = ld_word(words + 2ull * v), y = ld_word(words + 2ull * v + 1ull);
        const bool xd = (x & kDone) != 0ull, yd = (y & kDone) != 0ull;
        // a neighbour must be larger than v (the contraction's tree): anything
        // else is a defect of the records, stopped before it is followed
        const uint32_t p = link_node(x), qn = link_node(y);
        if ((!xd && p != kNil32 && (p >= a.n || p <= v)) || (!yd && qn != kNil32 && (qn >= a.n || qn <= v)))
          fail(PIP_EINVAL);
        unsigned long long nx = x, ny = y;
        if (!xd && p != kNil32 && p < a.n && p > v) nx = ld_word(words + 2ull * p);
        if (!yd && qn != kNil32 && qn < a.n && qn > v) ny = ld_word(words + 2ull * qn + 1ull);
        if (!xd) {
          if (p == kNil32) x = kDone | (link_weight(x) - 1ull);
          else if (nx & kDone) x = kDone | ((nx & ~kDone) + link_weight(x));
          if (x & kDone) st_word(words + 2ull * v, x);
        }
        if (!yd) {
          if (qn == kNil32) y = kDone | (link_weight(y) - 1ull);
          else if (ny & kDone) y = kDone | ((ny & ~kDone) + link_weight(y));
          if (y & kDone) st_word(words + 2ull * v + 1ull, y);
        }
        keep = !((x & kDone) && (y & kDone));
      }
      const unsigned mask = __ballot_sync(kFullL, keep);
      if (mask) {
        const int leader = __ffs(mask) - 1;
        uint32_t wbase = 0;
        if ((int)lane == leader) wbase = atomicAdd(&s_lcount, (uint32_t)__popc(mask));
        wbase = __shfl_sync(kFullL, wbase, leader);
        const uint32_t idx = wbase + __popc(mask & ((1u << lane) - 1u));
        const bool spill = keep && idx >= a.kloc;
        if (keep && !spill) loc_out[idx] = v;
        const unsigned smask = __ballot_sync(kFullL, spill);
        if (smask) {
          const int sl = __ffs(smask) - 1;
          uint32_t qbase = 0;
          if ((int)lane == sl) qbase = atomicAdd(cnt_out, (uint32_t)__popc(smask));
          qbase = __shfl_sync(kFullL, qbase, sl);
          if (spill) {
            const uint32_t qq = qbase + __popc(smask & ((1u << lane) - 1u));
            if (qq < a.kmax) stcg(Qout + qq, v);
            else fail(PIP_EINTERNAL);  // cannot happen: the throttle bounds the carried nodes by kmax
          }
        }
      }
    }
    __syncthreads();  // s_lcount is final
    const uint32_t lc = s_lcount;
    const uint32_t spilled = lc > a.kloc ? lc - a.kloc : 0u;
    round_barrier(&ctrl->bw[r % 3u], gridDim.x, lc, spilled, s_err != 0u, &ctrl->status, a.timeout_ns, true,
                  [&](bool ok, const RoundSum& sum) {
                    if (!ok) {
                      s_stop = 2u;
                      return;
                    }
                    if (sum.errors != 0u) {
                      s_stop = 1u;
                      return;
                    }
                    const uint32_t m0 = s_m, D0 = s_D, kept = sum.count0;
                    if (kept >= m0) {  // nothing finished: the records are not a contraction's output
                      set_status(&ctrl->status, PIP_EINTERNAL);
                      s_stop = 1u;
                      return;
                    }
                    const uint32_t fn = min(min(a.F, D0), a.kmax - m0 + 1u);
                    const uint32_t rr = s_rounds + 1u;
                    s_rounds = rr;
                    s_D = D0 - fn;
                    s_f = fn;
                    s_g = sum.count1;
                    s_m = kept + fn;
                    s_nloc[rr & 1u] = min(s_lcount, a.kloc);
                    s_lcount = 0;
                    s_stop = (kept + fn == 0u) ? 1u : 0u;
                    if (rr >= a.max_rounds) {
                      set_status(&ctrl->status, PIP_EINTERNAL);
                      s_stop = 1u;
                    }
                  });
    if (s_stop != 0u) break;
  }
done:
  if (threadIdx.x == 0) {
    const uint32_t st = ld_relaxed_u32(&ctrl->status);
    if (st != 0u) atomicCAS(a.latch, 0u, st);
    if (blockIdx.x == 0 && a.stats != nullptr && st != 0u) a.stats->status = st;
  }
}

// Full input check (PIP_FLAG_VALIDATE_INPUT): every pointer in range or NIL,
// and prev / next consistent; any violation is recorded as PIP_EINVAL before
// the contraction kernel touches the lists.  It costs two random reads per
// node, about half of a contraction, so it is opt-in; without it the
// contraction kernel still checks the range of every pointer before using it.
__global__ void validate_list_kernel(const ulonglong2* __restrict__ rec, uint32_t n, Ctrl* ctrl) {
  bool bad = false;
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const ulonglong2 v = rec[i];
    if (v.x != kNil) bad |= v.x >= n || rec[v.x].y != i;
    if (v.y != kNil) bad |= v.y >= n || rec[v.y].x != i;
  }
  if (__syncthreads_or(bad) && threadIdx.x == 0) set_status(&ctrl->status, PIP_EINVAL);
}

uint64_t align256(uint64_t x) { return (x + 255) / 256 * 256; }

int list_blocks_per_sm(uint32_t threads, uint64_t smem) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  static std::mutex mu;
  static std::map<std::tuple<int, uint32_t, uint64_t>, int> cache;
  std::lock_guard<std::mutex> lk(mu);
  const auto key = std::make_tuple(dev, threads, smem);
  auto it = cache.find(key);
  if (it == cache.end()) {
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, list_rounds_kernel<false>, (int)threads, (size_t)smem) !=
        cudaSuccess) {
      cudaGetLastError();
      return 0;
    }
    it = cache.emplace(key, per_sm).first;
  }
  return it->second;
}

}  // namespace

// Plan of one list contraction: prefix F within the scratch bound, grid shape,
// scratch layout (Ctrl, then two overflow queues of kmax words).
pip_status make_list_plan(uint64_t n, double eps, const pip_options* opt, ListPlan* out,
                          int (*blocks_per_sm)(uint32_t threads, uint64_t smem), uint32_t cache_per_thread) {
  if (!(eps > 0.0 && eps < 1.0) || n < 2 || n >= 0xFFFFFFFFull) return PIP_EINVAL;
  pip_options o{};
  if (opt != nullptr) o = *opt;
  ListPlan p;
  p.n = (uint32_t)n;
  const double x = std::pow((double)n, 1.0 - eps);
  p.aux_bound = (uint64_t)std::floor(PIP_AUX_C * x) + 4096;
  uint32_t threads = o.block_threads ? o.block_threads : kListThreads;
  if (threads < 128 || threads > kListThreads || threads % 32 != 0) return PIP_EINVAL;
  p.threads = threads;
  p.cache_per_thread = cache_per_thread;
  DeviceInfo di;
  const bool have_dev = device_info(&di) == PIP_OK;
  double want = o.fresh_per_round ? (double)o.fresh_per_round : (o.prefix_c > 0.0 ? o.prefix_c : 4.0) * x;
  uint64_t F = (uint64_t)std::max(1.0, std::ceil(want));
  F = std::min<uint64_t>({F, n, 1600000ull});  // per-round counts travel in 22-bit fields (kmax = 2.5 F + 2)
  for (;;) {
    p.F = (uint32_t)F;
    p.kmax = (uint32_t)(F * 5 / 2 + 2);
    const uint64_t active_est = F + F / 8 + 1;
    // about one active item per thread, at most two blocks per SM: for small
    // prefixes fewer blocks make each grid barrier cheaper and leave room for
    // on-chip caches (at F = 56.5K on GB300, 128 blocks measured 30.7 ms for
    // lists and 41.4 ms for trees of 2e8 nodes, against 32.8 and 48.1 ms
    // with 304 blocks and 32.9 and 52.3 ms with 64)
    uint64_t want_b = (active_est + 2ull * threads - 1) / (2ull * threads);
    if (have_dev) want_b = std::max<uint64_t>(want_b, std::min<uint64_t>(2ull * di.sms, (active_est + threads - 1) / threads));
    if (o.grid_blocks) want_b = o.grid_blocks;
    want_b = std::max<uint64_t>(1, std::min<uint64_t>(want_b, 1023));
    p.kloc = (uint32_t)std::min<uint64_t>(4096, std::max<uint64_t>(32, ((F / 4 + want_b - 1) / want_b + 31) / 32 * 32));
    const int per_sm =
        !have_dev ? 0 : (blocks_per_sm ? blocks_per_sm(threads, p.block_smem()) : list_blocks_per_sm(threads, p.block_smem()));
    if (per_sm > 0) want_b = std::min<uint64_t>(want_b, (uint64_t)per_sm * di.sms);
    p.blocks = (uint32_t)want_b;
    // every block handles at most kMaxSlots items per thread and round
    // (a block's items are at most kmax / blocks + kloc + 2: its fresh and
    // overflow slices and its on-chip list; with kloc <= 8 slots of 512,
    // kmax <= 20 slots per thread keeps the sum within kMaxSlots)
    const uint64_t cap = (uint64_t)p.blocks * threads * 20;
    p.off_Q[0] = align256(sizeof(Ctrl));
    p.off_Q[1] = p.off_Q[0] + align256(4ull * p.kmax);
    p.aux_bytes = p.off_Q[1] + align256(4ull * p.kmax);
    p.smem_bytes = (uint64_t)p.blocks * p.block_smem();
    const bool fits = p.aux_bytes + p.smem_bytes <= p.aux_bound && p.kmax <= cap;
    if (fits || F <= 1) break;
    const double ratio = std::min((double)p.aux_bound / (double)(p.aux_bytes + p.smem_bytes),
                                  (double)cap / (double)p.kmax);
    F = std::max<uint64_t>(1, std::min<uint64_t>((uint64_t)std::floor((double)F * std::min(ratio, 0.999)), F - 1));
  }
  if (p.aux_bytes + p.smem_bytes > p.aux_bound) return PIP_EINVAL;
  p.timeout_ns = o.wait_timeout_ns ? o.wait_timeout_ns : 2000000000ull;
  p.deadline_ns = 60000000000ull + 4000ull * (p.n / p.F + 1) + 20ull * p.n;
  p.flags = o.flags;
  *out = p;
  return PIP_OK;
}

namespace {

ListArgs list_args(const ListPlan& plan, void* rec, void* aux, pip_stats* stats) {
  char* base = static_cast<char*>(aux);
  ListArgs a{};
  a.rec = static_cast<ulonglong2*>(rec);
  a.n = plan.n;
  a.F = plan.F;
  a.kmax = plan.kmax;
  a.kloc = plan.kloc;
  a.Q[0] = reinterpret_cast<uint32_t*>(base + plan.off_Q[0]);
  a.Q[1] = reinterpret_cast<uint32_t*>(base + plan.off_Q[1]);
  a.ctrl = reinterpret_cast<Ctrl*>(base);
  a.stats = stats;
  a.latch = error_latch_ptr();
  a.timeout_ns = plan.timeout_ns;
  a.deadline_ns = plan.deadline_ns;
  a.max_rounds = plan.n + 8u;
  a.flags = plan.flags;
  return a;
}

// Cooperative launch of one of the round kernels with the plan's shape,
// clamped to what that kernel can keep resident.
pip_status launch_rounds(const void* kernel, const ListPlan& plan, ListArgs a, cudaStream_t stream) {
  DeviceInfo di;
  if (device_info(&di) != PIP_OK) return PIP_ECUDA;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return PIP_ECUDA;
  }
  // occupancy of each kernel and shape, looked up once per device
  static std::mutex mu;
  static std::map<std::tuple<int, const void*, uint32_t, uint64_t>, int> cache;
  int per_sm = 0;
  {
    std::lock_guard<std::mutex> lk(mu);
    const auto key = std::make_tuple(dev, kernel, plan.threads, plan.block_smem());
    auto it = cache.find(key);
    if (it == cache.end()) {
      if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, (int)plan.threads,
                                                        (size_t)plan.block_smem()) != cudaSuccess) {
        cudaGetLastError();
        return PIP_ECUDA;
      }
      it = cache.emplace(key, per_sm).first;
    }
    per_sm = it->second;
  }
  if (per_sm < 1) return PIP_ECUDA;
  const uint32_t blocks = std::max(1u, std::min<uint32_t>({plan.blocks, (uint32_t)per_sm * (uint32_t)di.sms, 1023u}));
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = dim3(blocks);
  cfg.blockDim = dim3(plan.threads);
  cfg.dynamicSmemBytes = plan.block_smem();
  cfg.stream = stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  void* args[] = {&a};
  if (cudaLaunchKernelExC(&cfg, kernel, args) != cudaSuccess) {
    cudaGetLastError();
    return PIP_ECUDA;
  }
  return PIP_OK;
}

}  // namespace

pip_status launch_list_driver(const ListPlan& plan, void* rec, void* aux, pip_stats* stats, cudaStream_t stream) {
  ListArgs a = list_args(plan, rec, aux, stats);
  if (a.latch == nullptr) return PIP_ECUDA;
  if (cudaMemsetAsync(aux, 0, plan.aux_bytes, stream) != cudaSuccess) return PIP_ECUDA;
  if (plan.flags & PIP_FLAG_VALIDATE_INPUT) {
    const uint32_t vb = (uint32_t)std::min<uint64_t>(1024, (plan.n + 255) / 256);
    validate_list_kernel<<<vb, 256, 0, stream>>>(a.rec, plan.n, a.ctrl);
    if (cudaGetLastError() != cudaSuccess) return PIP_ECUDA;
  }
  return launch_rounds(reinterpret_cast<const void*>(&list_rounds_kernel<false>), plan, a, stream);
}

// List ranking: pack the records into link words, contract with weights,
// reconstruct downward, drop the marks -- all on `stream`, one scratch area.
pip_status launch_list_rank(const ListPlan& plan, void* rec, void* aux, pip_stats* stats, cudaStream_t stream) {
  ListArgs a = list_args(plan, rec, aux, stats);
  if (a.latch == nullptr) return PIP_ECUDA;
  const uint32_t eb = (uint32_t)std::min<uint64_t>(4096, (plan.n + 255) / 256);
  if (cudaMemsetAsync(aux, 0, plan.aux_bytes, stream) != cudaSuccess) return PIP_ECUDA;
  if (plan.flags & PIP_FLAG_VALIDATE_INPUT) {
    validate_list_kernel<<<std::min(eb, 1024u), 256, 0, stream>>>(a.rec, plan.n, a.ctrl);
    if (cudaGetLastError() != cudaSuccess) return PIP_ECUDA;
  }
  rank_pack_kernel<<<eb, 256, 0, stream>>>(a.rec, plan.n, a.ctrl);
  if (cudaGetLastError() != cudaSuccess) return PIP_ECUDA;
  pip_status st = launch_rounds(reinterpret_cast<const void*>(&list_rounds_kernel<true>), plan, a, stream);
  if (st != PIP_OK) return st;
  // the reconstruction starts from clean allocators and barrier words; the
  // status word (offset 12) keeps the contraction's outcome
  static_assert(offsetof(Ctrl, status) == 12 && offsetof(Ctrl, barrier) == 16 && offsetof(Ctrl, gate_count) == 48,
                "Ctrl layout");
  char* base = static_cast<char*>(aux);
  if (cudaMemsetAsync(base, 0, 12, stream) != cudaSuccess || cudaMemsetAsync(base + 16, 0, 32, stream) != cudaSuccess)
    return PIP_ECUDA;
  st = launch_rounds(reinterpret_cast<const void*>(&rank_rounds_kernel), plan, a, stream);
  if (st != PIP_OK) return st;
  rank_unmark_kernel<<<eb, 256, 0, stream>>>(a.rec, plan.n, a.ctrl);
  return cudaGetLastError() == cudaSuccess ? PIP_OK : PIP_ECUDA;
}

}  // namespace pip

// ------------------------------------------------------------------ C ABI
using namespace pip;

extern "C" {

pip_status pip_list_plan(uint64_t n, double eps, const pip_options* opt, pip_plan_info* out) {
  if (out == nullptr || !(eps > 0.0 && eps < 1.0) || n >= 0xFFFFFFFFull) return PIP_EINVAL;
  *out = pip_plan_info{};
  out->n = n;
  out->elem_bytes = 16;
  out->eps = eps;
  out->driver = 3;
  if (n <= 1) return PIP_OK;
  ListPlan p;
  const pip_status st = make_list_plan(n, eps, opt, &p);
  if (st != PIP_OK) return st;
  out->fresh_per_round = p.F;
  out->max_active = p.kmax;
  out->grid_blocks = p.blocks;
  out->block_threads = p.threads;
  out->aux_bytes = p.aux_bytes;
  out->smem_bytes = p.smem_bytes;
  out->aux_bound_bytes = p.aux_bound;
  out->min_rounds = (n + p.F - 1) / p.F;
  return PIP_OK;
}

pip_status pip_list_contract_ex(pip_list_node* nodes_dev, uint64_t n, double eps, const pip_options* opt,
                                void* aux_dev, uint64_t aux_bytes, pip_stats* stats_dev, void* stream) {
  if (!(eps > 0.0 && eps < 1.0) || n >= 0xFFFFFFFFull) return PIP_EINVAL;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (n <= 1) {
    if (stats_dev != nullptr) {
      pip_stats zero{};
      if (cudaMemcpyAsync(stats_dev, &zero, sizeof(zero), cudaMemcpyHostToDevice, s) != cudaSuccess) return PIP_ECUDA;
      if (cudaStreamSynchronize(s) != cudaSuccess) return PIP_ECUDA;
    }
    return PIP_OK;
  }
  if (nodes_dev == nullptr || reinterpret_cast<uintptr_t>(nodes_dev) % 16 != 0) return PIP_EINVAL;
  ListPlan plan;
  pip_status st = make_list_plan(n, eps, opt, &plan);
  if (st != PIP_OK) return st;
  void* aux = aux_dev;
  bool owned = false;
  if (aux != nullptr) {
    if (aux_bytes < plan.aux_bytes || (reinterpret_cast<uintptr_t>(aux) % 256) != 0) return PIP_EINVAL;
  } else {
    if (cudaMallocAsync(&aux, plan.aux_bytes, s) != cudaSuccess) {
      cudaGetLastError();
      return PIP_ENOMEM;
    }
    owned = true;
  }
  st = launch_list_driver(plan, nodes_dev, aux, stats_dev, s);
  if (owned && cudaFreeAsync(aux, s) != cudaSuccess && st == PIP_OK) st = PIP_ECUDA;
  return st;
}

pip_status pip_list_contract(pip_list_node* nodes_dev, uint64_t n, double eps, void* stream) {
  return pip_list_contract_ex(nodes_dev, n, eps, nullptr, nullptr, 0, nullptr, stream);
}

pip_status pip_list_rank_ex(pip_list_node* nodes_dev, uint64_t n, double eps, const pip_options* opt, void* aux_dev,
                            uint64_t aux_bytes, pip_stats* stats_dev, void* stream) {
  if (!(eps > 0.0 && eps < 1.0) || n >= (1ull << 31)) return PIP_EINVAL;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (nodes_dev == nullptr && n > 0) return PIP_EINVAL;
  if (n == 1) {  // one node alone in its list: nothing before or after it
    const pip_list_node zero{0, 0};
    if (cudaMemcpyAsync(nodes_dev, &zero, sizeof(zero), cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
      return PIP_ECUDA;
  }
  if (n <= 1) {
    if (stats_dev != nullptr) {
      pip_stats zero{};
      if (cudaMemcpyAsync(stats_dev, &zero, sizeof(zero), cudaMemcpyHostToDevice, s) != cudaSuccess) return PIP_ECUDA;
      if (cudaStreamSynchronize(s) != cudaSuccess) return PIP_ECUDA;
    }
    return PIP_OK;
  }
  if (reinterpret_cast<uintptr_t>(nodes_dev) % 16 != 0) return PIP_EINVAL;
  ListPlan plan;
  pip_status st = make_list_plan(n, eps, opt, &plan);
  if (st != PIP_OK) return st;
  void* aux = aux_dev;
  bool owned = false;
  if (aux != nullptr) {
    if (aux_bytes < plan.aux_bytes || (reinterpret_cast<uintptr_t>(aux) % 256) != 0) return PIP_EINVAL;
  } else {
    if (cudaMallocAsync(&aux, plan.aux_bytes, s) != cudaSuccess) {
      cudaGetLastError();
      return PIP_ENOMEM;
    }
    owned = true;
  }
  st = launch_list_rank(plan, nodes_dev, aux, stats_dev, s);
  if (owned && cudaFreeAsync(aux, s) != cudaSuccess && st == PIP_OK) st = PIP_ECUDA;
  return st;
}

pip_status pip_list_rank(pip_list_node* nodes_dev, uint64_t n, double eps, void* stream) {
  return pip_list_rank_ex(nodes_dev, n, eps, nullptr, nullptr, 0, nullptr, stream);
}

}  // extern "C"
