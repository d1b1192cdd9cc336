// In-place tree contraction (Section 4.2, the tree contraction paragraph) on
// the deterministic-reservation round engine: one cooperative launch
// contracts a forest of rooted binary trees (every internal node with two
// children) with no host round trip.
//
// Input: n records (parent, left, right, round) of 64-bit words,
// PIP_TREE_NIL for a missing pointer; a node is a leaf when its left word is
// NIL.  Raking a leaf l with parent p removes l and p; the other child s of p
// takes p's place under p's parent g.  Node i has priority i.  Round r works
// on the active set: the leaves carried from round r-1 plus the fresh block
// [U_{r-1}, U_r) of about n^(1-eps) node indices (the Decomposable Property:
// a prefix of the nodes per round), throttled as in the list driver.  A round
// has two phases:
//   A. every active leaf with a parent reads its neighbourhood and is marked
//      when no leaf among its sibling, its nephews (the sibling's children)
//      and its uncle (the other child of its grandparent) has a smaller
//      index; unmarked leaves are kept for the next round, internal nodes
//      and roots leave at once;
//   B. (after a grid barrier) every marked leaf rakes: s.parent = g, g's
//      child word that held p = s, and its own record becomes
//      (p, s, g, round).
// Two marked leaves are never sibling, uncle or nephew of each other, so the
// words one rake reads or writes in phase B are written by no other rake of
// the round (rakes that share a grandparent write its two different child
// words; one whose sibling is another's grandparent writes that node's parent
// word while the other writes a child word).  The smallest active leaf with a
// parent is always marked, so every round makes progress.  The result
// depends only on the plan's F and kmax: the set of active nodes of each
// round and every decision are functions of the state, not of the launch.
//
// As for lists, no array indexed by node is used: the marks live in a
// register bit mask of the thread that owns the node for the round, and the
// only scratch is the loser lists, on chip per block with an overflow queue.
//
// Input checks: phase A checks every pointer it follows (range, and that the
// parent lists the node as a child, and the grandparent the parent) and the
// first bad one stops the run at the next barrier with PIP_EINVAL before
// phase B could follow it; every pointer phase B follows was checked in
// phase A of the same round.  PIP_FLAG_VALIDATE_INPUT adds a full check of
// the forest before anything is modified.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <map>
#include <mutex>
#include <tuple>

#include "device.cuh"
#include "internal.h"

namespace pip {
namespace {

constexpr uint64_t kNil = PIP_TREE_NIL;
constexpr unsigned kFullT = 0xffffffffu;
constexpr uint32_t kMaxSlots = 32;  // items per thread and round (one mark bit each)
constexpr uint32_t kTreeThreads = 512;
// Slots of a thread decided together in phase A.  Two (twice the chains of
// random reads in flight) measured no faster on GB300 than one -- 24.9
// against 24.4 ms at eps = 0.25, 41.3 against 42.4 ms at eps = 0.5 for a tree
// of 2e8 nodes -- so the rounds are bound by the rate of random accesses, not
// by their latency; four spill registers.
#ifndef PIP_TREE_PHASE_A_WIDTH
#define PIP_TREE_PHASE_A_WIDTH 1
#endif
constexpr uint32_t kPhaseAWidth = PIP_TREE_PHASE_A_WIDTH;
// A marked leaf's sibling, grandparent and (when room allows) parent, found
// in phase A, are kept on chip for phase B (slots q < qc of each thread, two
// or three 32-bit words each; which child word of the grandparent to rewrite
// is a register bit), so that phase B only writes -- with the parent, the
// leaf's whole 32-byte record at once, a full sector that L2 need not fetch
// before writing it back.  Later slots read their records again.  The planner
// takes the first of 8, 4, 2, 1 slots of three words, then of two, that fits
// the scratch bound without lowering F.
#ifndef PIP_TREE_CACHE_PARENT
#define PIP_TREE_CACHE_PARENT 1
#endif
constexpr uint32_t kCacheSlotChoices[] = {8u, 4u, 2u, 1u};
constexpr uint32_t kNil32 = 0xFFFFFFFFu;
#ifndef PIP_TREE_MIN_BLOCKS
#define PIP_TREE_MIN_BLOCKS 2
#endif

// A record as two 16-byte halves: h[2i] = (parent, left), h[2i+1] = (right, round).
struct TreeArgs {
  ulonglong2* h;
  uint32_t n;
  uint32_t F;
  uint32_t kmax;
  uint32_t kloc;
  uint32_t* Q[2];  // overflow queues of carried leaves
  Ctrl* ctrl;
  pip_stats* stats;
  uint32_t* latch;
  uint64_t timeout_ns;
  uint64_t deadline_ns;
  uint32_t max_rounds;
  uint32_t qc;         // cached slots per thread (0, 1, 2, 4 or 8)
  uint32_t cache_par;  // 1: the cache holds the parent too (whole-record writes)
};

__device__ __forceinline__ uint64_t parent_of(const ulonglong2* h, uint64_t v) { return ldcg(&h[2 * v].x); }
__device__ __forceinline__ uint64_t left_of(const ulonglong2* h, uint64_t v) { return ldcg(&h[2 * v].y); }
__device__ __forceinline__ uint64_t right_of(const ulonglong2* h, uint64_t v) { return ldcg(&h[2 * v + 1].x); }

// A block's contiguous slice [off, off + cnt) of a fresh block of f nodes.
__device__ __forceinline__ void tree_slice(uint32_t f, uint32_t* off, uint32_t* cnt) {
  const uint32_t kf = (f + gridDim.x - 1u) / gridDim.x;
  const uint32_t f0 = min(f, blockIdx.x * kf);
  *off = f0;
  *cnt = min(f, f0 + kf) - f0;
}

// Phase A for K nodes i[k] of one thread at once: d[k] = 0 for no work
// (inactive, an internal node or a root), 1 when the leaf rakes this round,
// 2 when it is carried; *bad is set on a pointer that fails its check (that
// node then counts as no work).  For a leaf that rakes, s_out[k] and g_out[k]
// are its sibling and grandparent and g_right[k] tells that the parent is the
// grandparent's right child (p_out[k] its parent).  The K nodes go through the dependent loads
// (own record, parent, sibling and grandparent, then the nephews' and
// uncle's left words) stage by stage, so that a thread keeps K chains of
// random reads in flight instead of one.
template <int K>
__device__ __forceinline__ void tree_decide(const ulonglong2* h, const uint64_t (&i)[K], const bool (&act)[K],
                                            uint64_t n, bool* bad, uint32_t (&d)[K], uint64_t (&p_out)[K],
                                            uint64_t (&s_out)[K], uint64_t (&g_out)[K], bool (&g_right)[K]) {
  bool live[K];
  uint64_t p[K];
#pragma unroll
  for (int k = 0; k < K; ++k) {
    d[k] = 0u;
    s_out[k] = kNil;
    g_out[k] = kNil;
    g_right[k] = false;
    ulonglong2 me = make_ulonglong2(kNil, kNil);
    if (act[k]) me = ldcg(&h[2 * i[k]]);  // (parent, left)
    p[k] = me.x;
    live[k] = act[k] && me.y == kNil && me.x != kNil;  // a leaf with a parent
    if (live[k] && p[k] >= n) {
      *bad = true;
      live[k] = false;
    }
  }
  ulonglong2 P[K];
  uint64_t pr[K];
#pragma unroll
  for (int k = 0; k < K; ++k) {
    P[k] = make_ulonglong2(kNil, kNil);
    pr[k] = kNil;
    if (live[k]) {
      P[k] = ldcg(&h[2 * p[k]]);  // (g, left of p)
      pr[k] = right_of(h, p[k]);
    }
  }
  uint64_t s[K], g[K];
#pragma unroll
  for (int k = 0; k < K; ++k) {
    g[k] = P[k].x;
    s[k] = P[k].y == i[k] ? pr[k] : (pr[k] == i[k] ? P[k].y : kNil);
    if (live[k] && (s[k] >= n || (g[k] != kNil && g[k] >= n))) {
      *bad = true;
      live[k] = false;
    }
  }
  // the siblings' and the grandparents' child words, loaded together
  uint64_t sl[K], sr[K], gl[K], gr[K];
#pragma unroll
  for (int k = 0; k < K; ++k) {
    sl[k] = sr[k] = gl[k] = gr[k] = kNil;
    if (live[k]) {
      sl[k] = left_of(h, s[k]);
      sr[k] = right_of(h, s[k]);
      if (g[k] != kNil) {
        gl[k] = left_of(h, g[k]);
        gr[k] = right_of(h, g[k]);
      }
    }
  }
  bool win[K];
  uint64_t c0[K], c1[K], u[K];
#pragma unroll
  for (int k = 0; k < K; ++k) {
    win[k] = true;
    c0[k] = c1[k] = u[k] = kNil;
    if (!live[k]) continue;
    if (sl[k] == kNil) {
      win[k] = s[k] > i[k];  // the sibling is a leaf
    } else {
      if (sl[k] >= n || sr[k] >= n) {
        *bad = true;
        live[k] = false;
        continue;
      }
      c0[k] = sl[k] < i[k] ? sl[k] : kNil;  // nephews that could win
      c1[k] = sr[k] < i[k] ? sr[k] : kNil;
    }
    if (g[k] != kNil) {
      const uint64_t uu = gl[k] == p[k] ? gr[k] : (gr[k] == p[k] ? gl[k] : kNil);
      if (uu >= n) {
        *bad = true;
        live[k] = false;
        continue;
      }
      u[k] = uu < i[k] ? uu : kNil;
    }
  }
  // a smaller nephew or uncle beats i only if it is a leaf
  bool l0[K], l1[K], lu[K];
#pragma unroll
  for (int k = 0; k < K; ++k) {
    l0[k] = live[k] && c0[k] != kNil && left_of(h, c0[k]) == kNil;
    l1[k] = live[k] && c1[k] != kNil && left_of(h, c1[k]) == kNil;
    lu[k] = live[k] && u[k] != kNil && left_of(h, u[k]) == kNil;
  }
#pragma unroll
  for (int k = 0; k < K; ++k) {
    if (!live[k]) continue;
    d[k] = (win[k] && !l0[k] && !l1[k] && !lu[k]) ? 1u : 2u;
    p_out[k] = p[k];
    s_out[k] = s[k];
    g_out[k] = g[k];
    g_right[k] = g[k] != kNil && gr[k] == p[k];
  }
}

// Phase B for a marked leaf i in round r (0-based).  Every pointer it
// follows was checked in phase A of the same round; it is checked again
// (false return, nothing written) so that no state can send a store out of
// the array.
__device__ __forceinline__ bool tree_rake(ulonglong2* h, uint64_t i, uint32_t r, uint64_t n) {
  const uint64_t p = parent_of(h, i);
  if (p >= n) return false;
  const ulonglong2 P = ldcg(&h[2 * p]);
  const uint64_t pr = right_of(h, p);
  const uint64_t g = P.x;
  const uint64_t s = P.y == i ? pr : P.y;
  if (s >= n || (g != kNil && g >= n)) return false;
  using u64 = unsigned long long;
  stcg(&h[2 * s].x, (u64)g);
  if (g != kNil) {
    if (left_of(h, g) == p) stcg(&h[2 * g].y, (u64)s);
    else stcg(&h[2 * g + 1].x, (u64)s);
  }
  // the leaf's whole record (its parent word is unchanged): a full sector
  stcg(&h[2 * i], make_ulonglong2((u64)p, (u64)s));
  stcg(&h[2 * i + 1], make_ulonglong2(g, (unsigned long long)r + 1ull));
  return true;
}

__global__ void __launch_bounds__(kTreeThreads, PIP_TREE_MIN_BLOCKS) tree_rounds_kernel(const TreeArgs a) {
  extern __shared__ uint32_t s_loc[];  // two on-chip lists of a.kloc carried leaves, then the cache
  uint32_t* const c_sib = s_loc + 2u * a.kloc;       // [a.qc][blockDim.x]
  uint32_t* const c_gp = c_sib + a.qc * blockDim.x;   // [a.qc][blockDim.x]
  uint32_t* const c_par = c_gp + a.qc * blockDim.x;   // [a.qc][blockDim.x]
  __shared__ uint32_t s_nloc[2];
  __shared__ uint32_t s_lcount, s_err;
  __shared__ uint32_t s_U, s_f, s_g, s_m, s_stop;
  __shared__ unsigned long long s_attempts, s_losers, s_deadline;
  __shared__ uint32_t s_max_active, s_rounds, s_start_status;

  Ctrl* ctrl = a.ctrl;
  ulonglong2* h = a.h;
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
    const uint32_t U = s_U, f = s_f, g = s_g;
    const uint32_t eA = 2u * r + 1u, eB = 2u * r + 2u;
    const uint32_t* const loc_in = s_loc + (r & 1u) * a.kloc;
    uint32_t* const loc_out = s_loc + ((r + 1u) & 1u) * a.kloc;
    uint32_t* const Qout = a.Q[(r + 1u) & 1u];
    uint32_t* const cnt_out = &ctrl->cnt[(r + 1u) % 3u];
    // this block's items: a slice of the fresh block [U - f, U), then its
    // carried leaves (on-chip list, then a slice of the overflow queue)
    uint32_t f0, nf;
    tree_slice(f, &f0, &nf);
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

    // ---- phase A: mark the leaves that rake, keep the others
    // (kPhaseAWidth slots of a thread at a time)
    uint32_t marks = 0, rights = 0;
    const uint32_t nq = min(nslot, kMaxSlots);
    auto slot_item = [&](uint32_t q, uint32_t* i_out) -> bool {
      if (q >= nq) return false;
      if (q < nfs) {
        const uint32_t o = q * NT + threadIdx.x;
        *i_out = fbase + o;
        return o < nf;
      }
      const uint32_t pq = (q - nfs) * NT + threadIdx.x;
      if (pq >= nlg) return false;
      *i_out = (pq < nloc) ? loc_in[pq] : ldcg(Qg + pq);
      return true;
    };
    for (uint32_t q0 = 0; q0 < nq; q0 += kPhaseAWidth) {
      uint64_t iv[kPhaseAWidth];
      bool act[kPhaseAWidth];
      uint32_t d[kPhaseAWidth];
      uint64_t par[kPhaseAWidth], sib[kPhaseAWidth], gp[kPhaseAWidth];
      bool g_right[kPhaseAWidth];
#pragma unroll
      for (uint32_t k = 0; k < kPhaseAWidth; ++k) {
        uint32_t ii = 0;
        act[k] = slot_item(q0 + k, &ii);
        iv[k] = ii;
      }
      bool bad = false;
      tree_decide<(int)kPhaseAWidth>(h, iv, act, a.n, &bad, d, par, sib, gp, g_right);
      if (bad) fail(PIP_EINVAL);
#pragma unroll
      for (uint32_t k = 0; k < kPhaseAWidth; ++k) {
        const uint32_t q = q0 + k;
        if (q >= nq) break;  // uniform: nq is the same for the whole block
        if (d[k] == 1u && q < a.qc) {
          if (a.cache_par) c_par[q * NT + threadIdx.x] = (uint32_t)par[k];
          c_sib[q * NT + threadIdx.x] = (uint32_t)sib[k];
          c_gp[q * NT + threadIdx.x] = gp[k] == kNil ? kNil32 : (uint32_t)gp[k];
          if (g_right[k]) rights |= 1u << q;
        }
        if (d[k] == 1u) marks |= 1u << q;
        const uint32_t i = (uint32_t)iv[k];
        const bool keep = d[k] == 2u;
        const unsigned mask = __ballot_sync(kFullT, keep);
        if (mask) {
          const int leader = __ffs(mask) - 1;
          uint32_t wbase = 0;
          if ((int)lane == leader) wbase = atomicAdd(&s_lcount, (uint32_t)__popc(mask));
          wbase = __shfl_sync(kFullT, wbase, leader);
          const uint32_t idx = wbase + __popc(mask & ((1u << lane) - 1u));
          const bool spill = keep && idx >= a.kloc;
          if (keep && !spill) loc_out[idx] = i;
          const unsigned smask = __ballot_sync(kFullT, spill);
          if (smask) {
            const int sl = __ffs(smask) - 1;
            uint32_t qbase = 0;
            if ((int)lane == sl) qbase = atomicAdd(cnt_out, (uint32_t)__popc(smask));
            qbase = __shfl_sync(kFullT, qbase, sl);
            if (spill) {
              const uint32_t qq = qbase + __popc(smask & ((1u << lane) - 1u));
              if (qq < a.kmax) stcg(Qout + qq, i);
              else fail(PIP_EINTERNAL);  // cannot happen: the throttle bounds the carried leaves by kmax
            }
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
                      if (kept >= m0) {  // no progress: only possible on inconsistent input
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

    // ---- phase B: the marked leaves rake
    for (uint32_t q = 0; q < nslot && q < kMaxSlots; ++q) {
      if (!((marks >> q) & 1u)) continue;
      uint32_t i;
      if (q < nfs) {
        i = fbase + q * NT + threadIdx.x;
      } else {
        const uint32_t pq = (q - nfs) * NT + threadIdx.x;
        i = (pq < nloc) ? loc_in[pq] : ldcg(Qg + pq);
      }
      if (q < a.qc) {
        // cached: only writes (the values were checked in phase A)
        using u64 = unsigned long long;
        const uint64_t par = a.cache_par ? (uint64_t)c_par[q * NT + threadIdx.x] : 0u;
        const uint64_t sib = c_sib[q * NT + threadIdx.x];
        const uint32_t g32 = c_gp[q * NT + threadIdx.x];
        const uint64_t gp = g32 == kNil32 ? kNil : (uint64_t)g32;
        if (par >= a.n || sib >= a.n || (gp != kNil && gp >= a.n)) {
          fail(PIP_EINTERNAL);
          continue;
        }
        stcg(&h[2 * sib].x, (u64)gp);
        if (gp != kNil) {
          if ((rights >> q) & 1u) stcg(&h[2 * gp + 1].x, (u64)sib);
          else stcg(&h[2 * gp].y, (u64)sib);
        }
        // the leaf's record: whole when the parent is cached (its parent word
        // is unchanged), else from the left word on
        if (a.cache_par) stcg(&h[2 * (uint64_t)i], make_ulonglong2((u64)par, (u64)sib));
        else stcg(&h[2 * (uint64_t)i].y, (u64)sib);
        stcg(&h[2 * (uint64_t)i + 1], make_ulonglong2((u64)gp, (u64)r + 1ull));
      } else if (!tree_rake(h, i, r, a.n)) {
        fail(PIP_EINTERNAL);
      }
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) stcg(&ctrl->bw[(eB + 1u) % 3u], 0ull);  // word of barrier eB+1
    __syncthreads();  // s_err is final
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

// Full input check (PIP_FLAG_VALIDATE_INPUT): pointers in range or NIL, both
// child words NIL or both set and distinct, every child's parent pointing
// back, and every parent listing the node as a child; any violation is
// recorded as PIP_EINVAL before the contraction kernel touches the forest.
__global__ void validate_tree_kernel(const ulonglong2* __restrict__ h, uint32_t n, Ctrl* ctrl) {
  bool bad = false;
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const ulonglong2 a = h[2 * (uint64_t)i];
    const uint64_t p = a.x, l = a.y, r = h[2 * (uint64_t)i + 1].x;
    if ((l == kNil) != (r == kNil)) bad = true;
    if (l != kNil) bad |= l >= n || r >= n || l == r || (l < n && h[2 * l].x != i) || (r < n && h[2 * r].x != i);
    if (p != kNil) bad |= p >= n || (p < n && h[2 * p].y != i && h[2 * p + 1].x != i);
  }
  if (__syncthreads_or(bad) && threadIdx.x == 0) set_status(&ctrl->status, PIP_EINVAL);
}

// Resident blocks per SM for a launch of `threads` threads with `smem` bytes
// of dynamic shared memory (the kernel's limit is raised once to the
// device's opt-in maximum, so that any planned size is admissible).
int tree_blocks_per_sm(uint32_t threads, uint64_t smem) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  static std::mutex mu;
  static std::map<std::tuple<int, uint32_t, uint64_t>, int> cache;
  static std::map<int, bool> raised;
  std::lock_guard<std::mutex> lk(mu);
  if (!raised[dev]) {
    int optin = 0;
    cudaFuncAttributes fa{};
    if (cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess ||
        cudaFuncGetAttributes(&fa, tree_rounds_kernel) != cudaSuccess ||
        cudaFuncSetAttribute(tree_rounds_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             optin - (int)fa.sharedSizeBytes) != cudaSuccess) {
      cudaGetLastError();
      return 0;
    }
    raised[dev] = true;
  }
  const auto key = std::make_tuple(dev, threads, smem);
  auto it = cache.find(key);
  if (it == cache.end()) {
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, tree_rounds_kernel, (int)threads, (size_t)smem) !=
        cudaSuccess) {
      cudaGetLastError();
      return 0;
    }
    it = cache.emplace(key, per_sm).first;
  }
  return it->second;
}

}  // namespace

// Bytes of L2 per fresh node of the default prefix: phase A of a round reads
// the parent, sibling and grandparent records of its leaves (about half of
// the fresh nodes) at random, and the rounds ran fastest on GB300 (L2 of
// 129 MB) when those reads about filled L2, at F = 600K (21.8 ms for a tree
// of 2e8 nodes, against 23.3 ms at 300K and 900K and 24.3 ms at 1.25M).
constexpr uint64_t kTreeL2BytesPerFresh = 216;

// The list engine's plan, with the largest phase-B cache that fits the
// scratch bound without lowering F (or none).  Unless the caller fixes F,
// the default prefix C * n^(1-eps) is also capped at L2 / 216 bytes.
pip_status make_tree_plan(uint64_t n, double eps, const pip_options* opt, ListPlan* out) {
  pip_options o{};
  if (opt != nullptr) o = *opt;
  DeviceInfo di;
  if (o.fresh_per_round == 0 && eps > 0.0 && eps < 1.0 && device_info(&di) == PIP_OK && di.l2_bytes > 0) {
    const double want = (o.prefix_c > 0.0 ? o.prefix_c : 4.0) * std::pow((double)n, 1.0 - eps);
    const double cap = (double)di.l2_bytes / (double)kTreeL2BytesPerFresh;
    if (want > cap) o.fresh_per_round = (uint32_t)cap;
  }
  ListPlan plain;
  pip_status st = make_list_plan(n, eps, &o, &plain, &tree_blocks_per_sm, 0);
  if (st != PIP_OK) return st;
  *out = plain;
  for (const uint32_t words : {PIP_TREE_CACHE_PARENT ? 3u : 2u, 2u}) {
    for (const uint32_t qc : kCacheSlotChoices) {
      ListPlan cached;
      if (make_list_plan(n, eps, &o, &cached, &tree_blocks_per_sm, 4u * words * qc) == PIP_OK &&
          cached.F == plain.F) {
        cached.cache_slot_bytes = 4u * words;
        *out = cached;
        return PIP_OK;
      }
    }
  }
  return PIP_OK;
}

pip_status launch_tree_driver(const ListPlan& plan, void* rec, void* aux, pip_stats* stats, cudaStream_t stream) {
  char* base = static_cast<char*>(aux);
  TreeArgs a{};
  a.h = static_cast<ulonglong2*>(rec);
  a.n = plan.n;
  a.F = plan.F;
  a.kmax = plan.kmax;
  a.kloc = plan.kloc;
  a.Q[0] = reinterpret_cast<uint32_t*>(base + plan.off_Q[0]);
  a.Q[1] = reinterpret_cast<uint32_t*>(base + plan.off_Q[1]);
  a.ctrl = reinterpret_cast<Ctrl*>(base);
  a.stats = stats;
  a.latch = error_latch_ptr();
  if (a.latch == nullptr) return PIP_ECUDA;
  a.timeout_ns = plan.timeout_ns;
  a.deadline_ns = plan.deadline_ns;
  a.max_rounds = plan.n + 8u;
  a.cache_par = plan.cache_slot_bytes == 12u ? 1u : 0u;
  a.qc = plan.cache_slot_bytes != 0u ? plan.cache_per_thread / plan.cache_slot_bytes : 0u;
  if (cudaMemsetAsync(aux, 0, plan.aux_bytes, stream) != cudaSuccess) return PIP_ECUDA;
  if (plan.flags & PIP_FLAG_VALIDATE_INPUT) {
    const uint32_t vb = (uint32_t)std::min<uint64_t>(1024, (plan.n + 255) / 256);
    validate_tree_kernel<<<vb, 256, 0, stream>>>(a.h, plan.n, a.ctrl);
    if (cudaGetLastError() != cudaSuccess) return PIP_ECUDA;
  }
  DeviceInfo di;
  if (device_info(&di) != PIP_OK) return PIP_ECUDA;
  const int per_sm = tree_blocks_per_sm(plan.threads, plan.block_smem());
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
  if (cudaLaunchKernelExC(&cfg, reinterpret_cast<const void*>(&tree_rounds_kernel), args) != cudaSuccess) {
    cudaGetLastError();
    return PIP_ECUDA;
  }
  return PIP_OK;
}

}  // namespace pip

// ------------------------------------------------------------------ C ABI
using namespace pip;

extern "C" {

pip_status pip_tree_plan(uint64_t n, double eps, const pip_options* opt, pip_plan_info* out) {
  if (out == nullptr || !(eps > 0.0 && eps < 1.0) || n >= 0xFFFFFFFFull) return PIP_EINVAL;
  *out = pip_plan_info{};
  out->n = n;
  out->elem_bytes = 32;
  out->eps = eps;
  out->driver = 4;
  if (n <= 1) return PIP_OK;
  ListPlan p;
  const pip_status st = make_tree_plan(n, eps, opt, &p);
  if (st != PIP_OK) return st;
  out->fresh_per_round = p.F;
  out->max_active = p.kmax;
  out->grid_blocks = p.blocks;
  out->block_threads = p.threads;
  out->aux_bytes = p.aux_bytes;
  out->smem_bytes = p.smem_bytes;
  out->aux_bound_bytes = p.aux_bound;
  out->min_rounds = (n + p.F - 1) / p.F;
  out->slots = p.cache_per_thread;
  return PIP_OK;
}

pip_status pip_tree_contract_ex(pip_tree_node* nodes_dev, uint64_t n, double eps, const pip_options* opt,
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
  if (nodes_dev == nullptr || reinterpret_cast<uintptr_t>(nodes_dev) % 32 != 0) return PIP_EINVAL;
  ListPlan plan;
  pip_status st = make_tree_plan(n, eps, opt, &plan);
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
  st = launch_tree_driver(plan, nodes_dev, aux, stats_dev, s);
  if (owned && cudaFreeAsync(aux, s) != cudaSuccess && st == PIP_OK) st = PIP_ECUDA;
  return st;
}

pip_status pip_tree_contract(pip_tree_node* nodes_dev, uint64_t n, double eps, void* stream) {
  return pip_tree_contract_ex(nodes_dev, n, eps, nullptr, nullptr, 0, nullptr, stream);
}

}  // extern "C"
