// Persistent round driver: one cooperative launch walks every round of the
// deterministic-reservation Knuth shuffle (Algorithm 1 under the Decomposable
// Property, Section 4.1; round/prefix framework of Section 7.2 and
// Appendix A.1; reservation rule and dense window of RP-OneRes / RP-Final,
// Appendix A.2) with no host round trip.
//
// Round r (0-based) has an active set of m_r swaps: the n_r losers carried
// from round r-1 and the fresh block W_r = [L_r, L_{r-1}) (L_{-1} = n).
// Invariant: every unfinished step with index >= L_r is active, which is what
// makes a commit safe (Section 4.1: always work on the first unfinished swaps
// in sequential order).  A block keeps the losers it produced in an on-chip
// list and works on them again in the next round; only those beyond the
// list's capacity go to an overflow queue in device memory (Q[r&1]), which
// the next round deals out over all blocks.  Each block also takes one
// contiguous slice of W_r.
//
// The rounds are software-pipelined so that one grid barrier per round
// suffices.  Between barriers B_{r-1} and B_r, phase P_r
//   (a) decides round r: step i commits iff no active step targets location i
//       and i holds the maximum priority on its target; winners swap A[i] and
//       A[H[i]]; losers are kept for round r+1 and immediately reserve for it;
//   (b) lets the fresh block W_{r+1} reserve for round r+1;
//   (c) clears the tables of round r-1 (the cleaning phase of Appendix A.1).
// Reservations for round r+1 therefore land in a different table (S/D index
// (r+1)%3) from the one round r reads (r%3) and the one being cleared
// ((r+2)%3).
//
// Reservation structures of one round (priority of step i is i+1, 0 = unset):
//   S (slot table): nslots words; target t maps to slot slot_of(t) and the
//     word holds the max priority over all swaps whose target maps there.
//     Unlike the paper's keyed hash table this table is keyless, so a slot
//     shared by two targets can make a swap fail although it had no real
//     conflict.  Such spurious failures only delay a swap: a swap still
//     commits only if no higher-priority active swap touches either of its
//     locations, and the highest-priority active swap always commits, so
//     every round makes progress and the result is the sequential one.
//   D (window bitmap, the dense array of RP-Final reduced to one bit per
//     location): bit t - L_r is set when some active swap targets location
//     t of the fresh window W_r.  Any swap targeting t has a larger index
//     than t, so a set bit is exactly "a higher-priority swap targets t".
// Commit test of active step i with target h != i (OneRes rule, Appendix A.2):
//   own location free: bit i - L_r of D clear for fresh i, S[slot(i)] <= i+1
//     for a carried loser (every swap targeting i has a higher priority);
//   target won:        S[slot(h)] == i+1.
// With PIP_FLAG_TWO_RES the rule of Algorithm 1 as printed: every step also
// reserves its own location, and commits iff it holds the maximum on both
// slots (the same winners, at the cost of one more reservation per step).
// Self-loops (h == i) never reserve and finish at once (text under Alg. 1).
//
// Synchronisation: one bounded grid barrier per round through a per-round
// 64-bit word that also sums the blocks' loser counts and overflow counts, so
// the next round's active set is known when the barrier completes, with no
// further load; no global atomic is on the common path of a round.
#include <algorithm>
#include <cstdint>
#include <cstdlib>
#include <map>
#include <mutex>
#include <tuple>

#include "device.cuh"
#include "internal.h"

namespace pip {

// Per-device word holding the first error any round kernel of this library
// reported since the last pip_check(); 0 when none.
__device__ uint32_t g_error_latch;

namespace {

// Positions per thread in flight in the commit phase, and the launch bounds:
// two positions per thread, with registers for two 512-thread blocks per SM
// (64, no spills; the planner launches at most two blocks per SM), measured
// best on GB300: against a bound of three blocks per SM (40 registers, a few
// spills) 58.4 against 58.8 ms at n = 10^9 u64, eps = 0.25, 101.5 against
// 103.9 ms at eps = 0.5 and 112.4 against 117.4 ms for 2^30 16-byte records.
// Three positions per thread at the same bound measured 60.4 / 98.3 / 110.4
// against 58.0 / 97.4 / 109.0 ms; one position per thread at four blocks per
// SM was 2-8 % slower.
#ifndef PIP_KU
#define PIP_KU 2
#endif
#ifndef PIP_MIN_BLOCKS
#define PIP_MIN_BLOCKS 2
#endif
#ifndef PIP_MAX_THREADS
#define PIP_MAX_THREADS 512
#endif
constexpr int kU = PIP_KU;            // positions per thread in flight in the commit phase
constexpr uint32_t kGateGo = 1u, kGateAbort = 2u;  // start-gate decisions (Ctrl::gate_decision)
constexpr unsigned kFull = 0xffffffffu;


template <bool kExplicit>
__device__ __forceinline__ uint32_t target_of(const GridArgs& a, uint32_t i) {
  if constexpr (kExplicit) return __ldg(a.H + i);
  else return hashed_target(a.seed, i);
}

// Reserve target h for step i (priority i+1) in the tables of a round whose
// fresh window is [wlo, whi): the priority goes to the slot table, and a
// target inside the window also sets its bit in the window bitmap.  Under
// the two-reservation rule of Algorithm 1 (PIP_FLAG_TWO_RES) the step also
// reserves its own location i in the slot table.
__device__ __forceinline__ void reserve(uint32_t* D, uint32_t* S, uint32_t nslots, uint32_t wlo,
                                        uint32_t whi, uint32_t i, uint32_t h, bool two) {
  if (h >= wlo && h < whi) red_or(D + ((h - wlo) >> 5), 1u << ((h - wlo) & 31u));
  red_max(S + slot_of(h, nslots), i + 1u);
  if (two) red_max(S + slot_of(i, nslots), i + 1u);
}

// L2 policy of the array stores.  A stored line (both sides of a swap) is not
// read again soon, so by default it is marked evict-first, which leaves more
// of L2 to the reservation tables (measured 4 % faster at n = 10^9).
__device__ __forceinline__ uint64_t array_store_policy(uint32_t flags) {
  return (flags & PIP_FLAG_STORE_EVICT_NORMAL) ? policy_evict_normal() : policy_evict_first();
}

__device__ __forceinline__ void prefetch_l2(const void* p) {
  asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
}

// Fresh block [lo, hi) reserves for the round whose window it is.  With
// PIP_FLAG_PREFETCH the A lines that round will swap are pulled into L2 now,
// one round ahead of the commit that reads them.
template <typename Elem, bool kExplicit>
__device__ __forceinline__ void reserve_fresh(const GridArgs& a, uint32_t lo, uint32_t hi,
                                              uint32_t* D, uint32_t* S, uint32_t tid, uint32_t T) {
  const bool pf = (a.flags & PIP_FLAG_PREFETCH) != 0u;
  const Elem* A = static_cast<const Elem*>(a.A);
#pragma unroll 4
  for (uint32_t i = lo + tid; i < hi; i += T) {
    const uint32_t h = target_of<kExplicit>(a, i);
    if (h != i) {
      reserve(D, S, a.nslots, lo, hi, i, h, (a.flags & PIP_FLAG_TWO_RES) != 0u);
      if (pf) {
        prefetch_l2(A + h);
        if ((i & 7u) == 0u || i == lo + tid) prefetch_l2(A + i);
      }
    }
  }
}

// Start gate of a launch that is not cooperative (thread 0 of each block):
// nothing guarantees that every block is resident at once, so all of them
// first check in.  The first block that sees every arrival, or runs out of
// time, decides for all (compare-and-swap on one word); on an abort every
// block leaves before touching the array or the tables, and the run reports
// PIP_EBUSY.  Returns true when the blocks may go on.  `arrive == false`
// (a test hook) keeps this block from checking in, so the gate gives up.
__device__ __noinline__ bool start_gate(Ctrl* ctrl, uint64_t timeout_ns, bool arrive) {
  if (arrive) atomicAdd(&ctrl->gate_count, 1u);
  uint64_t t0 = 0;
  uint32_t polls = 0, d;
  while ((d = ld_relaxed_u32(&ctrl->gate_decision)) == 0u) {
    if (ld_relaxed_u32(&ctrl->gate_count) >= gridDim.x) {
      atomicCAS(&ctrl->gate_decision, 0u, kGateGo);
    } else if ((++polls & 63u) == 0u) {
      const uint64_t now = globaltimer_ns();
      if (t0 == 0) t0 = now;
      else if (now - t0 > timeout_ns) atomicCAS(&ctrl->gate_decision, 0u, kGateAbort);
    }
  }
  fence_acq_rel_gpu();
  if (d == kGateAbort) set_status(&ctrl->status, PIP_EBUSY);
  return d == kGateGo;
}

__device__ __forceinline__ void clear_words(uint32_t* p, uint32_t count, uint32_t tid, uint32_t T) {
  // 16-byte stores over the 16-byte aligned body, scalars for the tail
  const uint32_t n4 = count >> 2;
  uint4* p4 = reinterpret_cast<uint4*>(p);
  for (uint32_t j = tid; j < n4; j += T) stcg(p4 + j, make_uint4(0, 0, 0, 0));
  for (uint32_t j = (n4 << 2) + tid; j < count; j += T) stcg(p + j, 0u);
}

// Words of a window bitmap over F locations.
__host__ __device__ __forceinline__ uint32_t window_words(uint32_t F) { return (F + 31u) >> 5; }

template <typename Elem, bool kExplicit, bool kGate>
__global__ void __launch_bounds__(PIP_MAX_THREADS, PIP_MIN_BLOCKS) rounds_kernel(const GridArgs a) {
  // two on-chip loser lists of a.kloc words: the block's losers of the
  // previous round (worked on now) and of this round (worked on next)
  extern __shared__ uint32_t s_loc[];
  __shared__ uint32_t s_nloc[2];
  __shared__ uint32_t s_lcount, s_err;
  // Round state, identical in every block: thread 0 derives it from the
  // barrier word (kept in shared memory so that nothing but the round index
  // stays live in registers across the barrier).
  __shared__ uint32_t s_L, s_Lprev, s_g, s_m, s_stop;
  // run statistics and the deadline, kept by thread 0 (block 0's are reported)
  __shared__ unsigned long long s_attempts, s_losers, s_deadline;
  __shared__ uint32_t s_max_active, s_rounds, s_start_status;

  Elem* A = static_cast<Elem*>(a.A);
  Ctrl* ctrl = a.ctrl;
  const uint32_t NT = blockDim.x;
  const uint32_t lane = threadIdx.x & 31u;
  // records an error of this call and flags it in the block's next arrival
  auto fail = [&](uint32_t code) {
    set_status(&ctrl->status, code);
    s_err = 1u;
  };

  if (threadIdx.x == 0) {
    s_nloc[0] = 0;
    s_nloc[1] = 0;
    s_lcount = 0;
    s_err = 0;
    s_attempts = 0;
    s_losers = 0;
    s_max_active = 0;
    s_rounds = 0;
    s_deadline = globaltimer_ns() + a.deadline_ns;
    // round 0: no carried losers, fresh block W_0 = [n - f_0, n)
    s_Lprev = a.n;
    s_L = a.n - min(a.F, a.n - 1u);
    s_g = 0;
    s_m = min(a.F, a.n - 1u);
    s_stop = 0;
    // an invalid explicit target sequence reported by the validation pass
    // (read once for the block, so that the whole block leaves together)
    s_start_status = ld_relaxed_u32(&ctrl->status);
  }
  __syncthreads();
  if (s_start_status != 0u) goto done;
  if constexpr (kGate) {
    if (threadIdx.x == 0)
      s_stop = start_gate(ctrl, a.gate_timeout_ns, !((a.flags & PIP_FLAG_TEST_SKIP_BARRIER) && blockIdx.x == 0))
                   ? 0u
                   : 2u;
    __syncthreads();
    if (s_stop != 0u) goto done;
  }

  // ---- prologue: W_0 reserves for round 0 (barrier 0 uses word bw[0];
  // round r's barrier uses bw[(r+1)%3])
  reserve_fresh<Elem, kExplicit>(a, s_L, a.n, a.D[0], a.S[0], blockIdx.x * NT + threadIdx.x, gridDim.x * NT);
  round_barrier(&ctrl->bw[0], gridDim.x, 0u, 0u, false, &ctrl->status, a.timeout_ns,
                !((a.flags & PIP_FLAG_TEST_SKIP_BARRIER) && blockIdx.x == 0),
                [&](bool ok, const RoundSum&) { s_stop = ok ? 0u : 2u; });
  if (s_stop != 0u) goto done;

  for (uint32_t r = 0;; ++r) {
    const uint32_t L = s_L, Lprev = s_Lprev, m = s_m;
    const uint32_t b = r % 3u, b1 = (r + 1u) % 3u, b2 = (r + 2u) % 3u;
    uint32_t* const Dr = a.D[b];
    uint32_t* const Sr = a.S[b];
    uint32_t* const Dn = a.D[b1];
    uint32_t* const Sn = a.S[b1];
    const uint32_t* const loc_in = s_loc + (r & 1u) * a.kloc;
    uint32_t* const loc_out = s_loc + ((r + 1u) & 1u) * a.kloc;
    uint32_t* const Qout = a.Q[(r + 1u) & 1u];
    uint32_t* const cnt_out = &ctrl->cnt[b1];

    // next round's fresh block W_{r+1} = [Ln, L); throttled so that
    // m_{r+1} <= (m_r - 1) + fn <= kmax (at least one swap of round r
    // commits), which bounds the loser queue; the throttle only acts when
    // losers pile up beyond the queue's slack
    const uint32_t fn = min(min(a.F, L - 1u), a.kmax - m + 1u);
    const uint32_t Ln = L - fn;

    // This block's share of round r's active set, in slots of NT items (one
    // per thread): first its carried losers (its on-chip list, then a slice
    // of the overflow queue), then one contiguous slice of W_r.  (Dealing W_r
    // out grid-wide, W_r[c*T + blockIdx.x*NT + t], measured the same at large
    // F and 10-25 % slower per round at small F.)
    const uint32_t nloc = s_nloc[r & 1u];
    const uint32_t g = s_g;
    const uint32_t kg = (g + gridDim.x - 1u) / gridDim.x;
    const uint32_t g0 = min(g, blockIdx.x * kg);
    const uint32_t nlg = nloc + (min(g, g0 + kg) - g0);  // carried items of this block
    const uint32_t* const Qg = a.Q[r & 1u] + g0 - nloc;  // item p in [nloc, nlg) is Qg[p]
    const uint32_t f = Lprev - L;
    const uint32_t qs = (nlg + NT - 1u) / NT;  // slots of carried items
    const uint32_t kf = (f + gridDim.x - 1u) / gridDim.x;
    const uint32_t f0 = min(f, blockIdx.x * kf);
    const uint32_t nf = min(f, f0 + kf) - f0;
    const uint32_t nslot = qs + (nf + NT - 1u) / NT;

    if (blockIdx.x == 0 && threadIdx.x == 0) {
      // Words no block can still be using: the overflow allocator of round
      // r+2 (last used in phase r-1) and the barrier word of round r+1 (last
      // polled at barrier r-1, which every block has left since it arrived
      // at barrier r).
      stcg(&ctrl->cnt[b2], 0u);
      stcg(&ctrl->bw[b2], 0ull);
      if (globaltimer_ns() > s_deadline) fail(PIP_ETIMEOUT);
    }

    const bool two = (a.flags & PIP_FLAG_TWO_RES) != 0u;
    // (b) and (c) below, issued before the commit under
    // PIP_FLAG_EARLY_RESERVE (small prefixes): the fresh block reserves in
    // round r+1's tables and the cleaning touches round r-1's, neither of
    // which the commit of round r reads
    const bool early = (a.flags & PIP_FLAG_EARLY_RESERVE) != 0u;
    if (early) {
      reserve_fresh<Elem, kExplicit>(a, Ln, L, Dn, Sn, blockIdx.x * NT + threadIdx.x, gridDim.x * NT);
      clear_words(a.S[b2], a.nslots, blockIdx.x * NT + threadIdx.x, gridDim.x * NT);
      clear_words(a.D[b2], window_words(a.F), blockIdx.x * NT + threadIdx.x, gridDim.x * NT);
    }
    // ---- (a) commit round r.  Each thread takes kU slots at a time and
    // issues their loads together so that kU independent memory chains are
    // in flight per thread.
    for (uint32_t q0 = 0; q0 < nslot; q0 += kU) {
      uint32_t ii[kU], hh[kU], own[kU], rh[kU];
      bool act[kU];
#pragma unroll
      for (int j = 0; j < kU; ++j) {
        const uint32_t q = q0 + (uint32_t)j;
        ii[j] = 0;
        if (q < qs) {
          const uint32_t p = q * NT + threadIdx.x;
          act[j] = p < nlg;
          if (act[j]) ii[j] = (p < nloc) ? loc_in[p] : ldcg(Qg + p);
        } else {
          const uint32_t o = (q - qs) * NT + threadIdx.x;
          act[j] = q < nslot && o < nf;
          ii[j] = L + f0 + o;
        }
      }
#pragma unroll
      for (int j = 0; j < kU; ++j) {
        hh[j] = act[j] ? target_of<kExplicit>(a, ii[j]) : 0u;
        act[j] = act[j] && hh[j] != ii[j];  // self-loops finish at once
      }
      Elem x[kU], y[kU];
      // Exchange commit (PIP_FLAG_SWAP_EXCHANGE, set by the planner): the
      // own element is loaded together with the reservation checks (a
      // coalesced read for the fresh block, wasted for the swaps that lose),
      // and a winner exchanges it into A[h] at L2 and stores what comes back
      // at A[i].  Load-store commit otherwise: both elements are loaded after
      // the decision (or with it under PIP_FLAG_SPECULATE), both are stored.
      const bool xchg = (a.flags & PIP_FLAG_SWAP_EXCHANGE) != 0u;
      const bool spec = !xchg && (a.flags & PIP_FLAG_SPECULATE) != 0u;
      if (xchg || spec) {
#pragma unroll
        for (int j = 0; j < kU; ++j) {
          if (act[j]) {
            x[j] = ldcg(A + ii[j]);
            if (spec) y[j] = ldcg(A + hh[j]);
          }
        }
      }
#pragma unroll
      for (int j = 0; j < kU; ++j) {
        own[j] = 0;
        rh[j] = 0;
        if (act[j]) {
          const uint32_t i = ii[j], h = hh[j];
          own[j] = (i < Lprev && !two) ? ldcg(Dr + ((i - L) >> 5)) : ldcg(Sr + slot_of(i, a.nslots));
          rh[j] = ldcg(Sr + slot_of(h, a.nslots));
        }
      }
      bool win[kU];
#pragma unroll
      for (int j = 0; j < kU; ++j) {
        const uint32_t i = ii[j];
        // own location free: no active swap targets i (window bit clear),
        // or every swap mapping to the slot of i has a priority at most i+1
        // (two-reservation rule: the step holds the maximum on its own slot)
        const bool own_free = two ? own[j] == i + 1u
                              : (i < Lprev) ? (((own[j] >> ((i - L) & 31u)) & 1u) == 0u)
                                            : (own[j] <= i + 1u);
        win[j] = act[j] && own_free && rh[j] == i + 1u;
        if (win[j] && !xchg && !spec) {
          x[j] = ldcg(A + ii[j]);
          y[j] = ldcg(A + hh[j]);
        }
      }
      const uint64_t stpol = array_store_policy(a.flags);
      if (xchg) {
#pragma unroll
        for (int j = 0; j < kU; ++j)
          if (win[j]) y[j] = exch_hint(A + hh[j], x[j], stpol);
      }
#pragma unroll
      for (int j = 0; j < kU; ++j) {
        if (win[j]) {
          st_hint(A + ii[j], y[j], stpol);
          if (!xchg) st_hint(A + hh[j], x[j], stpol);
        }
      }
#pragma unroll
      for (int j = 0; j < kU; ++j) {
        // losers reserve for round r+1 at once and join the block's next
        // on-chip list, or the overflow queue once that list is full
        const bool lose = act[j] && !win[j];
        if (lose) reserve(Dn, Sn, a.nslots, Ln, L, ii[j], hh[j], two);
        const unsigned mask = __ballot_sync(kFull, lose);
        if (mask) {
          const int leader = __ffs(mask) - 1;
          uint32_t wbase = 0;
          if ((int)lane == leader) wbase = atomicAdd(&s_lcount, (uint32_t)__popc(mask));
          wbase = __shfl_sync(kFull, wbase, leader);
          const uint32_t idx = wbase + __popc(mask & ((1u << lane) - 1u));
          const bool spill = lose && idx >= a.kloc;
          if (lose && !spill) loc_out[idx] = ii[j];
          const unsigned smask = __ballot_sync(kFull, spill);
          if (smask) {
            const int sl = __ffs(smask) - 1;
            uint32_t qbase = 0;
            if ((int)lane == sl) qbase = atomicAdd(cnt_out, (uint32_t)__popc(smask));
            qbase = __shfl_sync(kFull, qbase, sl);
            if (spill) {
              const uint32_t q = qbase + __popc(smask & ((1u << lane) - 1u));
              if (q < a.kmax) stcg(Qout + q, ii[j]);
              else fail(PIP_EINTERNAL);  // cannot happen: the throttle bounds the losers by kmax
            }
          }
        }
      }
    }

    if (!early) {
      // ---- (b) fresh block of round r+1 reserves (after the commit for
      // large prefixes: issued before it, these atomics and stores measured
      // 3-8 % slower there)
      reserve_fresh<Elem, kExplicit>(a, Ln, L, Dn, Sn, blockIdx.x * NT + threadIdx.x, gridDim.x * NT);

      // ---- (c) clean round r-1's tables (they become round r+2's)
      clear_words(a.S[b2], a.nslots, blockIdx.x * NT + threadIdx.x, gridDim.x * NT);
      clear_words(a.D[b2], window_words(a.F), blockIdx.x * NT + threadIdx.x, gridDim.x * NT);
    }

    // ---- barrier B_r with this block's losers (all, and those spilled to
    // the overflow queue); thread 0 turns the sums into the next round's
    // state, which every block computes identically
    __syncthreads();  // s_lcount is final
    const uint32_t lc = s_lcount;
    const uint32_t spilled = lc > a.kloc ? lc - a.kloc : 0u;
    round_barrier(&ctrl->bw[b1], gridDim.x, lc, spilled, s_err != 0u, &ctrl->status, a.timeout_ns, true,
                  [&](bool ok, const RoundSum& sum) {
                    if (!ok) {
                      s_stop = 2u;
                      return;
                    }
                    if (sum.errors != 0u) {  // recorded in status by the block that failed
                      s_stop = 1u;
                      return;
                    }
                    const uint32_t m0 = s_m, L0 = s_L, losers = sum.count0;
                    const uint32_t fn0 = min(min(a.F, L0 - 1u), a.kmax - m0 + 1u);
                    if (losers >= m0) {  // no swap committed: impossible (the top active swap wins)
                      set_status(&ctrl->status, PIP_EINTERNAL);
                      s_stop = 1u;
                      return;
                    }
                    const uint32_t rr = s_rounds + 1u;
                    s_rounds = rr;
                    s_attempts += m0;
                    s_losers += losers;
                    s_max_active = max(s_max_active, m0);
                    const uint32_t mn = losers + fn0;
                    s_Lprev = L0;
                    s_L = L0 - fn0;
                    s_g = sum.count1;
                    s_m = mn;
                    s_nloc[(rr & 1u)] = min(s_lcount, a.kloc);
                    s_lcount = 0;
                    if (mn == 0u) {
                      s_stop = 1u;
                    } else if (mn > a.kmax || rr >= a.max_rounds) {
                      set_status(&ctrl->status, PIP_EINTERNAL);
                      s_stop = 1u;
                    }
                  });
    if (s_stop != 0u) break;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0 && a.stats != nullptr && s_stop == 1u) {
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

__global__ void validate_targets_kernel(const uint32_t* __restrict__ H, uint32_t n, Ctrl* ctrl) {
  const uint32_t T = gridDim.x * blockDim.x;
  bool bad = false;
  for (uint32_t i = 1u + blockIdx.x * blockDim.x + threadIdx.x; i < n; i += T) bad |= (H[i] > i);
  if (__syncthreads_or(bad) && threadIdx.x == 0) set_status(&ctrl->status, PIP_EINVAL);
}

template <typename Elem, bool kExplicit, bool kGate = false>
const void* kernel_ptr() {
  return reinterpret_cast<const void*>(&rounds_kernel<Elem, kExplicit, kGate>);
}

const void* select_kernel(uint32_t elem_bytes, bool explicit_h) {
  switch (elem_bytes) {
    case 4: return explicit_h ? kernel_ptr<uint32_t, true>() : kernel_ptr<uint32_t, false>();
    case 8: return explicit_h ? kernel_ptr<unsigned long long, true>() : kernel_ptr<unsigned long long, false>();
    case 16: return explicit_h ? kernel_ptr<uint4, true>() : kernel_ptr<uint4, false>();
    default: return nullptr;
  }
}

// The gated kernels (hashed targets only): serving lanes.
const void* select_gated_kernel(uint32_t elem_bytes) {
  switch (elem_bytes) {
    case 4: return kernel_ptr<uint32_t, false, true>();
    case 8: return kernel_ptr<unsigned long long, false, true>();
    case 16: return kernel_ptr<uint4, false, true>();
    default: return nullptr;
  }
}

}  // namespace

uint32_t* error_latch_ptr() {
  // the symbol's device address, looked up once per device
  static std::mutex mu;
  static uint32_t* cached[64] = {};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
    cudaGetLastError();
    return nullptr;
  }
  std::lock_guard<std::mutex> lk(mu);
  if (cached[dev] == nullptr) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_error_latch) != cudaSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    cached[dev] = static_cast<uint32_t*>(p);
  }
  return cached[dev];
}

pip_status take_error_latch(uint32_t* value) {
  uint32_t v = 0, zero = 0;
  if (cudaMemcpyFromSymbol(&v, g_error_latch, sizeof(v)) != cudaSuccess) return PIP_ECUDA;
  if (v != 0 && cudaMemcpyToSymbol(g_error_latch, &zero, sizeof(zero)) != cudaSuccess) return PIP_ECUDA;
  *value = v;
  return PIP_OK;
}

uint32_t grid_driver_max_blocks(uint32_t elem_bytes, bool explicit_h, uint32_t threads, uint32_t kloc) {
  const void* k = select_kernel(elem_bytes, explicit_h);
  if (k == nullptr) return 0;
  DeviceInfo di;
  if (device_info(&di) != PIP_OK) return 0;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  static std::mutex mu;
  static std::map<std::tuple<int, const void*, uint32_t, uint32_t>, int> cache;
  std::lock_guard<std::mutex> lk(mu);
  const auto key = std::make_tuple(dev, k, threads, kloc);
  auto it = cache.find(key);
  if (it == cache.end()) {
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, (int)threads, (size_t)grid_block_smem(kloc)) !=
        cudaSuccess) {
      cudaGetLastError();
      return 0;
    }
    it = cache.emplace(key, per_sm).first;
  }
  return (uint32_t)it->second * (uint32_t)di.sms;
}

namespace {

pip_status launch_grid_common(const Plan& plan, void* A, const uint32_t* H, uint64_t seed, void* aux,
                              pip_stats* stats, uint64_t gate_timeout_ns, cudaStream_t stream) {
  const bool gated = gate_timeout_ns != 0u;
  if (gated && H != nullptr) return PIP_EINVAL;
  const void* k = gated ? select_gated_kernel(plan.elem_bytes) : select_kernel(plan.elem_bytes, H != nullptr);
  if (k == nullptr) return PIP_EINVAL;
  char* base = static_cast<char*>(aux);
  GridArgs a{};
  a.A = A;
  a.H = H;
  a.seed = seed;
  a.n = plan.n;
  a.F = plan.F;
  a.kmax = plan.kmax;
  a.nslots = plan.nslots;
  for (int j = 0; j < 3; ++j) {
    a.S[j] = reinterpret_cast<uint32_t*>(base + plan.off_S[j]);
    a.D[j] = reinterpret_cast<uint32_t*>(base + plan.off_D[j]);
  }
  for (int j = 0; j < 2; ++j) a.Q[j] = reinterpret_cast<uint32_t*>(base + plan.off_Q[j]);
  a.kloc = plan.kloc;
  a.ctrl = reinterpret_cast<Ctrl*>(base);
  a.stats = stats;
  a.timeout_ns = plan.timeout_ns;
  a.max_rounds = plan.n + 8u;
  a.deadline_ns = plan.deadline_ns;
  a.flags = plan.flags;
  a.gate_timeout_ns = gate_timeout_ns;
  // a lane keeps its errors to itself: they are the request's, not the device's
  a.latch = gate_timeout_ns != 0u ? &a.ctrl->lane_status : error_latch_ptr();
  if (a.latch == nullptr) return PIP_ECUDA;

  if (cudaMemsetAsync(aux, 0, plan.aux_bytes, stream) != cudaSuccess) return PIP_ECUDA;
  if (H != nullptr) {
    const uint32_t vb = (uint32_t)std::min<uint64_t>(1024, (plan.n + 255) / 256);
    validate_targets_kernel<<<vb, 256, 0, stream>>>(H, plan.n, a.ctrl);
    if (cudaGetLastError() != cudaSuccess) return PIP_ECUDA;
  }
  // every block must be co-resident (the cooperative launch refuses otherwise;
  // a gated launch checks it at its start gate)
  uint32_t blocks = plan.blocks;
  const uint32_t maxb = grid_driver_max_blocks(plan.elem_bytes, H != nullptr, plan.threads, plan.kloc);
  if (maxb == 0) return PIP_ECUDA;
  blocks = std::max(1u, std::min({blocks, maxb, kBwMaxBlocks}));
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = dim3(blocks);
  cfg.blockDim = dim3(plan.threads);
  cfg.dynamicSmemBytes = grid_block_smem(plan.kloc);
  cfg.stream = stream;
  cudaLaunchAttribute attr[1];
  int na = 0;
  if (!gated) {
    attr[na].id = cudaLaunchAttributeCooperative;
    attr[na].val.cooperative = 1;
    ++na;
  }
  cfg.attrs = attr;
  cfg.numAttrs = na;
  void* args[] = {&a};
  if (cudaLaunchKernelExC(&cfg, k, args) != cudaSuccess) {
    cudaGetLastError();
    return PIP_ECUDA;
  }
  return PIP_OK;
}

}  // namespace

pip_status launch_grid_driver(const Plan& plan, void* A, const uint32_t* H, uint64_t seed, void* aux,
                              pip_stats* stats, cudaStream_t stream) {
  return launch_grid_common(plan, A, H, seed, aux, stats, 0, stream);
}

pip_status launch_grid_lane(const Plan& plan, void* A, uint64_t seed, void* aux, pip_stats* stats,
                            uint64_t gate_timeout_ns, cudaStream_t stream) {
  if (gate_timeout_ns == 0u) return PIP_EINVAL;
  return launch_grid_common(plan, A, nullptr, seed, aux, stats, gate_timeout_ns, stream);
}

}  // namespace pip
