// The block-resident round loop shared by the batched driver and the serving
// tick: one thread block runs the rounds of one array with its reservation
// tables in shared memory.
//
// Round structure (deterministic reservations over the first unfinished
// swaps, Algorithm 1 under the Decomposable Property, Section 4.1; RP-OneRes
// rule, Appendix A.2; cleaning phase, Appendix A.1).  The tables hold the
// reservations of every swap of the current round when it starts; then
//   1. commit: each active swap tests its two locations and, if it won both,
//      swaps A[i] and A[H[i]]; losers are appended to the next queue;
//   2. (bar.sync) the next fresh block is sized from the losers actually
//      left (so the active set never exceeds cta_kmax(F)); the tables are
//      cleared;
//   3. (bar.sync) the losers and the next fresh block reserve;
//   4. (bar.sync) the next round starts.
// One slot table and one window bitmap suffice because nothing reserves
// while the round's tests read them.  Fresh swaps come first in a round's
// order, from the top of the window down, so the thread that works on fresh
// swap i = L - 1 - t next round is known one round ahead (t = thread index).
//
// Reservation structures (priority of step i is i+1, 0 = unset):
//   S: nslots words; target t maps to slot slot_of(t), which holds the
//      maximum priority of the swaps whose target maps there (keyless, so a
//      shared slot can only make a swap fail spuriously, never commit
//      wrongly);
//   D: one bit per location of the fresh window [L, Lprev), set when an
//      active swap targets it (any such swap has a higher priority).
// Commit test of active step i with target h != i:
//   own location free: D bit clear for a fresh i, S[slot(i)] <= i+1 for a
//   carried loser; target won: S[slot(h)] == i+1.  Self-loops finish at once.
// Under the two-reservation rule (Algorithm 1 as printed) every step also
// reserves its own location, and the own-location test is S[slot(i)] == i+1.
//
// Pipelining (lone arrays): while a round commits, thread t already loads
// the two array elements of the fresh swap it will take next round,
// i' = L - 1 - t.  A location can change in this round only if some swap of
// this round targets it (the own locations of this round's swaps are all at
// or above L), so the early values are used next round when the current
// slot table shows no reservation on either location, and reloaded
// otherwise.  A thread whose first position next round is a carried loser
// loads that swap's elements while reserving for it (after this round's
// stores), which needs no check.
//
// A run can stop after a number of rounds and resume later (serving): at a
// round boundary the state is the frontier L, the end of the current fresh
// block, and the carried losers; on resume the tables are rebuilt from them
// (the reservations depend on nothing else).
#pragma once

#include <cstdint>

#include "device.cuh"
#include "internal.h"

namespace pip {

constexpr unsigned kCtaFull = 0xffffffffu;
constexpr int kCtaU = 4;  // positions per thread whose array loads are in flight together

__device__ __forceinline__ uint32_t job_target(const BatchJob& j, uint32_t i) {
  return j.H != nullptr ? __ldg(j.H + i) : hashed_target(j.seed, i);
}

// Reserve target h for step i (priority i+1): the priority in the slot table,
// and the window bit when h lies in the fresh window [wlo, whi).
// Under the two-reservation rule of Algorithm 1 the step also reserves its
// own location i.
__device__ __forceinline__ void sreserve(uint32_t* D, uint32_t* S, uint32_t ns, uint32_t wlo, uint32_t whi,
                                         uint32_t i, uint32_t h, bool two) {
  if (h >= wlo && h < whi) atomicOr(D + ((h - wlo) >> 5), 1u << ((h - wlo) & 31u));
  atomicMax(S + slot_of(h, ns), i + 1u);
  if (two) atomicMax(S + slot_of(i, ns), i + 1u);
}

// Zeroes count words at p (16-byte aligned): 16-byte stores, then the tail.
__device__ __forceinline__ void sclear(uint32_t* p, uint32_t count) {
  uint4* p4 = reinterpret_cast<uint4*>(p);
  const uint32_t n4 = count >> 2;
  for (uint32_t j = threadIdx.x; j < n4; j += blockDim.x) p4[j] = make_uint4(0u, 0u, 0u, 0u);
  for (uint32_t j = (n4 << 2) + threadIdx.x; j < count; j += blockDim.x) p[j] = 0u;
}

// Rounds between two reads of the clock (deadline, serving time slice).
constexpr uint32_t kClockEvery = 8;

// Runs the shuffle of one array inside the calling block: to completion when
// rs is null, else at most `budget` rounds starting from (and saving back to)
// *rs.  `pipelined` turns on the one-round-ahead loads (and L2 prefetches for
// fresh swaps beyond the first block-full); `two` selects the
// two-reservation rule of Algorithm 1 (commit iff the step holds the
// maximum on the slots of both its locations).  Returns the status (0 = ok).
// All control decisions are block-uniform.
template <typename Elem>
__device__ uint32_t run_job(const BatchJob& job, uint32_t* smem, uint32_t fmax, uint32_t sigma, uint64_t deadline_ns,
                            uint64_t t_start, pip_job_stats* st, ResumeState* rs, uint32_t budget,
                            bool pipelined = false, uint64_t slice_ns = 0, bool two = false) {
  __shared__ uint32_t s_cnt[2];
  __shared__ uint32_t s_abort;
  __shared__ uint32_t s_pause;
  const uint64_t t_item = (rs != nullptr && slice_ns != 0) ? globaltimer_ns() : 0;
  const uint32_t n = job.n;
  const uint32_t F = job.F;
  const uint32_t ns = sigma * F + 32u;
  const uint32_t kmax = cta_kmax(F);
  const uint32_t KMAX = cta_kmax(fmax);
  uint32_t* const S = smem;
  uint32_t* const D = smem + cta_table_words(fmax, sigma);
  uint32_t* const Q_base = D + cta_window_words(fmax);  // two queues of KMAX words
  Elem* A = static_cast<Elem*>(job.A);
  const uint32_t tid = threadIdx.x, NT = blockDim.x, lane = tid & 31u;

  uint32_t rounds = 0, max_active = 0;
  uint64_t attempts = 0, losers_total = 0;
  uint32_t status = 0;
  bool done = true;
  if (rs != nullptr) {
    rounds = rs->rounds;
    max_active = rs->max_active;
    attempts = rs->attempts;
    losers_total = rs->losers;
    done = rs->done != 0u;
    status = rs->status;
    if (!rs->started) done = n < 2u;
  } else {
    done = n < 2u;
  }
  uint32_t m = 0;
  if (!done && status == 0u) {
    sclear(S, ns);
    sclear(D, cta_window_words(F));
    if (tid == 0) {
      s_cnt[0] = 0;
      s_cnt[1] = 0;
      s_abort = 0;
    }
    uint32_t Lprev, L, nl;
    if (rs == nullptr || !rs->started) {
      Lprev = n;
      L = n - min(F, n - 1u);
      nl = 0;
    } else {  // resume: reload the carried losers
      L = rs->L;
      Lprev = rs->Lprev;
      nl = rs->nl;
      for (uint32_t p = tid; p < nl; p += NT) Q_base[p] = ldcg(rs->Q + p);
    }
    m = nl + (Lprev - L);
    __syncthreads();
    // tables of the first round: every active swap reserves
    for (uint32_t p = tid; p < m; p += NT) {
      const uint32_t f0 = Lprev - L;
      const uint32_t i = (p < f0) ? Lprev - 1u - p : Q_base[p - f0];
      const uint32_t h = job_target(job, i);
      if (h != i) sreserve(D, S, ns, L, Lprev, i, h, two);
    }
    __syncthreads();
    uint32_t b = 0;  // queue buffer holding the current round's carried losers
    // values loaded one round ahead for this thread's next fresh swap
    Elem px{}, py{};
    uint32_t ph = 0;
    bool pok = false;
    for (uint32_t r = 0;; ++r) {
      const uint32_t f = Lprev - L;  // fresh swaps of this round, [L, Lprev)
      uint32_t* const Qb = Q_base + b * KMAX;
      uint32_t* const Qn = Q_base + (b ^ 1u) * KMAX;
      // ---- early loads for next round's fresh swap i' = L - 1 - tid
      Elem nx{}, ny{};
      uint32_t nh = 0;
      bool nok = false;
      if (pipelined && tid < min(F, L - 1u)) {
        const uint32_t ip = L - 1u - tid;
        nh = job_target(job, ip);
        if (nh != ip) {
          nx = ldcg(A + ip);
          ny = ldcg(A + nh);
          // valid unless a swap of this round targets either location
          nok = S[slot_of(ip, ns)] == 0u && S[slot_of(nh, ns)] == 0u;
        }
      }
      // ---- 1. commit: kCtaU positions per thread, array loads together
      for (uint32_t p0 = tid & ~31u; p0 < m; p0 += kCtaU * NT) {
        uint32_t ii[kCtaU], hh[kCtaU];
        bool win[kCtaU], lose[kCtaU], pre[kCtaU];
#pragma unroll
        for (int j = 0; j < kCtaU; ++j) {
          const uint32_t p = p0 + lane + (uint32_t)j * NT;
          win[j] = false;
          lose[j] = false;
          // the first position of this thread (p == tid) may have its array
          // values and target loaded already
          pre[j] = j == 0 && p0 == (tid & ~31u) && pok && p < m;
          ii[j] = 0;
          hh[j] = 0;
          if (p < m) {
            const uint32_t i = (p < f) ? Lprev - 1u - p : Qb[p - f];
            const uint32_t h = pre[j] ? ph : job_target(job, i);
            ii[j] = i;
            hh[j] = h;
            if (h != i) {
              const uint32_t own = (i < Lprev && !two) ? D[(i - L) >> 5] : S[slot_of(i, ns)];
              const uint32_t rh = S[slot_of(h, ns)];
              const bool own_free = two ? own == i + 1u
                                    : (i < Lprev) ? (((own >> ((i - L) & 31u)) & 1u) == 0u)
                                                  : (own <= i + 1u);
              win[j] = own_free && rh == i + 1u;
              lose[j] = !win[j];
            }
          }
        }
        Elem x[kCtaU], y[kCtaU];
#pragma unroll
        for (int j = 0; j < kCtaU; ++j) {
          if (win[j]) {
            if (pre[j]) {
              x[j] = px;
              y[j] = py;
            } else {
              x[j] = ldcg(A + ii[j]);
              y[j] = ldcg(A + hh[j]);
            }
          }
        }
#pragma unroll
        for (int j = 0; j < kCtaU; ++j) {
          if (win[j]) {
            stcg(A + ii[j], y[j]);
            stcg(A + hh[j], x[j]);
          }
        }
#pragma unroll
        for (int j = 0; j < kCtaU; ++j) {
          const unsigned mask = __ballot_sync(kCtaFull, lose[j]);
          if (mask) {
            const int leader = __ffs(mask) - 1;
            uint32_t base = 0;
            if ((int)lane == leader) base = atomicAdd(&s_cnt[b ^ 1u], (uint32_t)__popc(mask));
            base = __shfl_sync(kCtaFull, base, leader);
            if (lose[j]) {
              const uint32_t q = base + __popc(mask & ((1u << lane) - 1u));
              if (q < kmax) Qn[q] = ii[j];
              else s_abort = PIP_EINTERNAL;
            }
          }
        }
      }
      __syncthreads();
      // ---- 2. size the next fresh block from the losers left; clean
      const uint32_t nl_next = s_cnt[b ^ 1u];
      const uint32_t fn = min(min(F, L - 1u), kmax - min(kmax, nl_next));
      const uint32_t Ln = L - fn;
      sclear(S, ns);
      sclear(D, cta_window_words(F));
      if (tid == 0) {
        s_cnt[b] = 0;
        if (nl_next >= m) s_abort = PIP_EINTERNAL;  // no commit: impossible
        if ((r % kClockEvery) == 0u) {
          const uint64_t now = globaltimer_ns();
          if (now - t_start > deadline_ns) s_abort = PIP_ETIMEOUT;
          // a resumable run also pauses once its time slice is used up
          s_pause = (t_item != 0 && now - t_item >= slice_ns) ? 1u : 0u;
        }
      }
      __syncthreads();
      // ---- 3. the next round's swaps reserve: fresh [Ln, L) from the top
      // down, then the carried losers.  A thread whose first position next
      // round is a carried loser starts that swap's array loads now (this
      // round's stores are complete, so they need no check).
      const uint32_t mn = nl_next + fn;
      for (uint32_t p = tid; p < mn; p += NT) {
        const uint32_t i = (p < fn) ? L - 1u - p : Qn[p - fn];
        const uint32_t h = (p == tid && p < fn && pipelined && tid < min(F, L - 1u)) ? nh : job_target(job, i);
        if (h != i) {
          sreserve(D, S, ns, Ln, L, i, h, two);
          if (pipelined) {
            if (p == tid && p >= fn) {
              nx = ldcg(A + i);
              ny = ldcg(A + h);
              nh = h;
              nok = true;
            } else if (p >= NT && p < fn) {  // beyond the early loads: pull the lines into L2
              asm volatile("prefetch.global.L2 [%0];" ::"l"(A + h));
              asm volatile("prefetch.global.L2 [%0];" ::"l"(A + i));
            }
          }
        }
      }
      __syncthreads();
      rounds += 1u;
      attempts += m;
      losers_total += nl_next;
      max_active = max(max_active, m);
      if (s_abort != 0u) {
        status = s_abort;
        break;
      }
      Lprev = L;
      L = Ln;
      nl = nl_next;
      m = mn;
      b ^= 1u;
      px = nx;
      py = ny;
      ph = nh;
      pok = nok;
      if (m == 0u) break;
      if (m > kmax || rounds > n + 8u) {
        status = PIP_EINTERNAL;
        break;
      }
      if (rs != nullptr && (r + 1u >= budget || s_pause != 0u)) {
        // pause at the round boundary: save the carried losers and the frontier
        const uint32_t* const Qc = Q_base + b * KMAX;
        for (uint32_t p = tid; p < nl; p += NT) stcg(rs->Q + p, Qc[p]);
        if (tid == 0) {
          rs->L = L;
          rs->Lprev = Lprev;
          rs->nl = nl;
          rs->m = m;
        }
        done = false;
        break;
      }
      done = true;
    }
    if (m == 0u || status != 0u) done = true;
  }
  if (tid == 0) {
    if (st != nullptr) {
      st->status = status;
      st->rounds = rounds;
      st->attempts = attempts;
      st->losers = losers_total;
      st->max_active = max_active;
    }
    if (rs != nullptr) {
      rs->started = 1u;
      rs->done = done ? 1u : 0u;
      rs->status = status;
      rs->rounds = rounds;
      rs->attempts = attempts;
      rs->losers = losers_total;
      rs->max_active = max_active;
    }
  }
  __syncthreads();  // the block's smem is reused by its next job
  return status;
}

}  // namespace pip
