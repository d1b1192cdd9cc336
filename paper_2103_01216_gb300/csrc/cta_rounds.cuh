// The block-resident round loop shared by the batched driver and the serving
// tick: one thread block runs the rounds of one array with its reservation
// tables in shared memory.
//
// Round structure (deterministic reservations over the first unfinished
// swaps, Algorithm 1 under the Decomposable Property, Section 4.1; RP-OneRes
// rule and RP-Final dense window, Appendix A.2): round r commits with the
// tables of round r while its losers and the fresh block W_{r+1} reserve into
// the other buffer; after a bar.sync the tables of round r are cleared (the
// cleaning phase of Appendix A.1) and a second bar.sync opens round r+1.
//
// A run can stop after a number of rounds and resume later (serving): at a
// round boundary the state is the frontier L, the end of the current fresh
// block, and the carried losers; on resume the tables of the next round are
// rebuilt from them (the reservations depend on nothing else).
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

__device__ __forceinline__ void sreserve(uint32_t* D, uint32_t* S, uint32_t ns, uint32_t wlo, uint32_t whi,
                                         uint32_t h, uint32_t prio) {
  if (h >= wlo && h < whi) atomicMax(D + (h - wlo), prio);
  else atomicMax(S + slot_of(h, ns), prio);
}

__device__ __forceinline__ void sclear(uint32_t* p, uint32_t count) {
  for (uint32_t j = threadIdx.x; j < count; j += blockDim.x) p[j] = 0u;
}

// Runs the shuffle of one array inside the calling block: to completion when
// rs is null, else at most `budget` rounds starting from (and saving back to)
// *rs.  Returns the status (0 = ok).  All control decisions are block-uniform.
template <typename Elem>
__device__ uint32_t run_job(const BatchJob& job, uint32_t* smem, uint32_t fmax, uint32_t sigma, uint64_t deadline_ns,
                            uint64_t t_start, pip_job_stats* st, ResumeState* rs, uint32_t budget,
                            bool prefetch = false, uint64_t slice_ns = 0) {
  __shared__ uint32_t s_cnt[2];
  __shared__ uint32_t s_abort;
  __shared__ uint32_t s_pause;
  const uint64_t t_item = (rs != nullptr && slice_ns != 0) ? globaltimer_ns() : 0;
  const uint32_t n = job.n;
  const uint32_t F = job.F;
  const uint32_t ns = sigma * F + 32u;
  const uint32_t kmax = F * 5u / 2u + 2u;
  const uint32_t NS = sigma * fmax + 32u;
  const uint32_t KMAX = fmax * 5u / 2u + 2u;
  // buffer k of each table (k = round parity), addressed arithmetically so
  // that nothing is indexed through a local array
  uint32_t* const S_base = smem;
  uint32_t* const D_base = smem + 2 * NS;
  uint32_t* const Q_base = smem + 2 * NS + 2 * fmax;
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
  if (!done && status == 0u) {
    sclear(S_base, ns);
    sclear(S_base + NS, ns);
    sclear(D_base, F);
    sclear(D_base + fmax, F);
    if (tid == 0) {
      s_cnt[0] = 0;
      s_cnt[1] = 0;
      s_abort = 0;
    }
    uint32_t Lprev, L, nl, m;
    if (rs == nullptr || !rs->started) {
      __syncthreads();
      Lprev = n;
      L = n - min(F, n - 1u);
      nl = 0;
      m = Lprev - L;
      for (uint32_t i = L + tid; i < Lprev; i += NT) {
        const uint32_t h = job_target(job, i);
        if (h != i) sreserve(D_base, S_base, ns, L, Lprev, h, i + 1u);
      }
    } else {
      // resume: reload the carried losers and rebuild this round's tables
      L = rs->L;
      Lprev = rs->Lprev;
      nl = rs->nl;
      m = rs->m;
      for (uint32_t p = tid; p < nl; p += NT) Q_base[p] = ldcg(rs->Q + p);
      __syncthreads();
      for (uint32_t p = tid; p < m; p += NT) {
        const uint32_t i = (p < nl) ? Q_base[p] : L + (p - nl);
        const uint32_t h = job_target(job, i);
        if (h != i) sreserve(D_base, S_base, ns, L, Lprev, h, i + 1u);
      }
    }
    __syncthreads();
    for (uint32_t r = 0;; ++r) {
      const uint32_t b = r & 1u, nb = b ^ 1u;
      uint32_t* const Sb = S_base + b * NS;
      uint32_t* const Snb = S_base + nb * NS;
      uint32_t* const Db = D_base + b * fmax;
      uint32_t* const Dnb = D_base + nb * fmax;
      uint32_t* const Qb = Q_base + b * KMAX;
      uint32_t* const Qnb = Q_base + nb * KMAX;
      uint32_t fn = min(F, L - 1u);
      fn = min(fn, kmax - m + 1u);
      const uint32_t Ln = L - fn;
      // ---- commit round r: kCtaU positions per thread, array loads together
      for (uint32_t p0 = tid & ~31u; p0 < m; p0 += kCtaU * NT) {
        uint32_t ii[kCtaU], hh[kCtaU];
        bool win[kCtaU], lose[kCtaU];
#pragma unroll
        for (int j = 0; j < kCtaU; ++j) {
          const uint32_t p = p0 + lane + (uint32_t)j * NT;
          win[j] = false;
          lose[j] = false;
          ii[j] = 0;
          hh[j] = 0;
          if (p < m) {
            const uint32_t i = (p < nl) ? Qb[p] : L + (p - nl);
            const uint32_t h = job_target(job, i);
            ii[j] = i;
            hh[j] = h;
            if (h != i) {
              const uint32_t own = (i < Lprev) ? Db[i - L] : Sb[slot_of(i, ns)];
              const uint32_t rh = (h >= L && h < Lprev) ? Db[h - L] : Sb[slot_of(h, ns)];
              const bool own_free = (i < Lprev) ? (own == 0u) : (own <= i + 1u);
              win[j] = own_free && rh == i + 1u;
              lose[j] = !win[j];
            }
          }
        }
        Elem x[kCtaU], y[kCtaU];
#pragma unroll
        for (int j = 0; j < kCtaU; ++j) {
          if (win[j]) {
            x[j] = ldcg(A + ii[j]);
            y[j] = ldcg(A + hh[j]);
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
          if (lose[j]) sreserve(Dnb, Snb, ns, Ln, L, hh[j], ii[j] + 1u);
          const unsigned mask = __ballot_sync(kCtaFull, lose[j]);
          if (mask) {
            const int leader = __ffs(mask) - 1;
            uint32_t base = 0;
            if ((int)lane == leader) base = atomicAdd(&s_cnt[nb], (uint32_t)__popc(mask));
            base = __shfl_sync(kCtaFull, base, leader);
            if (lose[j]) {
              const uint32_t q = base + __popc(mask & ((1u << lane) - 1u));
              if (q < kmax) Qnb[q] = ii[j];
              else s_abort = PIP_EINTERNAL;
            }
          }
        }
      }
      // ---- fresh block W_{r+1} reserves (and, for a lone array, pulls the
      // array lines it will swap into L2 one round ahead)
      for (uint32_t i = Ln + tid; i < L; i += NT) {
        const uint32_t h = job_target(job, i);
        if (h != i) {
          sreserve(Dnb, Snb, ns, Ln, L, h, i + 1u);
          if (prefetch) {
            asm volatile("prefetch.global.L2 [%0];" ::"l"(A + h));
            asm volatile("prefetch.global.L2 [%0];" ::"l"(A + i));
          }
        }
      }
      __syncthreads();
      const uint32_t nl_next = s_cnt[nb];
      // ---- clean round r's tables; they take round r+2's reservations
      sclear(Sb, ns);
      sclear(Db, F);
      if (tid == 0) {
        s_cnt[b] = 0;
        if (nl_next >= m) s_abort = PIP_EINTERNAL;  // no commit: impossible
        const uint64_t now = globaltimer_ns();
        if (now - t_start > deadline_ns) s_abort = PIP_ETIMEOUT;
        // a resumable run also pauses once its time slice is used up
        s_pause = (t_item != 0 && now - t_item >= slice_ns) ? 1u : 0u;
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
      m = nl_next + fn;
      if (m == 0u) break;
      if (m > kmax || rounds > n + 8u) {
        status = PIP_EINTERNAL;
        break;
      }
      if (rs != nullptr && (r + 1u >= budget || s_pause != 0u)) {
        // pause at the round boundary: save the carried losers (buffer nb
        // holds the next round's queue) and the frontier
        for (uint32_t p = tid; p < nl; p += NT) stcg(rs->Q + p, Qnb[p]);
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
