// Persistent round driver: one cooperative launch walks every round of the
// deterministic-reservation Knuth shuffle (Algorithm 1 under the Decomposable
// Property, Section 4.1; round/prefix framework of Section 7.2 and
// Appendix A.1; reservation rule and dense window of RP-OneRes / RP-Final,
// Appendix A.2) with no host round trip.
//
// Round r (0-based) has an active set of m_r swaps: the n_r losers carried
// from round r-1 (queue Q[r&1]) followed by the fresh block W_r = [L_r, L_{r-1})
// (L_{-1} = n).  Invariant: every unfinished step with index >= L_r is active,
// which is what makes a commit safe (Section 4.1: always work on the first
// unfinished swaps in sequential order).
//
// The rounds are software-pipelined so that one grid barrier per round
// suffices.  Between barriers B_{r-1} and B_r, phase P_r
//   (a) decides round r: step i commits iff no active step targets location i
//       and i holds the maximum priority on its target; winners swap A[i] and
//       A[H[i]]; losers are queued for round r+1 and immediately reserve for it;
//   (b) lets the fresh block W_{r+1} reserve for round r+1;
//   (c) clears the tables of round r-1 (the cleaning phase of Appendix A.1).
// Reservations for round r+1 therefore land in a different table (S/D index
// (r+1)%3) from the one round r reads (r%3) and the one being cleared
// ((r+2)%3).
//
// Reservation structures of one round (priority of step i is i+1, 0 = unset):
//   D (dense window, RP-Final): one word per location of W_r, exact
//     max-priority of the swaps targeting that location.
//   S (slot table): nslots words; a location t outside W_r maps to slot
//     slot_of(t) and the word holds the max priority over all swaps whose
//     target maps there.  Unlike the paper's keyed hash table this table is
//     keyless, so a slot shared by two targets can make a swap fail although
//     it had no real conflict.  Such spurious failures only delay a swap: a
//     swap still commits only if no higher-priority active swap touches either
//     of its locations, and the highest-priority active swap always commits,
//     so every round makes progress and the result is the sequential one.
// Commit test of active step i with target h != i (OneRes rule, Appendix A.2):
//   own location free: D[i - L_r] == 0 for fresh i, S[slot(i)] <= i+1 for a
//     carried loser (every swap targeting i has a higher priority than i);
//   target won:        (h in W_r ? D[h - L_r] : S[slot(h)]) == i+1.
// Self-loops (h == i) never reserve and finish at once (text under Alg. 1).
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

constexpr uint32_t kLoserBuf = 2048;  // per-block staging of losers (8 KB)
// Positions per thread in flight in the commit phase, and the launch bounds:
// 32 registers and 2048 resident threads per SM measured best on GB300 (more
// warps beat deeper per-thread batches for this random-access mix).
#ifndef PIP_KU
#define PIP_KU 2
#endif
#ifndef PIP_MIN_BLOCKS
#define PIP_MIN_BLOCKS 4
#endif
#ifndef PIP_MAX_THREADS
#define PIP_MAX_THREADS 512
#endif
constexpr int kU = PIP_KU;            // positions per thread in flight in the commit phase
constexpr unsigned kFull = 0xffffffffu;


template <bool kExplicit>
__device__ __forceinline__ uint32_t target_of(const GridArgs& a, uint32_t i) {
  if constexpr (kExplicit) return __ldg(a.H + i);
  else return hashed_target(a.seed, i);
}

// Reserve target h for step i in the tables of a round whose fresh window is
// [wlo, whi).
__device__ __forceinline__ void reserve(uint32_t* D, uint32_t* S, uint32_t nslots, uint32_t wlo,
                                        uint32_t whi, uint32_t h, uint32_t prio, uint64_t tpol) {
  if (h >= wlo && h < whi) red_max_hint(D + (h - wlo), prio, tpol);
  else red_max_hint(S + slot_of(h, nslots), prio, tpol);
}

// L2 policies of one thread: for the array and for the reservation tables.
struct Policies {
  uint64_t arr, arr_st, tab;
};
__device__ __forceinline__ Policies make_policies(uint32_t flags) {
  Policies p;
  p.arr = (flags & PIP_FLAG_ARRAY_EVICT_FIRST) ? policy_evict_first() : policy_evict_normal();
  p.arr_st = (flags & (PIP_FLAG_ARRAY_EVICT_FIRST | PIP_FLAG_ARRAY_STORE_EVICT_FIRST)) ? policy_evict_first()
                                                                                        : policy_evict_normal();
  p.tab = (flags & PIP_FLAG_TABLE_EVICT_LAST) ? policy_evict_last() : policy_evict_normal();
  return p;
}

__device__ __forceinline__ void prefetch_l2(const void* p) {
  asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
}

// Fresh block [lo, hi) reserves for the round whose window it is.  With
// PIP_FLAG_PREFETCH the A lines that round will swap are pulled into L2 now,
// one round ahead of the commit that reads them.
template <typename Elem, bool kExplicit>
__device__ __forceinline__ void reserve_fresh(const GridArgs& a, uint32_t lo, uint32_t hi,
                                              uint32_t* D, uint32_t* S, uint32_t tid, uint32_t T,
                                              uint64_t tpol) {
  const bool pf = (a.flags & PIP_FLAG_PREFETCH) != 0u;
  const Elem* A = static_cast<const Elem*>(a.A);
#pragma unroll 4
  for (uint32_t i = lo + tid; i < hi; i += T) {
    const uint32_t h = target_of<kExplicit>(a, i);
    if (h != i) {
      reserve(D, S, a.nslots, lo, hi, h, i + 1, tpol);
      if (pf) {
        prefetch_l2(A + h);
        if ((i & 7u) == 0u || i == lo + tid) prefetch_l2(A + i);
      }
    }
  }
}

__device__ __forceinline__ void clear_words(uint32_t* p, uint32_t count, uint32_t tid, uint32_t T,
                                            uint64_t tpol) {
  // 16-byte stores over the 16-byte aligned body, scalars for the tail
  const uint32_t n4 = count >> 2;
  uint4* p4 = reinterpret_cast<uint4*>(p);
  for (uint32_t j = tid; j < n4; j += T) st_hint(p4 + j, make_uint4(0, 0, 0, 0), tpol);
  for (uint32_t j = (n4 << 2) + tid; j < count; j += T) st_hint(p + j, 0u, tpol);
}

template <typename Elem, bool kExplicit>
__global__ void __launch_bounds__(PIP_MAX_THREADS, PIP_MIN_BLOCKS) rounds_kernel(const GridArgs a) {
  __shared__ uint32_t s_lbuf[kLoserBuf];
  __shared__ uint32_t s_lcount, s_flush, s_base;

  Elem* A = static_cast<Elem*>(a.A);
  Ctrl* ctrl = a.ctrl;
  const uint32_t T = gridDim.x * blockDim.x;
  const uint32_t tid = blockIdx.x * blockDim.x + threadIdx.x;
  const uint32_t lane = threadIdx.x & 31u;
  uint64_t epoch = 0;
  const uint64_t t_start = globaltimer_ns();
  const Policies pol = make_policies(a.flags);

  if (threadIdx.x == 0) s_lcount = 0;
  // an invalid explicit target sequence was reported by the validation pass
  if (ld_relaxed_u32(&ctrl->status) != 0u) goto done;

  {
    // ---- prologue: fresh block W_0 = [n - f_0, n) reserves for round 0
    uint32_t Lprev = a.n;
    uint32_t f = min(a.F, a.n - 1u);
    uint32_t L = a.n - f;
    uint32_t nl = 0;
    uint32_t m = f;
    uint64_t attempts = 0, losers_total = 0;
    uint32_t max_active = 0, rounds = 0;
    reserve_fresh<Elem, kExplicit>(a, L, Lprev, a.D[0], a.S[0], tid, T, pol.tab);
    const bool arrive = !((a.flags & PIP_FLAG_TEST_SKIP_BARRIER) && blockIdx.x == 0);
    if (!grid_barrier(&ctrl->barrier, gridDim.x, epoch, &ctrl->status, a.timeout_ns, arrive)) goto done;

    for (uint32_t r = 0;; ++r) {
      const uint32_t b = r % 3u, b1 = (r + 1u) % 3u, b2 = (r + 2u) % 3u;
      uint32_t* const Dr = a.D[b];
      uint32_t* const Sr = a.S[b];
      uint32_t* const Dn = a.D[b1];
      uint32_t* const Sn = a.S[b1];
      uint32_t* const Qin = a.Q[r & 1u];
      uint32_t* const Qout = a.Q[(r + 1u) & 1u];
      uint32_t* const cnt_out = &ctrl->cnt[b1];

      // next round's fresh block W_{r+1} = [Ln, L); throttled so that
      // m_{r+1} <= (m_r - 1) + fn <= kmax (at least one swap of round r
      // commits), which bounds the loser queue; with kmax = 2.5 F the
      // throttle only acts when more than half a block of losers piles up
      uint32_t fn = min(a.F, L - 1u);
      fn = min(fn, a.kmax - m + 1u);
      const uint32_t Ln = L - fn;

      if (tid == 0) {
        stcg(&ctrl->cnt[b2], 0u);  // counter of round r+2's losers
        if (globaltimer_ns() - t_start > a.deadline_ns) set_status(&ctrl->status, PIP_ETIMEOUT);
      }

      // ---- (a) commit round r.  Each thread takes kU positions at a time
      // (p, p+T, ..., p+(kU-1)T) and issues their loads together so that kU
      // independent memory chains are in flight per thread.
      for (uint32_t p0 = tid & ~31u; p0 < m; p0 += kU * T) {
        uint32_t ii[kU], hh[kU], own[kU], rh[kU];
        bool act[kU];
#pragma unroll
        for (int j = 0; j < kU; ++j) {
          const uint32_t p = p0 + lane + (uint32_t)j * T;
          act[j] = p < m;
          ii[j] = 0;
          if (act[j]) ii[j] = (p < nl) ? ld_hint(Qin + p, pol.tab) : L + (p - nl);
        }
#pragma unroll
        for (int j = 0; j < kU; ++j) {
          hh[j] = act[j] ? target_of<kExplicit>(a, ii[j]) : 0u;
          act[j] = act[j] && hh[j] != ii[j];  // self-loops finish at once
        }
        Elem x[kU], y[kU];
        const bool spec = (a.flags & PIP_FLAG_SPECULATE) != 0u;
        if (spec) {  // array loads issued before the decision (wasted for losers)
#pragma unroll
          for (int j = 0; j < kU; ++j) {
            if (act[j]) {
              x[j] = ld_hint(A + ii[j], pol.arr);
              y[j] = ld_hint(A + hh[j], pol.arr);
            }
          }
        }
#pragma unroll
        for (int j = 0; j < kU; ++j) {
          own[j] = 0;
          rh[j] = 0;
          if (act[j]) {
            const uint32_t i = ii[j], h = hh[j];
            own[j] = (i < Lprev) ? ld_hint(Dr + (i - L), pol.tab) : ld_hint(Sr + slot_of(i, a.nslots), pol.tab);
            rh[j] = (h >= L && h < Lprev) ? ld_hint(Dr + (h - L), pol.tab)
                                          : ld_hint(Sr + slot_of(h, a.nslots), pol.tab);
          }
        }
        bool win[kU];
#pragma unroll
        for (int j = 0; j < kU; ++j) {
          const uint32_t i = ii[j];
          // own location free: exact window word unset, or every swap mapping to
          // the slot of i has a priority at most i+1 (so none targets i)
          const bool own_free = (i < Lprev) ? (own[j] == 0u) : (own[j] <= i + 1u);
          win[j] = act[j] && own_free && rh[j] == i + 1u;
          if (win[j] && !spec) {
            x[j] = ld_hint(A + ii[j], pol.arr);
            y[j] = ld_hint(A + hh[j], pol.arr);
          }
        }
#pragma unroll
        for (int j = 0; j < kU; ++j) {
          if (win[j]) {
            st_hint(A + ii[j], y[j], pol.arr_st);
            st_hint(A + hh[j], x[j], pol.arr_st);
          }
        }
#pragma unroll
        for (int j = 0; j < kU; ++j) {
          const bool lose = act[j] && !win[j];
          if (lose) reserve(Dn, Sn, a.nslots, Ln, L, hh[j], ii[j] + 1u, pol.tab);
          const unsigned mask = __ballot_sync(kFull, lose);
          if (mask) {
            const int leader = __ffs(mask) - 1;
            uint32_t wbase = 0;
            if ((int)lane == leader) wbase = atomicAdd(&s_lcount, (uint32_t)__popc(mask));
            wbase = __shfl_sync(kFull, wbase, leader);
            if (lose) {
              const uint32_t idx = wbase + __popc(mask & ((1u << lane) - 1u));
              if (idx < kLoserBuf) {
                s_lbuf[idx] = ii[j];
              } else {  // staging full: direct append
                const uint32_t q = atomicAdd(cnt_out, 1u);
                if (q < a.kmax) st_hint(Qout + q, ii[j], pol.tab);
                else set_status(&ctrl->status, PIP_EINTERNAL);
              }
            }
          }
        }
      }
      // flush the block's staged losers with one global atomic
      __syncthreads();
      if (threadIdx.x == 0) {
        const uint32_t c = min(s_lcount, kLoserBuf);
        s_flush = c;
        s_base = c ? atomicAdd(cnt_out, c) : 0u;
        s_lcount = 0;
      }
      __syncthreads();
      if (s_base + s_flush <= a.kmax) {
        for (uint32_t j = threadIdx.x; j < s_flush; j += blockDim.x) st_hint(Qout + s_base + j, s_lbuf[j], pol.tab);
      } else if (threadIdx.x == 0) {
        set_status(&ctrl->status, PIP_EINTERNAL);  // cannot happen: some swap commits every round
      }

      // ---- (b) fresh block of round r+1 reserves
      reserve_fresh<Elem, kExplicit>(a, Ln, L, Dn, Sn, tid, T, pol.tab);

      // ---- (c) clean round r-1's tables (they become round r+2's)
      clear_words(a.S[b2], a.nslots, tid, T, pol.tab);
      clear_words(a.D[b2], a.F, tid, T, pol.tab);

      if (!grid_barrier(&ctrl->barrier, gridDim.x, epoch, &ctrl->status, a.timeout_ns)) goto done;

      const uint32_t nl_next = ldcg(cnt_out);
      if (nl_next >= m) {  // no swap committed: impossible (the top active swap always wins)
        if (tid == 0) set_status(&ctrl->status, PIP_EINTERNAL);
        break;
      }
      rounds = r + 1u;
      attempts += m;
      losers_total += nl_next;
      max_active = max(max_active, m);
      Lprev = L;
      L = Ln;
      nl = nl_next;
      m = nl_next + fn;
      if (m == 0u) break;
      if (m > a.kmax || rounds >= a.max_rounds) {
        if (tid == 0) set_status(&ctrl->status, PIP_EINTERNAL);
        break;
      }
    }
    if (tid == 0 && a.stats != nullptr) {
      a.stats->rounds = rounds;
      a.stats->attempts = attempts;
      a.stats->losers = losers_total;
      a.stats->max_active = max_active;
      a.stats->grid_blocks = gridDim.x;
    }
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

template <typename Elem, bool kExplicit>
const void* kernel_ptr() {
  return reinterpret_cast<const void*>(&rounds_kernel<Elem, kExplicit>);
}

const void* select_kernel(uint32_t elem_bytes, bool explicit_h) {
  switch (elem_bytes) {
    case 4: return explicit_h ? kernel_ptr<uint32_t, true>() : kernel_ptr<uint32_t, false>();
    case 8: return explicit_h ? kernel_ptr<unsigned long long, true>() : kernel_ptr<unsigned long long, false>();
    case 16: return explicit_h ? kernel_ptr<uint4, true>() : kernel_ptr<uint4, false>();
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

uint32_t grid_driver_max_blocks(uint32_t elem_bytes, bool explicit_h, uint32_t threads) {
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
  static std::map<std::tuple<int, const void*, uint32_t>, int> cache;
  std::lock_guard<std::mutex> lk(mu);
  const auto key = std::make_tuple(dev, k, threads);
  auto it = cache.find(key);
  if (it == cache.end()) {
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, (int)threads, 0) != cudaSuccess) {
      cudaGetLastError();
      return 0;
    }
    it = cache.emplace(key, per_sm).first;
  }
  return (uint32_t)it->second * (uint32_t)di.sms;
}

pip_status launch_grid_driver(const Plan& plan, void* A, const uint32_t* H, uint64_t seed, void* aux,
                              pip_stats* stats, cudaStream_t stream) {
  const void* k = select_kernel(plan.elem_bytes, H != nullptr);
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
  a.ctrl = reinterpret_cast<Ctrl*>(base);
  a.stats = stats;
  a.timeout_ns = plan.timeout_ns;
  a.max_rounds = plan.n + 8u;
  a.deadline_ns = plan.deadline_ns;
  a.flags = plan.flags;
  a.latch = error_latch_ptr();
  if (a.latch == nullptr) return PIP_ECUDA;

  if (cudaMemsetAsync(aux, 0, plan.aux_bytes, stream) != cudaSuccess) return PIP_ECUDA;
  if (H != nullptr) {
    const uint32_t vb = (uint32_t)std::min<uint64_t>(1024, (plan.n + 255) / 256);
    validate_targets_kernel<<<vb, 256, 0, stream>>>(H, plan.n, a.ctrl);
    if (cudaGetLastError() != cudaSuccess) return PIP_ECUDA;
  }
  // every block must be co-resident (the cooperative launch refuses otherwise)
  uint32_t blocks = plan.blocks;
  const uint32_t maxb = grid_driver_max_blocks(plan.elem_bytes, H != nullptr, plan.threads);
  if (maxb == 0) return PIP_ECUDA;
  blocks = std::max(1u, std::min(blocks, maxb));
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = dim3(blocks);
  cfg.blockDim = dim3(plan.threads);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  void* args[] = {&a};
  if (cudaLaunchKernelExC(&cfg, k, args) != cudaSuccess) {
    cudaGetLastError();
    return PIP_ECUDA;
  }
  return PIP_OK;
}

}  // namespace pip
