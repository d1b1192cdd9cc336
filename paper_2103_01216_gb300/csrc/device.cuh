// Device primitives shared by the round kernels: the swap-target generator,
// the reservation-slot map, L2-coherent loads/stores and the bounded grid
// barrier.  sm_103a only.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "pip.h"

namespace pip {

// ---------------------------------------------------------------- targets
// Swap target of step i (Section 4.1: H[i] uniform on [0, i], 0-based).
// H[i] = mulhi64(splitmix64(seed ^ i), i + 1): one SplitMix64 output step
// (Steele, Lea, Flood 2014) from state seed^i, reduced to [0, i] by the high
// half of a 64x64-bit product (multiply-shift range reduction).
__device__ __forceinline__ uint64_t splitmix64(uint64_t x) {
  uint64_t z = x + 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

__device__ __forceinline__ uint32_t hashed_target(uint64_t seed, uint32_t i) {
  return (uint32_t)__umul64hi(splitmix64(seed ^ (uint64_t)i), (uint64_t)i + 1ull);
}

// ---------------------------------------------------------------- slot map
// Location -> reservation slot in [0, nslots): a 32-bit finaliser (the
// MurmurHash3 fmix32 mixing steps) followed by a multiply-high range
// reduction, so any slot count works.  Collisions only cost spurious retries.
__device__ __forceinline__ uint32_t slot_of(uint32_t loc, uint32_t nslots) {
  uint32_t h = loc;
  h ^= h >> 16;
  h *= 0x85EBCA6Bu;
  h ^= h >> 13;
  h *= 0xC2B2AE35u;
  h ^= h >> 16;
  return __umulhi(h, nslots);
}

// ---------------------------------------------------------------- memory
// Everything that other blocks write during the kernel is read at L2 (".cg")
// so that no stale L1 line is ever used; stores go to L2 as well.
template <typename T>
__device__ __forceinline__ T ldcg(const T* p) { return __ldcg(p); }
template <typename T>
__device__ __forceinline__ void stcg(T* p, T v) { __stcg(p, v); }

// ---- L2 eviction-priority policies (createpolicy) and hinted accesses.
// The array A is streamed through L2 once per swap, so its accesses can be
// marked evict-first; the reservation tables are reused within a round and
// can be marked evict-last, so that the array does not push them out.
__device__ __forceinline__ uint64_t policy_evict_first() {
  uint64_t p;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
  return p;
}
__device__ __forceinline__ uint64_t policy_evict_last() {
  uint64_t p;
  asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
  return p;
}
__device__ __forceinline__ uint64_t policy_evict_normal() {
  uint64_t p;
  asm volatile("createpolicy.fractional.L2::evict_normal.b64 %0, 1.0;" : "=l"(p));
  return p;
}

__device__ __forceinline__ uint32_t ld_hint(const uint32_t* p, uint64_t pol) {
  uint32_t v;
  asm volatile("ld.global.cg.L2::cache_hint.u32 %0, [%1], %2;" : "=r"(v) : "l"(p), "l"(pol) : "memory");
  return v;
}
__device__ __forceinline__ unsigned long long ld_hint(const unsigned long long* p, uint64_t pol) {
  unsigned long long v;
  asm volatile("ld.global.cg.L2::cache_hint.u64 %0, [%1], %2;" : "=l"(v) : "l"(p), "l"(pol) : "memory");
  return v;
}
__device__ __forceinline__ uint4 ld_hint(const uint4* p, uint64_t pol) {
  uint4 v;
  asm volatile("ld.global.cg.L2::cache_hint.v4.u32 {%0, %1, %2, %3}, [%4], %5;"
               : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
               : "l"(p), "l"(pol)
               : "memory");
  return v;
}
__device__ __forceinline__ void st_hint(uint32_t* p, uint32_t v, uint64_t pol) {
  asm volatile("st.global.cg.L2::cache_hint.u32 [%0], %1, %2;" ::"l"(p), "r"(v), "l"(pol) : "memory");
}
__device__ __forceinline__ void st_hint(unsigned long long* p, unsigned long long v, uint64_t pol) {
  asm volatile("st.global.cg.L2::cache_hint.u64 [%0], %1, %2;" ::"l"(p), "l"(v), "l"(pol) : "memory");
}
__device__ __forceinline__ void st_hint(uint4* p, uint4 v, uint64_t pol) {
  asm volatile("st.global.cg.L2::cache_hint.v4.u32 [%0], {%1, %2, %3, %4}, %5;" ::"l"(p), "r"(v.x), "r"(v.y),
               "r"(v.z), "r"(v.w), "l"(pol)
               : "memory");
}
// Fire-and-forget atomic max (no value returned to the thread).
__device__ __forceinline__ void red_max_hint(uint32_t* p, uint32_t v, uint64_t pol) {
  asm volatile("red.relaxed.gpu.global.max.L2::cache_hint.u32 [%0], %1, %2;" ::"l"(p), "r"(v), "l"(pol)
               : "memory");
}

__device__ __forceinline__ uint64_t ld_acquire_u64(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ uint32_t ld_relaxed_u32(const uint32_t* p) {
  uint32_t v;
  asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void red_release_add_u64(unsigned long long* p, unsigned long long v) {
  asm volatile("red.release.gpu.global.add.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

__device__ __forceinline__ uint64_t globaltimer_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Records the first error of a run; later errors are dropped.
__device__ __forceinline__ void set_status(uint32_t* status, uint32_t code) {
  atomicCAS(status, 0u, code);
}

// ---------------------------------------------------------------- barrier
// Bounded grid-wide barrier over `nblocks` co-resident blocks.  `counter` is
// a monotone 64-bit arrival count: barrier number b (0-based) completes when
// it reaches (b+1)*nblocks, so it never needs resetting.  Thread 0 of each
// block arrives with release semantics and waits with acquire loads; the
// block's bar.sync on either side extends the ordering to all its threads.
// The wait gives up after `timeout_ns`, or as soon as another block has
// recorded an error, and the function then returns false (status set) so the
// caller can leave the kernel; every block then exits at its next barrier.
// One thread's part of the barrier: arrive (release) unless `arrive` is
// false, then wait (acquire) for barrier number `epoch` to complete, bounded
// by `timeout_ns` and by an error recorded elsewhere.  Returns 1 on success.
__device__ __forceinline__ uint32_t barrier_arrive_wait(unsigned long long* counter, uint32_t nblocks,
                                                        uint64_t epoch, uint32_t* status, uint64_t timeout_ns,
                                                        bool arrive) {
  uint32_t ok = 1;
  const uint64_t target = (epoch + 1) * (uint64_t)nblocks;
  if (arrive) {
    __threadfence();
    red_release_add_u64(counter, 1ull);
  }
  uint64_t t0 = 0;
  uint32_t polls = 0;
  while (ld_acquire_u64(counter) < target) {
    if ((++polls & 63u) == 0) {
      if (ld_relaxed_u32(status) != 0u) { ok = 0; break; }
      const uint64_t now = globaltimer_ns();
      if (t0 == 0) t0 = now;
      else if (now - t0 > timeout_ns) {
        set_status(status, PIP_ETIMEOUT);
        ok = 0;
        break;
      }
    }
  }
  if (ok && ld_relaxed_u32(status) != 0u) ok = 0;
  return ok;
}

__device__ __forceinline__ bool grid_barrier(unsigned long long* counter, uint32_t nblocks,
                                             uint64_t& epoch, uint32_t* status,
                                             uint64_t timeout_ns, bool arrive = true) {
  __shared__ uint32_t s_ok;
  __syncthreads();
  if (threadIdx.x == 0) s_ok = barrier_arrive_wait(counter, nblocks, epoch, status, timeout_ns, arrive);
  __syncthreads();
  epoch += 1;
  return s_ok != 0u;
}

}  // namespace pip
