// Device primitives shared by the round kernels: the swap-target generator,
// the reservation-slot map, L2-coherent loads/stores and the bounded grid
// barrier with its per-round counting word.  sm_103a only.
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

// ---- L2 eviction-priority policies (createpolicy) and hinted stores.
__device__ __forceinline__ uint64_t policy_evict_first() {
  uint64_t p;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
  return p;
}
__device__ __forceinline__ uint64_t policy_evict_normal() {
  uint64_t p;
  asm volatile("createpolicy.fractional.L2::evict_normal.b64 %0, 1.0;" : "=l"(p));
  return p;
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
// Exchange at L2: stores v into *p and returns the previous content, as one
// atomic read-modify-write performed in the L2 slice that owns the line.  A
// swap's random side done this way costs one L2 transaction instead of a
// load and a later store of the same line (measured on GB300 at 10^9 random
// targets: 44 ms against 60 ms for 8-byte elements, 51 against 68 ms for
// 16-byte ones).  16-byte elements use the b128 form (16-byte aligned p).
__device__ __forceinline__ uint32_t exch_hint(uint32_t* p, uint32_t v, uint64_t pol) {
  uint32_t old;
  asm volatile("atom.relaxed.gpu.global.exch.L2::cache_hint.b32 %0, [%1], %2, %3;"
               : "=r"(old)
               : "l"(p), "r"(v), "l"(pol)
               : "memory");
  return old;
}
__device__ __forceinline__ unsigned long long exch_hint(unsigned long long* p, unsigned long long v, uint64_t pol) {
  unsigned long long old;
  asm volatile("atom.relaxed.gpu.global.exch.L2::cache_hint.b64 %0, [%1], %2, %3;"
               : "=l"(old)
               : "l"(p), "l"(v), "l"(pol)
               : "memory");
  return old;
}
__device__ __forceinline__ uint4 exch_hint(uint4* p, uint4 v, uint64_t pol) {
  const unsigned long long vlo = ((unsigned long long)v.y << 32) | v.x;
  const unsigned long long vhi = ((unsigned long long)v.w << 32) | v.z;
  unsigned long long lo, hi;
  asm volatile(
      "{\n\t.reg .b128 nv, ov;\n\t"
      "mov.b128 nv, {%2, %3};\n\t"
      "atom.relaxed.gpu.global.exch.L2::cache_hint.b128 ov, [%4], nv, %5;\n\t"
      "mov.b128 {%0, %1}, ov;\n\t}"
      : "=l"(lo), "=l"(hi)
      : "l"(vlo), "l"(vhi), "l"(p), "l"(pol)
      : "memory");
  return make_uint4((uint32_t)lo, (uint32_t)(lo >> 32), (uint32_t)hi, (uint32_t)(hi >> 32));
}
// Fire-and-forget atomic max and or (no value returned to the thread).
__device__ __forceinline__ void red_max(uint32_t* p, uint32_t v) {
  asm volatile("red.relaxed.gpu.global.max.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ void red_or(uint32_t* p, uint32_t v) {
  asm volatile("red.relaxed.gpu.global.or.b32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ void fence_acq_rel_gpu() { asm volatile("fence.acq_rel.gpu;" ::: "memory"); }

__device__ __forceinline__ uint64_t ld_relaxed_u64(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void red_relaxed_add_u64(unsigned long long* p, unsigned long long v) {
  asm volatile("red.relaxed.gpu.global.add.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

__device__ __forceinline__ void red_release_add_u64(unsigned long long* p, unsigned long long v) {
  asm volatile("red.release.gpu.global.add.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

__device__ __forceinline__ unsigned long long ld_acquire_u64(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ uint32_t ld_relaxed_u32(const uint32_t* p) {
  uint32_t v;
  asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ uint64_t globaltimer_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// The status word as one value for the whole block: thread 0 reads it and
// shares it.  A decision that changes a block's control flow around a
// barrier must be taken from this, never from each thread's own read: a word
// that another block sets while this block's warps read it would otherwise
// send part of the block past a __syncthreads the rest still waits at.
__device__ __forceinline__ uint32_t block_status(const uint32_t* status) {
  __shared__ uint32_t s_block_status;
  __syncthreads();  // earlier readers of s_block_status are done
  if (threadIdx.x == 0) s_block_status = ld_relaxed_u32(status);
  __syncthreads();
  return s_block_status;
}

// Records the first error of a run; later errors are dropped.
__device__ __forceinline__ void set_status(uint32_t* status, uint32_t code) {
  atomicCAS(status, 0u, code);
}

// ---------------------------------------------------------------- barrier
// Bounded grid-wide barrier through one 64-bit word per round, which also
// carries per-block sums:
//   bits  0..9   arriving blocks (at most 1023 blocks),
//   bits 10..19  blocks that recorded an error during the phase,
//   bits 20..41  sum of count0 (at most 2^22 - 1),
//   bits 42..63  sum of count1 (at most 2^22 - 1).
// Thread 0 of each block publishes the block's work (the bar.sync, then its
// contribution added with a gpu-scope release) and then polls with acquire
// loads until the arrival field reaches nblocks; a closing bar.sync hands
// the ordering to the whole block.  The word must be zero before the first arrival and is reset by the
// caller once no block can still be polling it.  The wait gives up after
// `timeout_ns`, or as soon as another block has recorded an error in
// `status` (recording PIP_ETIMEOUT on a timeout).  `arrive == false` skips
// the arrival (a test hook that makes every other block's wait run out).
constexpr uint32_t kBwArriveBits = 10, kBwErrBits = 10, kBwCountBits = 22;
constexpr uint64_t kBwArriveMask = (1ull << kBwArriveBits) - 1ull;
constexpr uint32_t kBwMaxBlocks = (1u << kBwArriveBits) - 1u;
constexpr uint32_t kBwMaxCount = (1u << kBwCountBits) - 1u;

struct RoundSum {
  uint32_t count0, count1;  // sums over all blocks
  uint32_t errors;          // blocks that flagged an error
};

// Thread 0's part: arrive, then wait; returns the completed word, or ~0 when
// the wait gave up.
__device__ __forceinline__ unsigned long long round_barrier_wait(unsigned long long* word, uint32_t nblocks,
                                                                 unsigned long long add, uint32_t* status,
                                                                 uint64_t timeout_ns, bool arrive) {
  // The arrival is a release and every poll an acquire (measured 2-12 %
  // cheaper per barrier than a relaxed add and relaxed polls between two
  // acq_rel fences, the same ordering).
  if (arrive) red_release_add_u64(word, add);
  uint64_t t0 = 0;
  uint32_t polls = 0;
  unsigned long long v;
  while (((v = ld_acquire_u64(word)) & kBwArriveMask) < nblocks) {
    if ((++polls & 63u) == 0) {
      if (ld_relaxed_u32(status) != 0u) return ~0ull;
      const uint64_t now = globaltimer_ns();
      if (t0 == 0) t0 = now;
      else if (now - t0 > timeout_ns) {
        set_status(status, PIP_ETIMEOUT);
        return ~0ull;
      }
    }
  }
  return v;
}

// The whole block: bar.sync, thread 0 arrives with (count0, count1, error
// flag) and waits, then calls on_done(ok, sums) -- ok is false when the wait
// gave up -- and a closing bar.sync publishes what on_done wrote to shared
// memory.
template <typename OnDone>
__device__ __forceinline__ void round_barrier(unsigned long long* word, uint32_t nblocks, uint32_t count0,
                                              uint32_t count1, bool err, uint32_t* status, uint64_t timeout_ns,
                                              bool arrive, OnDone on_done) {
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned long long add = 1ull + ((unsigned long long)(err ? 1u : 0u) << kBwArriveBits) +
                                   ((unsigned long long)count0 << (kBwArriveBits + kBwErrBits)) +
                                   ((unsigned long long)count1 << (kBwArriveBits + kBwErrBits + kBwCountBits));
    const unsigned long long v = round_barrier_wait(word, nblocks, add, status, timeout_ns, arrive);
    RoundSum sum;
    sum.errors = (uint32_t)((v >> kBwArriveBits) & ((1ull << kBwErrBits) - 1ull));
    sum.count0 = (uint32_t)((v >> (kBwArriveBits + kBwErrBits)) & kBwMaxCount);
    sum.count1 = (uint32_t)(v >> (kBwArriveBits + kBwErrBits + kBwCountBits));
    on_done(v != ~0ull, sum);
  }
  __syncthreads();
}

}  // namespace pip
