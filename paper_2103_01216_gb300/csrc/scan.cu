// In-place exclusive scan (Section 5.1, Algorithm 3: the output of
// In-Place-Scan, exclusive prefix sums and the total, computed in place with
// only a bounded amount of auxiliary space).
//
// The GPU design is a single pass over the array in tiles of 96 KB with
// decoupled look-back: block b of a grid of G resident blocks takes tiles
// b, b + G, ..., moves each into shared memory with a bulk asynchronous copy
// (cp.async.bulk, completion on an mbarrier; the next tile's copy is in
// flight while the current one is scanned), scans it there, publishes the
// tile's sum in a descriptor, derives the sum of everything before the tile
// from its predecessors' descriptors (the look-back, 32 descriptors per
// round trip), publishes the inclusive prefix, adds the prefix and writes
// the tile back with a bulk copy from shared memory.  Each element is read
// once and written once: the pass is bound by HBM bandwidth.
//
// The descriptors form a ring of kRing entries reused modulo kRing, tagged
// with the tile index; at most two tiles per resident block are in flight
// (one being scanned, the next one loading) and a look-back reaches back at
// most that far, so a ring of more than four times the resident blocks is
// never overwritten while it is read.  The auxiliary
// space is therefore a constant (the ring and a control block, about 32 KB),
// whatever n -- the space bound of the paper's strong PIP algorithm.
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

// Tile size and block size: 96 KB tiles (two per block, one block per SM)
// and 1024 threads measured best on GB300 (57 % of the HBM copy bandwidth at
// 10^9 elements, against 44-56 % for 32-64 KB tiles): a tile's look-back
// costs a few L2 round trips whatever its size, so larger tiles spend less
// of the pass waiting for it.
#ifndef PIP_SCAN_THREADS
#define PIP_SCAN_THREADS 1024
#endif
#ifndef PIP_SCAN_TILE_KB
#define PIP_SCAN_TILE_KB 96
#endif
constexpr uint32_t kScanThreads = PIP_SCAN_THREADS;
constexpr uint32_t kTileBytes = PIP_SCAN_TILE_KB * 1024;  // per block and tile
constexpr uint32_t kRing = 4096;        // descriptors, a power of two
constexpr uint64_t kFlagAgg = 1, kFlagPrefix = 2;

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

struct ScanDesc {
  unsigned long long w[2];
};

__device__ __forceinline__ unsigned long long desc_word(uint64_t tile, uint64_t flag, uint32_t half) {
  return ((tile & kTagMask) << 40) | (flag << 38) | (unsigned long long)half;
}

template <typename T>
__device__ __forceinline__ void desc_publish(ScanDesc* d, uint64_t tile, uint64_t flag, T value) {
  const unsigned long long v = (unsigned long long)value;
  __stcg(&d->w[1], desc_word(tile, flag, (uint32_t)(v >> 32)));
  __stcg(&d->w[0], desc_word(tile, flag, (uint32_t)v));
}

// 0 when the descriptor does not (yet) describe `tile`; else its flag, with
// the value in *value.
template <typename T>
__device__ __forceinline__ uint64_t desc_read(const ScanDesc* d, uint64_t tile, T* value) {
  const unsigned long long a = __ldcg(&d->w[0]);
  const unsigned long long b = __ldcg(&d->w[1]);
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

// Warp 0's part of a tile: the decoupled look-back.  Lane k reads the
// descriptor of tile t-1-k, 32 predecessors per round trip, and the warp
// adds the aggregates back to the nearest published inclusive prefix.
// Returns the exclusive prefix of tile t (in every lane), or sets *fail.
template <typename T>
__device__ __forceinline__ T look_back(const ScanDesc* ring, uint64_t t, uint32_t lane, ScanCtrl* ctrl,
                                       uint64_t timeout_ns, uint32_t* fail) {
  T prefix = 0;
  int64_t top = (int64_t)t - 1;  // highest predecessor not yet accounted for
  uint64_t t0 = 0;
  uint32_t polls = 0;
  while (top >= 0) {
    const int64_t j = top - (int64_t)lane;
    uint64_t flag = 1;  // lanes beyond tile 0 count as ready aggregates of 0
    T val = 0;
    if (j >= 0) flag = desc_read<T>(ring + (j & (kRing - 1)), (uint64_t)j, &val);
    // the window is usable up to (and including) the nearest inclusive
    // prefix; every descriptor before it must be ready
    const unsigned pmask = __ballot_sync(0xffffffffu, flag == kFlagPrefix);
    const uint32_t stop = pmask ? (uint32_t)(__ffs(pmask) - 1) : 31u;
    const unsigned rmask = __ballot_sync(0xffffffffu, flag != 0);
    const unsigned need = stop == 31u ? 0xffffffffu : ((1u << (stop + 1u)) - 1u);
    if ((rmask & need) == need) {
      T v = lane <= stop ? val : T(0);
#pragma unroll
      for (uint32_t d = 16; d >= 1; d >>= 1) v += __shfl_xor_sync(0xffffffffu, v, d);
      prefix += v;
      if (pmask || top < 32) break;  // reached a prefix, or tile 0
      top -= 32;
      continue;
    }
    if ((++polls & 63u) == 0u) {
      uint32_t bad = 0;
      if (lane == 0) {
        if (ld_relaxed_u32(&ctrl->status) != 0u) bad = 1;
        const uint64_t now = globaltimer_ns();
        if (t0 == 0) t0 = now;
        else if (now - t0 > timeout_ns) {
          set_status(&ctrl->status, PIP_ETIMEOUT);
          bad = 1;
        }
      }
      if (__shfl_sync(0xffffffffu, bad, 0)) {
        *fail = 1u;
        return 0;
      }
    }
  }
  return prefix;
}

// One pass over tiles of kItems elements (kItems / kScanThreads per thread).
// Block b takes tiles b, b + G, b + 2G, ... (G = grid size, every block
// resident), with two tile buffers so that the next tile's bulk load
// overlaps the current tile's scan and write-back.
template <typename T>
__global__ void __launch_bounds__(kScanThreads) scan_kernel(T* A, uint64_t n, T* total_out, ScanCtrl* ctrl,
                                                            ScanDesc* ring, uint64_t timeout_ns, uint32_t* latch) {
  constexpr uint32_t kItems = kTileBytes / sizeof(T);
  constexpr uint32_t kPer = kItems / kScanThreads;
  extern __shared__ __align__(128) unsigned char s_raw[];
  T* const s_buf = reinterpret_cast<T*>(s_raw);  // two tiles of kItems
  __shared__ __align__(8) uint64_t s_bar[2];
  __shared__ T s_warp[kScanThreads / 32];
  __shared__ T s_prefix;
  __shared__ uint32_t s_fail;
  const uint32_t tid = threadIdx.x, lane = tid & 31u, warp = tid >> 5;
  const uint64_t ntiles = (n + kItems - 1) / kItems;
  const uint64_t G = gridDim.x;
  if (tid == 0) {
    mbar_init(&s_bar[0], 1);
    mbar_init(&s_bar[1], 1);
    s_fail = 0;
  }
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  __syncthreads();
  // starts the bulk load of tile u into buffer b (full tiles; the ragged last
  // one is read with plain loads when it is processed)
  auto start_load = [&](uint64_t u, uint32_t b) {
    if (tid == 0 && u < ntiles && (u + 1) * kItems <= n) {
      mbar_expect_tx(&s_bar[b], kTileBytes);
      bulk_load(s_buf + b * kItems, A + u * kItems, kTileBytes, &s_bar[b]);
    }
  };
  uint32_t phase[2] = {0u, 0u};
  uint32_t b = 0;
  start_load(blockIdx.x, 0);
  for (uint64_t t = blockIdx.x; t < ntiles; t += G, b ^= 1u) {
    T* const tile = s_buf + b * kItems;
    // the other buffer's bulk store has read its source, then the next
    // tile's load starts there
    if (tid == 0) bulk_wait_read();
    start_load(t + G, b ^ 1u);
    const uint64_t base = t * kItems;
    const bool full = base + kItems <= n;
    const uint32_t cnt = full ? kItems : (uint32_t)(n - base);
    if (full) {
      if (!mbar_wait(&s_bar[b], phase[b], timeout_ns)) {
        set_status(&ctrl->status, PIP_ETIMEOUT);
        s_fail = 1u;
      }
      phase[b] ^= 1u;
    } else {
      for (uint32_t j = tid; j < kItems; j += kScanThreads) tile[j] = j < cnt ? ldcg(A + base + j) : T(0);
    }
    __syncthreads();
    if (s_fail != 0u) break;
    // ---- scan: each thread its kPer consecutive elements, then the block
    T v[kPer];
    T run = 0;
#pragma unroll
    for (uint32_t k = 0; k < kPer; ++k) {
      v[k] = run;
      run += tile[tid * kPer + k];
    }
    const T incl = warp_incl_scan(run, lane);
    if (lane == 31) s_warp[warp] = incl;
    __syncthreads();
    if (warp == 0) {
      const T w = lane < kScanThreads / 32 ? s_warp[lane] : T(0);
      const T wi = warp_incl_scan(w, lane);
      if (lane < kScanThreads / 32) s_warp[lane] = wi - w;  // exclusive warp offsets
      const T agg = __shfl_sync(0xffffffffu, wi, 31);       // the tile's sum
      ScanDesc* d = ring + (t & (kRing - 1));
      T prefix = 0;
      if (t == 0) {
        if (lane == 0) desc_publish<T>(d, t, kFlagPrefix, agg);
      } else {
        if (lane == 0) desc_publish<T>(d, t, kFlagAgg, agg);
        uint32_t fail = 0;
        prefix = look_back<T>(ring, t, lane, ctrl, timeout_ns, &fail);
        if (fail) {
          if (lane == 0) s_fail = 1u;
        } else if (lane == 0) {
          desc_publish<T>(d, t, kFlagPrefix, (T)(prefix + agg));
        }
      }
      if (lane == 0) {
        s_prefix = prefix;
        if (t == ntiles - 1 && total_out != nullptr) stcg(total_out, (T)(prefix + agg));
      }
    }
    __syncthreads();
    if (s_fail != 0u) break;
    // ---- write the exclusive prefixes back (every thread has read its
    // inputs, so the tile is overwritten in place)
    const T off = s_prefix + s_warp[warp] + (incl - run);
#pragma unroll
    for (uint32_t k = 0; k < kPer; ++k) tile[tid * kPer + k] = off + v[k];
    if (full) {
      fence_proxy_async();
      __syncthreads();
      if (tid == 0) bulk_store(A + base, tile, kTileBytes);
    } else {
      __syncthreads();
      for (uint32_t j = tid; j < cnt; j += kScanThreads) stcg(A + base + j, tile[j]);
    }
    __syncthreads();
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
    if (cudaFuncSetAttribute(scan_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, 2 * kTileBytes) !=
            cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, scan_kernel<T>, (int)kScanThreads, 2 * kTileBytes) !=
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
  // at most kRing / 4 - 1 blocks (two tiles in flight each), so that the
  // ring outlasts every look-back; the tags hold 24 bits of the tile index,
  // far more than the tiles in flight
  const uint64_t ntiles = (n + kTileBytes / sizeof(T) - 1) / (kTileBytes / sizeof(T));
  const uint32_t blocks = (uint32_t)std::max<uint64_t>(
      1, std::min<uint64_t>({(uint64_t)per_sm * di.sms, (uint64_t)kRing / 4 - 1, ntiles}));
  if (cudaMemsetAsync(aux, 0, scan_aux_bytes(), s) != cudaSuccess) return PIP_ECUDA;
  ScanCtrl* ctrl = static_cast<ScanCtrl*>(aux);
  ScanDesc* ring = reinterpret_cast<ScanDesc*>(static_cast<char*>(aux) + sizeof(ScanCtrl));
  // every block must be resident (a tile's look-back waits on the tiles of
  // other blocks), which the cooperative launch guarantees
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = dim3(blocks);
  cfg.blockDim = dim3(kScanThreads);
  cfg.dynamicSmemBytes = 2 * kTileBytes;
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
