// Block-resident round driver: one thread block runs every round of one
// array's shuffle with its reservation tables in shared memory, so a round
// costs two bar.syncs instead of a grid barrier.  A persistent grid of such
// blocks pulls arrays from a job list (largest first), which is the batched
// path: thousands of independent arrays in one launch.
//
// The round loop itself (cta_rounds.cuh) follows the grid driver's structure
// (Algorithm 1 under the Decomposable Property, Section 4.1; RP-OneRes rule
// and RP-Final window, Appendix A.2).
#include <algorithm>
#include <cstdint>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <vector>

#include "cta_rounds.cuh"
#include "device.cuh"
#include "internal.h"

namespace pip {

namespace {

template <typename Elem>
__global__ void __launch_bounds__(1024) cta_batch_kernel(const BatchHeader* hdr, const BatchJob* jobs,
                                                        pip_job_stats* stats) {
  extern __shared__ uint32_t smem[];
  __shared__ uint32_t s_job;
  BatchHeader* h = const_cast<BatchHeader*>(hdr);
  const uint64_t t_start = globaltimer_ns();
  // explicit targets are validated before this launch; stop on a reported error
  if (block_status(&h->status) != 0u) return;
  for (;;) {
    if (threadIdx.x == 0) s_job = atomicAdd(&h->next, 1u);
    __syncthreads();
    const uint32_t j = s_job;
    __syncthreads();
    if (j >= hdr->count) break;
    const BatchJob job = jobs[j];
    const uint32_t st = run_job<Elem>(job, smem, hdr->fmax, hdr->sigma, hdr->deadline_ns, t_start,
                                      stats != nullptr ? stats + job.slot : nullptr, nullptr, 0u,
                                      (hdr->flags & PIP_FLAG_PREFETCH) != 0u);
    if (st != 0u && threadIdx.x == 0) {
      set_status(&h->status, st);
      atomicCAS(hdr->latch, 0u, st);
    }
  }
}

__global__ void validate_batch_kernel(BatchHeader* hdr, const BatchJob* jobs) {
  const BatchJob job = jobs[blockIdx.y];
  if (job.H == nullptr) return;
  bool bad = false;
  for (uint32_t i = 1u + blockIdx.x * blockDim.x + threadIdx.x; i < job.n; i += gridDim.x * blockDim.x)
    bad |= (job.H[i] > i);
  if (__syncthreads_or(bad) && threadIdx.x == 0) {
    set_status(&hdr->status, PIP_EINVAL);
    atomicCAS(hdr->latch, 0u, (uint32_t)PIP_EINVAL);
  }
}

// One array on one block (the planner's choice for small prefixes).
template <typename Elem>
__global__ void __launch_bounds__(1024) cta_single_kernel(const BatchJob job, uint32_t sigma, uint64_t deadline_ns,
                                                         Ctrl* ctrl, pip_stats* stats, uint32_t* latch,
                                                         uint32_t flags) {
  extern __shared__ uint32_t smem[];
  __shared__ pip_job_stats s_st;
  if (block_status(&ctrl->status) != 0u) {  // invalid explicit targets
    if (threadIdx.x == 0) {
      atomicCAS(latch, 0u, ld_relaxed_u32(&ctrl->status));
      if (stats != nullptr) stats->status = ld_relaxed_u32(&ctrl->status);
    }
    return;
  }
  const uint32_t st =
      run_job<Elem>(job, smem, job.F, sigma, deadline_ns, globaltimer_ns(), &s_st, nullptr, 0u,
                    (flags & PIP_FLAG_PREFETCH) != 0u, 0, (flags & PIP_FLAG_TWO_RES) != 0u);
  if (threadIdx.x == 0) {
    if (st != 0u) {
      set_status(&ctrl->status, st);
      atomicCAS(latch, 0u, st);
    }
    if (stats != nullptr) {
      stats->status = st;
      stats->rounds = s_st.rounds;
      stats->attempts = s_st.attempts;
      stats->losers = s_st.losers;
      stats->max_active = s_st.max_active;
      stats->grid_blocks = 1;
    }
  }
}

__global__ void validate_single_kernel(const uint32_t* __restrict__ H, uint32_t n, Ctrl* ctrl) {
  bool bad = false;
  for (uint32_t i = 1u + blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    bad |= (H[i] > i);
  if (__syncthreads_or(bad) && threadIdx.x == 0) set_status(&ctrl->status, PIP_EINVAL);
}

template <typename Elem>
const void* cta_single_ptr() {
  return reinterpret_cast<const void*>(&cta_single_kernel<Elem>);
}

const void* select_cta_single(uint32_t elem_bytes) {
  switch (elem_bytes) {
    case 4: return cta_single_ptr<uint32_t>();
    case 8: return cta_single_ptr<unsigned long long>();
    case 16: return cta_single_ptr<uint4>();
    default: return nullptr;
  }
}

template <typename Elem>
const void* cta_kernel_ptr() {
  return reinterpret_cast<const void*>(&cta_batch_kernel<Elem>);
}

const void* select_cta_kernel(uint32_t elem_bytes) {
  switch (elem_bytes) {
    case 4: return cta_kernel_ptr<uint32_t>();
    case 8: return cta_kernel_ptr<unsigned long long>();
    case 16: return cta_kernel_ptr<uint4>();
    default: return nullptr;
  }
}

// Per-device cache of the kernel attributes set and the occupancy found, so
// that a launch issues no attribute or occupancy call once warmed up (which
// keeps it legal inside stream capture).
struct LaunchCacheKey {
  int dev;
  const void* k;
  uint32_t threads;
  uint64_t smem;
  bool operator<(const LaunchCacheKey& o) const {
    if (dev != o.dev) return dev < o.dev;
    if (k != o.k) return k < o.k;
    if (threads != o.threads) return threads < o.threads;
    return smem < o.smem;
  }
};
std::mutex g_cache_mu;
std::map<LaunchCacheKey, int> g_occ;

// Sets the dynamic shared-memory attribute and returns the resident blocks
// per SM (0 on failure).
int prepare_kernel(const void* k, uint32_t threads, uint64_t smem) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  std::lock_guard<std::mutex> lk(g_cache_mu);
  const LaunchCacheKey key{dev, k, threads, smem};
  auto it = g_occ.find(key);
  if (it != g_occ.end()) return it->second;
  // the attribute is per kernel, so it is raised once to the device's opt-in
  // maximum (never lowered): every cached launch size stays admissible
  int optin = 0;
  if (cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  cudaFuncAttributes fa{};
  if (cudaFuncGetAttributes(&fa, k) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  const int dyn_max = optin - (int)fa.sharedSizeBytes;
  if ((uint64_t)dyn_max < smem ||
      cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, dyn_max) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, (int)threads, (size_t)smem) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  g_occ[key] = per_sm;
  return per_sm;
}

}  // namespace

uint64_t cta_smem_bytes(uint32_t fmax, uint32_t sigma) {
  // one slot table, one window bitmap, two loser queues (cta_rounds.cuh)
  return 4ull * ((uint64_t)cta_table_words(fmax, sigma) + cta_window_words(fmax) + 2ull * cta_kmax(fmax));
}

uint32_t cta_max_fmax(uint32_t sigma) {
  int dev = 0, optin = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess) {
    cudaGetLastError();
    optin = 227 * 1024;
  }
  const uint64_t budget = (uint64_t)optin - 1024;  // static shared variables
  uint32_t f = 1;
  while (cta_smem_bytes(f * 2, sigma) <= budget) f *= 2;
  // then refine linearly
  uint32_t lo = f, hi = f * 2;
  while (hi - lo > 1) {
    const uint32_t mid = (lo + hi) / 2;
    if (cta_smem_bytes(mid, sigma) <= budget) lo = mid;
    else hi = mid;
  }
  return lo;
}

pip_status launch_cta_driver(const BatchLaunch& bl, cudaStream_t stream) {
  const void* k = select_cta_kernel(bl.elem_bytes);
  if (k == nullptr) return PIP_EINVAL;
  const uint64_t smem = cta_smem_bytes(bl.fmax, bl.sigma);
  const int per_sm = prepare_kernel(k, bl.threads, smem);
  if (per_sm < 1) return PIP_EINVAL;
  DeviceInfo di;
  if (device_info(&di) != PIP_OK) return PIP_ECUDA;
  uint32_t blocks = std::min<uint64_t>((uint64_t)per_sm * di.sms, bl.count);
  if (bl.max_blocks) blocks = std::min(blocks, bl.max_blocks);
  blocks = std::max(1u, blocks);
  if (bl.any_explicit) {
    validate_batch_kernel<<<dim3(64, bl.count), 256, 0, stream>>>(bl.hdr, bl.jobs);
    if (cudaGetLastError() != cudaSuccess) return PIP_ECUDA;
  }
  void* args[] = {(void*)&bl.hdr, (void*)&bl.jobs, (void*)&bl.stats};
  if (cudaLaunchKernel(k, dim3(blocks), dim3(bl.threads), args, (size_t)smem, stream) != cudaSuccess) {
    cudaGetLastError();
    return PIP_ECUDA;
  }
  return PIP_OK;
}

pip_status launch_cta_single(const Plan& plan, void* A, const uint32_t* H, uint64_t seed, void* aux,
                             pip_stats* stats, cudaStream_t stream) {
  const void* k = select_cta_single(plan.elem_bytes);
  if (k == nullptr) return PIP_EINVAL;
  const uint64_t smem = plan.smem_bytes;
  if (prepare_kernel(k, plan.threads, smem) < 1) return PIP_EINVAL;
  uint32_t* latch = error_latch_ptr();
  if (latch == nullptr) return PIP_ECUDA;
  Ctrl* ctrl = static_cast<Ctrl*>(aux);
  if (cudaMemsetAsync(aux, 0, sizeof(Ctrl), stream) != cudaSuccess) return PIP_ECUDA;
  if (H != nullptr) {
    const uint32_t vb = (uint32_t)std::min<uint64_t>(1024, (plan.n + 255) / 256);
    validate_single_kernel<<<vb, 256, 0, stream>>>(H, plan.n, ctrl);
    if (cudaGetLastError() != cudaSuccess) return PIP_ECUDA;
  }
  BatchJob job{};
  job.A = A;
  job.H = H;
  job.seed = seed;
  job.n = plan.n;
  job.F = plan.F;
  uint32_t sigma = plan.sigma;
  uint64_t deadline = plan.deadline_ns;
  uint32_t flags = plan.flags & (PIP_FLAG_PREFETCH | PIP_FLAG_TWO_RES);
  void* args[] = {&job, &sigma, &deadline, &ctrl, &stats, &latch, &flags};
  if (cudaLaunchKernel(k, dim3(1), dim3(plan.threads), args, (size_t)smem, stream) != cudaSuccess) {
    cudaGetLastError();
    return PIP_ECUDA;
  }
  return PIP_OK;
}

}  // namespace pip
