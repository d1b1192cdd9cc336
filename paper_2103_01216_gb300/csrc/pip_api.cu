// C-ABI entry points (include/pip.h): argument checks, planning, scratch
// allocation and launch.  Every computational step runs in the kernels of
// grid_driver.cu; this file only marshals.
#include <algorithm>
#include <cstdint>
#include <cstring>
#include <cstdlib>
#include <vector>

#include "internal.h"

using namespace pip;

namespace {

pip_status check_shape(uint64_t n, pip_dtype dtype, double eps) {
  if (elem_bytes_of(dtype) == 0) return PIP_EINVAL;
  if (!(eps > 0.0 && eps < 1.0)) return PIP_EINVAL;
  if (n >= (1ull << 32)) return PIP_EINVAL;
  return PIP_OK;
}

pip_status check_args(const void* A, uint64_t n, pip_dtype dtype, double eps) {
  if (check_shape(n, dtype, eps) != PIP_OK) return PIP_EINVAL;
  const uint32_t eb = elem_bytes_of(dtype);
  if (n > 1 && A == nullptr) return PIP_EINVAL;
  if (A != nullptr && (reinterpret_cast<uintptr_t>(A) % eb) != 0) return PIP_EINVAL;
  return PIP_OK;
}

}  // namespace

extern "C" {

pip_status pip_plan(uint64_t n, pip_dtype dtype, double eps, const pip_options* opt, pip_plan_info* out) {
  if (out == nullptr) return PIP_EINVAL;
  if (check_shape(n, dtype, eps) != PIP_OK) return PIP_EINVAL;
  std::memset(out, 0, sizeof(*out));
  out->n = n;
  out->elem_bytes = elem_bytes_of(dtype);
  out->eps = eps;
  if (n <= 1) return PIP_OK;
  Plan p;
  const pip_status st = make_plan(n, dtype, eps, opt, &p);
  if (st != PIP_OK) return st;
  out->fresh_per_round = p.F;
  out->max_active = p.kmax;
  out->slots = p.nslots;
  out->grid_blocks = p.blocks;
  out->block_threads = p.threads;
  out->aux_bytes = p.aux_bytes;
  out->aux_bound_bytes = p.aux_bound;
  out->min_rounds = (n - 1 + p.F - 1) / p.F;
  out->driver = p.driver;
  out->flags = p.flags;
  out->smem_bytes = p.smem_bytes;
  return PIP_OK;
}

uint64_t pip_aux_bytes(uint64_t n, pip_dtype dtype, double eps) {
  pip_plan_info info;
  if (pip_plan(n, dtype, eps, nullptr, &info) != PIP_OK) return 0;
  return info.aux_bytes;
}

pip_status pip_shuffle_ex(void* A_dev, uint64_t n, pip_dtype dtype, uint64_t seed, const uint32_t* H_dev,
                          double eps, const pip_options* opt, void* aux_dev, uint64_t aux_bytes,
                          pip_stats* stats_dev, void* stream) {
  pip_status st = check_args(A_dev, n, dtype, eps);
  if (st != PIP_OK) return st;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (n <= 1) {
    if (stats_dev != nullptr) {
      pip_stats zero{};
      if (cudaMemcpyAsync(stats_dev, &zero, sizeof(zero), cudaMemcpyHostToDevice, s) != cudaSuccess) return PIP_ECUDA;
      if (cudaStreamSynchronize(s) != cudaSuccess) return PIP_ECUDA;
    }
    return PIP_OK;
  }
  Plan plan;
  st = make_plan(n, dtype, eps, opt, &plan);
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
  if (plan.driver == kDriverCta) st = launch_cta_single(plan, A_dev, H_dev, seed, aux, stats_dev, s);
  else if (plan.driver == kDriverCluster) st = launch_cluster_driver(plan, A_dev, H_dev, seed, aux, stats_dev, s);
  else if ((plan.flags & PIP_FLAG_TEST_GATED) && H_dev == nullptr)
    st = launch_grid_lane(plan, A_dev, seed, aux, stats_dev, plan.timeout_ns, s);
  else st = launch_grid_driver(plan, A_dev, H_dev, seed, aux, stats_dev, s);
  if (owned && cudaFreeAsync(aux, s) != cudaSuccess && st == PIP_OK) st = PIP_ECUDA;
  return st;
}

pip_status pip_shuffle(void* A_dev, uint64_t n, pip_dtype dtype, uint64_t seed, double eps, void* stream) {
  return pip_shuffle_ex(A_dev, n, dtype, seed, nullptr, eps, nullptr, nullptr, 0, nullptr, stream);
}

pip_status pip_shuffle_explicit_h(void* A_dev, uint64_t n, pip_dtype dtype, const uint32_t* H_dev, double eps,
                                  void* stream) {
  if (n > 1 && H_dev == nullptr) return PIP_EINVAL;
  return pip_shuffle_ex(A_dev, n, dtype, 0, H_dev, eps, nullptr, nullptr, 0, nullptr, stream);
}

pip_status pip_batch_plan_make(const pip_batch_item* items, uint32_t count, pip_dtype dtype, double eps,
                               const pip_options* opt, pip_batch_plan* out) {
  if (out == nullptr || (count > 0 && items == nullptr)) return PIP_EINVAL;
  if (check_shape(0, dtype, eps) != PIP_OK) return PIP_EINVAL;
  pip_options o{};
  if (opt != nullptr) o = *opt;
  // arrays of a batch share the device: C = 1 keeps each block's shared
  // memory small enough for several resident arrays per SM
  if (!(o.prefix_c > 0.0) && o.fresh_per_round == 0) o.prefix_c = 1.0;
  opt = &o;
  const uint32_t sigma = o.slot_factor ? o.slot_factor : 4u;
  if (sigma < 2 || sigma > 16) return PIP_EINVAL;
  const uint32_t threads = o.block_threads ? o.block_threads : 1024u;  // measured best for the 8192-array mix
  if (threads < 128 || threads > 1024 || threads % 32 != 0) return PIP_EINVAL;
  const uint32_t eb = elem_bytes_of(dtype);
  const uint32_t fcap = cta_max_fmax(sigma);
  std::memset(out, 0, sizeof(*out));
  out->count = count;
  out->elem_bytes = eb;
  out->slot_factor = sigma;
  out->block_threads = threads;
  out->max_blocks = o.grid_blocks;
  out->eps = eps;
  uint32_t fmax = 1;
  for (uint32_t j = 0; j < count; ++j) {
    const pip_batch_item& it = items[j];
    if (it.n >= (1ull << 32)) return PIP_EINVAL;
    if (it.n > 1 && (it.A_dev == nullptr || reinterpret_cast<uintptr_t>(it.A_dev) % eb != 0)) return PIP_EINVAL;
    if (it.H_dev != nullptr) out->any_explicit = 1;
    out->total_elems += it.n;
    if (it.n >= 2) fmax = std::max(fmax, cta_fresh(it.n, eps, opt, sigma, fcap));
  }
  out->fmax = fmax;
  out->smem_bytes = cta_smem_bytes(fmax, sigma);
  out->jobs_bytes = sizeof(BatchHeader) + (uint64_t)count * sizeof(BatchJob);
  return PIP_OK;
}

pip_status pip_batch_prepare(const pip_batch_item* items, const pip_batch_plan* plan, const pip_options* opt,
                             void* jobs_dev) {
  if (plan == nullptr || jobs_dev == nullptr || (plan->count > 0 && items == nullptr)) return PIP_EINVAL;
  if (reinterpret_cast<uintptr_t>(jobs_dev) % 256 != 0) return PIP_EINVAL;
  const uint32_t fcap = cta_max_fmax(plan->slot_factor);
  pip_options o{};
  if (opt != nullptr) o = *opt;
  if (!(o.prefix_c > 0.0) && o.fresh_per_round == 0) o.prefix_c = 1.0;  // as in pip_batch_plan_make
  opt = &o;
  std::vector<char> host(plan->jobs_bytes, 0);
  BatchHeader* hdr = reinterpret_cast<BatchHeader*>(host.data());
  BatchJob* jobs = reinterpret_cast<BatchJob*>(host.data() + sizeof(BatchHeader));
  std::vector<uint32_t> order(plan->count);
  for (uint32_t j = 0; j < plan->count; ++j) order[j] = j;
  // largest arrays first: the longest jobs start early (LPT order)
  std::stable_sort(order.begin(), order.end(), [&](uint32_t a, uint32_t b) { return items[a].n > items[b].n; });
  uint64_t deadline = 60000000000ull;
  for (uint32_t k = 0; k < plan->count; ++k) {
    const pip_batch_item& it = items[order[k]];
    BatchJob& jb = jobs[k];
    jb.A = it.A_dev;
    jb.H = it.H_dev;
    jb.seed = it.seed;
    jb.n = (uint32_t)it.n;
    jb.F = it.n >= 2 ? std::min(plan->fmax, cta_fresh(it.n, plan->eps, opt, plan->slot_factor, fcap)) : 1u;
    jb.slot = order[k];
    deadline += 5000ull * (it.n / jb.F + 1) + 20ull * it.n;
  }
  if (const char* e = std::getenv("PIP_DEADLINE_MS")) {
    const long long ms = std::atoll(e);
    if (ms > 0) deadline = (uint64_t)ms * 1000000ull;
  }
  hdr->count = plan->count;
  hdr->fmax = plan->fmax;
  hdr->sigma = plan->slot_factor;
  hdr->flags = o.flags & PIP_FLAG_PREFETCH;
  hdr->deadline_ns = deadline;
  hdr->latch = error_latch_ptr();
  if (hdr->latch == nullptr) return PIP_ECUDA;
  if (cudaMemcpy(jobs_dev, host.data(), host.size(), cudaMemcpyHostToDevice) != cudaSuccess) {
    cudaGetLastError();
    return PIP_ECUDA;
  }
  return PIP_OK;
}

pip_status pip_batch_run(const pip_batch_plan* plan, void* jobs_dev, pip_job_stats* stats_dev, void* stream) {
  if (plan == nullptr || jobs_dev == nullptr) return PIP_EINVAL;
  if (plan->count == 0) return PIP_OK;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (cudaMemsetAsync(jobs_dev, 0, 8, s) != cudaSuccess) return PIP_ECUDA;  // next, status
  BatchLaunch bl{};
  bl.hdr = static_cast<BatchHeader*>(jobs_dev);
  bl.jobs = reinterpret_cast<BatchJob*>(static_cast<char*>(jobs_dev) + sizeof(BatchHeader));
  bl.stats = stats_dev;
  bl.count = plan->count;
  bl.elem_bytes = plan->elem_bytes;
  bl.fmax = plan->fmax;
  bl.sigma = plan->slot_factor;
  bl.threads = plan->block_threads;
  bl.max_blocks = plan->max_blocks;
  bl.any_explicit = plan->any_explicit != 0;
  return launch_cta_driver(bl, s);
}

pip_status pip_shuffle_batch(void* const* A_devs, const uint64_t* ns, const uint64_t* seeds, uint32_t count,
                             pip_dtype dtype, double eps, void* stream) {
  if (count == 0) return PIP_OK;
  if (A_devs == nullptr || ns == nullptr || seeds == nullptr) return PIP_EINVAL;
  std::vector<pip_batch_item> items(count);
  for (uint32_t j = 0; j < count; ++j) items[j] = pip_batch_item{A_devs[j], nullptr, ns[j], seeds[j]};
  pip_batch_plan plan;
  pip_status st = pip_batch_plan_make(items.data(), count, dtype, eps, nullptr, &plan);
  if (st != PIP_OK) return st;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  void* jobs = nullptr;
  if (cudaMallocAsync(&jobs, plan.jobs_bytes, s) != cudaSuccess) {
    cudaGetLastError();
    return PIP_ENOMEM;
  }
  // the job list is written synchronously; order it after the allocation
  if (cudaStreamSynchronize(s) != cudaSuccess) {
    cudaGetLastError();
    return PIP_ECUDA;
  }
  st = pip_batch_prepare(items.data(), &plan, nullptr, jobs);
  if (st == PIP_OK) st = pip_batch_run(&plan, jobs, nullptr, stream);
  if (cudaFreeAsync(jobs, s) != cudaSuccess && st == PIP_OK) st = PIP_ECUDA;
  return st;
}

pip_status pip_check(void* stream) {
  if (cudaStreamSynchronize(static_cast<cudaStream_t>(stream)) != cudaSuccess) {
    cudaGetLastError();
    return PIP_ECUDA;
  }
  uint32_t v = 0;
  if (take_error_latch(&v) != PIP_OK) return PIP_ECUDA;
  return static_cast<pip_status>(v);
}

const char* pip_status_string(pip_status s) {
  switch (s) {
    case PIP_OK: return "ok";
    case PIP_EINVAL: return "invalid argument";
    case PIP_ENOMEM: return "out of memory";
    case PIP_ECUDA: return "CUDA runtime error";
    case PIP_ETIMEOUT: return "device-side wait timed out";
    case PIP_EAGAIN: return "not finished yet";
    case PIP_EBUSY: return "queued behind the memory budget";
    case PIP_EINTERNAL: return "internal consistency check failed";
    case PIP_ETOOLARGE: return "needs more scratch than the fixed no-allocation area holds";
    default: return "unknown status";
  }
}

const char* pip_version(void) { return "pip-gb300 0.1.0 (sm_103a)"; }

}  // extern "C"
