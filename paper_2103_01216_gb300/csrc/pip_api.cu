// C-ABI entry points (include/pip.h): argument checks, planning, scratch
// allocation and launch.  Every computational step runs in the kernels of
// grid_driver.cu; this file only marshals.
#include <cstdint>
#include <cstring>

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
  st = launch_grid_driver(plan, A_dev, H_dev, seed, aux, stats_dev, s);
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
    default: return "unknown status";
  }
}

const char* pip_version(void) { return "pip-gb300 0.1.0 (sm_103a)"; }

}  // extern "C"
