// Calibration probe (benchmark only; it destroys its input): the bare memory
// traffic of a shuffle's swaps, without any conflict resolution.  Every step
// i in [1, n) exchanges A[i] and A[h] with h = H[i] from the same target
// generator, all steps at once, so the result is NOT a valid shuffle (steps
// that share a location race).  It measures how fast this GPU moves the data
// of n-1 random swaps: coalesced accesses on the i side, and on the h side
// either one atomic exchange at L2 or a load and a store, the two commit
// modes of the round drivers.
// The benchmark reports the round drivers' time against this floor.  The
// paper has no counterpart: it is a measurement tool, not part of the method.
#include <algorithm>
#include <cstdint>

#include "device.cuh"
#include "internal.h"

namespace pip {
namespace {

template <typename Elem, bool kExchange>
__global__ void __launch_bounds__(256) swap_floor_kernel(Elem* A, uint32_t n, uint64_t seed) {
  const uint64_t pol = policy_evict_first();
  for (uint32_t i = 1u + blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const uint32_t h = hashed_target(seed, i);
    const Elem x = ldcg(A + i);
    if constexpr (kExchange) {
      st_hint(A + i, exch_hint(A + h, x, pol), pol);
    } else {
      const Elem y = ldcg(A + h);
      st_hint(A + i, y, pol);
      st_hint(A + h, x, pol);
    }
  }
}

template <typename Elem>
void launch_floor(void* A, uint32_t n, uint64_t seed, int mode, uint32_t blocks, cudaStream_t s) {
  if (mode == PIP_FLOOR_EXCHANGE) swap_floor_kernel<Elem, true><<<blocks, 256, 0, s>>>(static_cast<Elem*>(A), n, seed);
  else swap_floor_kernel<Elem, false><<<blocks, 256, 0, s>>>(static_cast<Elem*>(A), n, seed);
}

}  // namespace
}  // namespace pip

extern "C" pip_status pip_calibrate_swap_floor(void* A_dev, uint64_t n, pip_dtype dtype, uint64_t seed, int mode,
                                               void* stream) {
  using namespace pip;
  const uint32_t eb = elem_bytes_of(dtype);
  if (eb == 0 || n >= (1ull << 32)) return PIP_EINVAL;
  if (mode != PIP_FLOOR_EXCHANGE && mode != PIP_FLOOR_LOADSTORE) return PIP_EINVAL;
  if (n <= 1) return PIP_OK;
  if (A_dev == nullptr || reinterpret_cast<uintptr_t>(A_dev) % eb != 0) return PIP_EINVAL;
  DeviceInfo di;
  if (device_info(&di) != PIP_OK) return PIP_ECUDA;
  const uint32_t blocks = (uint32_t)std::min<uint64_t>((uint64_t)di.sms * 8, (n + 255) / 256);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  switch (eb) {
    case 4: launch_floor<uint32_t>(A_dev, (uint32_t)n, seed, mode, blocks, s); break;
    case 8: launch_floor<unsigned long long>(A_dev, (uint32_t)n, seed, mode, blocks, s); break;
    default: launch_floor<uint4>(A_dev, (uint32_t)n, seed, mode, blocks, s); break;
  }
  return cudaGetLastError() == cudaSuccess ? PIP_OK : PIP_ECUDA;
}
