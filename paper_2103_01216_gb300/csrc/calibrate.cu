// Calibration probe: the bare memory traffic of a shuffle's swaps, without
// any conflict resolution.  Every step i in [1, n) exchanges A[i] and A[h]
// with h = H[i] from the same target generator, all steps at once, so the
// result is NOT a valid shuffle (steps that share a location race).  It
// measures how fast this GPU moves the data of n-1 random swaps: coalesced
// accesses on the i side, one random element read and write on the h side.
// The benchmark reports the round drivers' time against this floor.  The
// paper has no counterpart: it is a measurement tool, not part of the method.
#include <algorithm>
#include <cstdint>

#include "device.cuh"
#include "internal.h"

namespace pip {
namespace {

template <typename Elem>
__global__ void __launch_bounds__(256) swap_floor_kernel(Elem* A, uint32_t n, uint64_t seed) {
  for (uint32_t i = 1u + blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const uint32_t h = hashed_target(seed, i);
    const Elem x = ldcg(A + i);
    const Elem y = ldcg(A + h);
    stcg(A + i, y);
    stcg(A + h, x);
  }
}

}  // namespace
}  // namespace pip

extern "C" pip_status pip_calibrate_swap_floor(void* A_dev, uint64_t n, pip_dtype dtype, uint64_t seed,
                                               void* stream) {
  using namespace pip;
  const uint32_t eb = elem_bytes_of(dtype);
  if (eb == 0 || n >= (1ull << 32)) return PIP_EINVAL;
  if (n <= 1) return PIP_OK;
  if (A_dev == nullptr || reinterpret_cast<uintptr_t>(A_dev) % eb != 0) return PIP_EINVAL;
  DeviceInfo di;
  if (device_info(&di) != PIP_OK) return PIP_ECUDA;
  const uint32_t blocks = (uint32_t)std::min<uint64_t>((uint64_t)di.sms * 8, (n + 255) / 256);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  switch (eb) {
    case 4: swap_floor_kernel<uint32_t><<<blocks, 256, 0, s>>>(static_cast<uint32_t*>(A_dev), (uint32_t)n, seed); break;
    case 8:
      swap_floor_kernel<unsigned long long><<<blocks, 256, 0, s>>>(static_cast<unsigned long long*>(A_dev),
                                                                    (uint32_t)n, seed);
      break;
    default: swap_floor_kernel<uint4><<<blocks, 256, 0, s>>>(static_cast<uint4*>(A_dev), (uint32_t)n, seed); break;
  }
  return cudaGetLastError() == cudaSuccess ? PIP_OK : PIP_ECUDA;
}
