// pip_shuffle_noalloc: the persistent grid shuffle with its scratch taken
// from a fixed area compiled into this library instead of from the device
// allocator.
//
// Who needs it: callers that cannot allocate device memory when they call
// the library.  For example an application that reserved all of the GPU's
// memory up front for its own pool (an allocation would fail or evict its
// data), a latency-critical path that must not enter the CUDA allocator
// (cudaMallocAsync can block on the pool or fail under memory pressure), or
// code that holds a lock the allocator itself may need.
//
// How it works: a file-scope static device array of kStaticScratchBytes
// (16 MiB) holds the shuffle's reservation tables, loser queues and control
// words.  Its device address is looked up once per device with
// cudaGetSymbolAddress (the host-side name is only a stand-in for it).  With
// CUDA's lazy module loading (the default since CUDA 12.2) the driver
// reserves the 16 MiB only when that first lookup loads this file's module,
// not when the library is loaded; from then on the device keeps the area
// until the process exits.  So the first call on a device -- a call with
// n = 0 does only this set-up -- must come before the caller reserves the
// rest of the GPU's memory for itself, and before any stream capture.  If
// the driver cannot reserve the area then, the call returns PIP_ENOMEM.
// Each call clears the part of the area its plan uses before the kernel
// starts (the queued memset), and the area keeps the last call's contents
// afterwards.  All calls on a device share the one area: two calls whose
// work overlaps on the GPU (different streams, no ordering between them)
// race on it and give wrong results, so order them on one stream.
//
// Requests whose plan needs more scratch than the area holds are refused
// with PIP_ETOOLARGE before anything is queued; pip_shuffle handles those.
// A pointer the device cannot use as device memory (host memory that was
// not registered, or a failed lookup) is refused with PIP_EINVAL.  The call
// allocates nothing: no cudaMalloc, cudaMallocAsync, cudaFree or allocating
// library routine on any path.
#include <cstdint>
#include <mutex>

#include "internal.h"

#define PIP_STATIC_SCRATCH_BYTES (16ull << 20)

// The fixed scratch area (one per device that loads the library).
static __device__ __align__(256) unsigned char g_pip_static_scratch[PIP_STATIC_SCRATCH_BYTES];

namespace pip {
namespace {

constexpr uint64_t kStaticScratchBytes = PIP_STATIC_SCRATCH_BYTES;

std::mutex g_mu;
void* g_scratch_ptr[64] = {};

// Device address of the area on the current device, looked up on first use.
pip_status static_scratch(void** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
    cudaGetLastError();
    return PIP_ECUDA;
  }
  std::lock_guard<std::mutex> lk(g_mu);
  if (g_scratch_ptr[dev] == nullptr) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_pip_static_scratch);
    if (e != cudaSuccess || p == nullptr) {
      cudaGetLastError();
      // the module holding the area could not be loaded for lack of memory
      return e == cudaErrorMemoryAllocation ? PIP_ENOMEM : PIP_ECUDA;
    }
    g_scratch_ptr[dev] = p;
  }
  *out = g_scratch_ptr[dev];
  return PIP_OK;
}

// Device memory (or managed memory) that kernels of the current device can
// address; host memory is refused, registered or not, since the kernel would
// scatter random accesses over the host link.
pip_status check_device_pointer(const void* p) {
  cudaPointerAttributes at{};
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return PIP_EINVAL;
  }
  if (at.type != cudaMemoryTypeDevice && at.type != cudaMemoryTypeManaged) return PIP_EINVAL;
  return PIP_OK;
}

}  // namespace
}  // namespace pip

extern "C" pip_status pip_shuffle_noalloc(void* A_dev, uint64_t n, pip_dtype dtype, uint64_t seed, double eps,
                                          void* stream) {
  using namespace pip;
  const uint32_t eb = elem_bytes_of(dtype);
  if (eb == 0 || !(eps > 0.0 && eps < 1.0) || n >= (1ull << 32)) return PIP_EINVAL;
  void* area = nullptr;
  if (n == 0) return static_scratch(&area);  // set-up only: reserve and look up the area
  if (n == 1) return PIP_OK;
  if (A_dev == nullptr || reinterpret_cast<uintptr_t>(A_dev) % eb != 0) return PIP_EINVAL;
  const pip_status sp = check_device_pointer(A_dev);
  if (sp != PIP_OK) return sp;
  pip_options opt{};
  opt.flags = PIP_FLAG_FORCE_GRID;  // the grid driver is the one whose scratch lives in device memory
  Plan plan;
  const pip_status st = make_plan(n, dtype, eps, &opt, &plan);
  if (st != PIP_OK) return st;
  if (plan.aux_bytes > kStaticScratchBytes) return PIP_ETOOLARGE;
  const pip_status s2 = static_scratch(&area);
  if (s2 != PIP_OK) return s2;
  return launch_grid_driver(plan, A_dev, nullptr, seed, area, nullptr, static_cast<cudaStream_t>(stream));
}
