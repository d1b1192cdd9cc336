// Shuffles of arrays held in host memory, with the copies overlapped with
// the shuffles: the path a caller whose data lives on the host takes.
//
// A shuffle reads and writes its whole array at random, so one array's
// copies cannot overlap its own shuffle.  Over a sequence of arrays they can
// overlap their neighbours' shuffles: array j is copied in while array j-1 is
// shuffled, and copied out while array j+1 is.  Three streams carry the work
// -- host-to-device copies, shuffles, device-to-host copies -- ordered by
// events, over device buffers used in turn: with two, array j+1's copy in
// would wait for array j-1's copy out (same buffer), serialising the two
// directions (38 + 41 ms for 8 GB each way on GB300, more than a 65 ms
// shuffle); with three they run together (51 ms for both).  A buffer still
// goes round copy in, shuffle and copy out before it takes its next array,
// so with B buffers no array can take less than a B-th of the three stages
// in a row: with three, a box whose copies slow to ~70 ms under a shuffle's
// traffic is held to (61 + 70 + 70) / 3 ms per array, above the shuffle.
// Four buffers are used where there is room for them (always when the
// library allocates them), three at least.  The shuffles stay on one stream,
// so two of the persistent round kernels (each wanting the whole GPU) never
// run at once.
#include <cstdint>

#include "internal.h"

namespace pip {
namespace {

struct StreamSet {
  cudaStream_t h2d = nullptr, comp = nullptr, d2h = nullptr;
  cudaEvent_t ready = nullptr;
  static constexpr int kBufs = 4;   // at most; kMinBufs suffice
  cudaEvent_t in_done[kBufs] = {}, shuf_done[kBufs] = {}, out_done[kBufs] = {};

  pip_status create() {
    const unsigned f = cudaStreamNonBlocking;
    if (cudaStreamCreateWithFlags(&h2d, f) != cudaSuccess || cudaStreamCreateWithFlags(&comp, f) != cudaSuccess ||
        cudaStreamCreateWithFlags(&d2h, f) != cudaSuccess)
      return PIP_ECUDA;
    if (cudaEventCreateWithFlags(&ready, cudaEventDisableTiming) != cudaSuccess) return PIP_ECUDA;
    for (int b = 0; b < kBufs; ++b)
      for (cudaEvent_t* e : {&in_done[b], &shuf_done[b], &out_done[b]})
        if (cudaEventCreateWithFlags(e, cudaEventDisableTiming) != cudaSuccess) return PIP_ECUDA;
    return PIP_OK;
  }
  // Streams and events are released once their queued work is done.
  ~StreamSet() {
    if (ready != nullptr) cudaEventDestroy(ready);
    for (int b = 0; b < kBufs; ++b)
      for (cudaEvent_t e : {in_done[b], shuf_done[b], out_done[b]})
        if (e != nullptr) cudaEventDestroy(e);
    for (cudaStream_t s : {h2d, comp, d2h})
      if (s != nullptr) cudaStreamDestroy(s);
  }
};

}  // namespace
}  // namespace pip

using namespace pip;

extern "C" {

pip_status pip_shuffle_host_stream(const void* const* in_hosts, void* const* out_hosts, const uint64_t* seeds,
                                   uint32_t count, uint64_t n, pip_dtype dtype, double eps, void* dev_buf,
                                   uint64_t dev_bytes, void* stream) {
  if (count == 0) return PIP_OK;
  if (in_hosts == nullptr || out_hosts == nullptr || seeds == nullptr) return PIP_EINVAL;
  if (dtype != PIP_U32 && dtype != PIP_U64 && dtype != PIP_REC128) return PIP_EINVAL;
  if (!(eps > 0.0 && eps < 1.0)) return PIP_EINVAL;
  for (uint32_t j = 0; j < count; ++j)
    if (n > 0 && (in_hosts[j] == nullptr || out_hosts[j] == nullptr)) return PIP_EINVAL;
  const uint64_t eb = dtype == PIP_U32 ? 4u : (dtype == PIP_U64 ? 8u : 16u);
  if (n == 0) return PIP_OK;
  const uint64_t bytes = n * eb;
  const uint64_t slot = (bytes + 255) / 256 * 256;  // each buffer 256-byte aligned
  constexpr uint32_t kMinBufs = 3;
  // buffers: one per array up to four; a caller's area gives as many as it
  // holds, and must hold min(count, 3)
  uint32_t nbuf = count < (uint32_t)StreamSet::kBufs ? count : (uint32_t)StreamSet::kBufs;
  cudaStream_t user = static_cast<cudaStream_t>(stream);

  // the scratch of one shuffle, reused by every shuffle (they are serial)
  const uint64_t aux_bytes = n > 1 ? pip_aux_bytes(n, dtype, eps) : 0;
  if (n > 1 && aux_bytes == 0) return PIP_EINVAL;

  pip_status st = PIP_OK;
  StreamSet ss;
  if ((st = ss.create()) != PIP_OK) {
    cudaGetLastError();
    return st;
  }
  char* buf = static_cast<char*>(dev_buf);
  void* aux = nullptr;
  bool own_buf = false;
  if (buf != nullptr) {
    const uint32_t need = nbuf < kMinBufs ? nbuf : kMinBufs;
    if (dev_bytes < need * slot || reinterpret_cast<uintptr_t>(buf) % 256 != 0) return PIP_EINVAL;
    if (dev_bytes / slot < nbuf) nbuf = (uint32_t)(dev_bytes / slot);
  } else {
    if (cudaMallocAsync(reinterpret_cast<void**>(&buf), nbuf * slot, user) != cudaSuccess) {
      cudaGetLastError();
      // no room for the fourth buffer: three still overlap the copies
      if (nbuf <= kMinBufs || cudaMallocAsync(reinterpret_cast<void**>(&buf), kMinBufs * slot, user) != cudaSuccess) {
        cudaGetLastError();
        return PIP_ENOMEM;
      }
      nbuf = kMinBufs;
    }
    own_buf = true;
  }
  if (aux_bytes > 0 && cudaMallocAsync(&aux, aux_bytes, user) != cudaSuccess) {
    cudaGetLastError();
    if (own_buf) cudaFreeAsync(buf, user);
    return PIP_ENOMEM;
  }
  // whatever the caller queued before this call (and the allocations) comes
  // first
  if (cudaEventRecord(ss.ready, user) != cudaSuccess || cudaStreamWaitEvent(ss.h2d, ss.ready, 0) != cudaSuccess ||
      cudaStreamWaitEvent(ss.comp, ss.ready, 0) != cudaSuccess) {
    st = PIP_ECUDA;
  }
  for (uint32_t j = 0; j < count && st == PIP_OK; ++j) {
    const uint32_t b = j % nbuf;
    void* d = buf + (uint64_t)b * slot;
    // the buffer's previous array has been copied out
    if (j >= nbuf && cudaStreamWaitEvent(ss.h2d, ss.out_done[b], 0) != cudaSuccess) st = PIP_ECUDA;
    if (st == PIP_OK && (cudaMemcpyAsync(d, in_hosts[j], bytes, cudaMemcpyHostToDevice, ss.h2d) != cudaSuccess ||
                         cudaEventRecord(ss.in_done[b], ss.h2d) != cudaSuccess ||
                         cudaStreamWaitEvent(ss.comp, ss.in_done[b], 0) != cudaSuccess))
      st = PIP_ECUDA;
    if (st == PIP_OK)
      st = pip_shuffle_ex(d, n, dtype, seeds[j], nullptr, eps, nullptr, aux, aux_bytes, nullptr, ss.comp);
    if (st == PIP_OK && (cudaEventRecord(ss.shuf_done[b], ss.comp) != cudaSuccess ||
                         cudaStreamWaitEvent(ss.d2h, ss.shuf_done[b], 0) != cudaSuccess ||
                         cudaMemcpyAsync(out_hosts[j], d, bytes, cudaMemcpyDeviceToHost, ss.d2h) != cudaSuccess ||
                         cudaEventRecord(ss.out_done[b], ss.d2h) != cudaSuccess))
      st = PIP_ECUDA;
  }
  // the caller's stream waits for every copy out (the last one is ordered
  // after all others on the copy-out stream, and each after its shuffle),
  // then the buffers are released in its order.  After a failure part of the
  // work may be queued without those events: wait for all of it first.
  const uint32_t last = (count - 1) % nbuf;
  if (st == PIP_OK && cudaStreamWaitEvent(user, ss.out_done[last], 0) != cudaSuccess) st = PIP_ECUDA;
  if (st != PIP_OK) {
    cudaGetLastError();
    cudaStreamSynchronize(ss.h2d);
    cudaStreamSynchronize(ss.comp);
    cudaStreamSynchronize(ss.d2h);
    cudaGetLastError();
  }
  if (aux != nullptr) cudaFreeAsync(aux, user);
  if (own_buf) cudaFreeAsync(buf, user);
  return st;
}

}  // extern "C"
