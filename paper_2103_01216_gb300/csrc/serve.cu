// Serving: a request loop over shuffle requests of uneven sizes with
// memory-budgeted admission and continuous batching.
//
// A background thread owns one CUDA stream and repeats a "tick":
//   1. admit waiting requests in arrival order while the device budget
//      allows, charging each its array (n * element bytes) plus its
//      O(n^(1-eps)) scratch (the relaxed PIP bound of Section 3.2, not a
//      second copy of the array); admitted requests get their array (when
//      the server allocates it) and their carried-loser queue;
//   2. launch one tick kernel in which persistent blocks pull resident
//      requests and advance each by at most `rounds_per_tick` rounds of the
//      block-resident round loop (Section 4.1 under the Decomposable
//      Property), saving its round state in device memory;
//   3. read back the round states, stamp and retire finished requests, free
//      their scratch, and wake the clients waiting on them.
// Requests that arrive while others are on the GPU join at the next tick,
// and the work of all resident requests overlaps on the device.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "cta_rounds.cuh"
#include "device.cuh"
#include "internal.h"

namespace pip {
namespace {

struct ServeSlot {
  BatchJob job;
  uint32_t elem_bytes;
  uint32_t pad;
  ResumeState rs;
};

int64_t now_ns() {
  return std::chrono::duration_cast<std::chrono::nanoseconds>(std::chrono::steady_clock::now().time_since_epoch())
      .count();
}

__global__ void __launch_bounds__(1024) serve_tick_kernel(ServeSlot* slots, const uint32_t* work, uint32_t count,
                                                          uint32_t* next, uint32_t fmax, uint32_t sigma,
                                                          uint32_t budget, uint64_t deadline_ns, uint64_t slice_ns) {
  extern __shared__ uint32_t smem[];
  __shared__ uint32_t s_w;
  const uint64_t t0 = globaltimer_ns();
  for (;;) {
    if (threadIdx.x == 0) s_w = atomicAdd(next, 1u);
    __syncthreads();
    const uint32_t w = s_w;
    __syncthreads();
    if (w >= count) break;
    ServeSlot* sl = slots + work[w];
    const BatchJob job = sl->job;
    uint32_t st;
    if (sl->elem_bytes == 4)
      st = run_job<uint32_t>(job, smem, fmax, sigma, deadline_ns, t0, nullptr, &sl->rs, budget, false, slice_ns);
    else if (sl->elem_bytes == 8)
      st = run_job<unsigned long long>(job, smem, fmax, sigma, deadline_ns, t0, nullptr, &sl->rs, budget, false,
                                       slice_ns);
    else st = run_job<uint4>(job, smem, fmax, sigma, deadline_ns, t0, nullptr, &sl->rs, budget, false, slice_ns);
    (void)st;  // the status is in the request's round state
  }
}

// Initial content of a server-allocated array: A[i] = i, or the records
// {key = i, payload = SplitMix64 mix of i} for 16-byte elements.
__global__ void init_array_kernel(void* A, uint32_t n, uint32_t elem_bytes) {
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    if (elem_bytes == 4) static_cast<uint32_t*>(A)[i] = i;
    else if (elem_bytes == 8) static_cast<unsigned long long*>(A)[i] = i;
    else static_cast<ulonglong2*>(A)[i] = make_ulonglong2(i, splitmix64(i));
  }
}

struct Req {
  uint64_t ticket = 0;
  uint64_t n = 0;
  uint32_t elem_bytes = 8;
  uint64_t seed = 0;
  double eps = 0.5;
  void* A = nullptr;
  bool owned = false;
  uint32_t F = 1;
  uint32_t* Q = nullptr;
  uint64_t array_bytes = 0;
  uint64_t aux_bytes = 0;
  int slot = -1;
  bool done = false;
  bool released = false;
  uint32_t status = 0;
  uint32_t rounds = 0;
  uint64_t attempts = 0, losers = 0;
  uint32_t ticks = 0;
  int64_t submit_ns = 0, admit_ns = 0, done_ns = 0;
};

}  // namespace
}  // namespace pip

struct pip_server {
  int device = 0;
  uint64_t budget = 0;
  uint64_t used = 0;
  uint64_t peak_used = 0;
  pip_serve_options opt{};
  uint32_t sigma = 4, fmax = 1024, threads = 512, max_resident = 1024, rounds_per_tick = 128;
  uint64_t tick_ns = 1000000;
  uint64_t smem = 0;
  uint32_t blocks = 0;
  cudaStream_t stream = nullptr;
  pip::ServeSlot* d_slots = nullptr;
  pip::ServeSlot* h_slots = nullptr;
  uint32_t* d_work = nullptr;
  uint32_t* h_work = nullptr;
  uint32_t* d_next = nullptr;
  std::vector<int> free_slots;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<pip::Req*> waiting;
  std::vector<pip::Req*> resident;
  std::unordered_map<uint64_t, pip::Req*> reqs;
  std::vector<void*> to_free;  // released server-owned arrays, freed by the loop thread
  std::deque<uint64_t> finished;  // tickets in completion order, not yet handed out by next_done
  uint64_t next_ticket = 1;
  uint64_t submitted = 0, admitted = 0, completed = 0, ticks = 0;
  bool stop = false;
  pip_status loop_error = PIP_OK;
  std::thread th;
  void loop();
};

namespace pip {
namespace {

uint64_t req_aux_bytes(uint32_t F) { return (uint64_t)cta_kmax(F) * 4 + sizeof(ServeSlot); }

}  // namespace
}  // namespace pip

void pip_server::loop() {
  using namespace pip;
  cudaSetDevice(device);
  std::vector<Req*> admit_now;
  for (;;) {
    {
      std::unique_lock<std::mutex> lk(mu);
      cv_work.wait(lk, [&] { return stop || !waiting.empty() || !resident.empty() || !to_free.empty(); });
      if (stop && resident.empty()) break;
      for (void* p : to_free) cudaFreeAsync(p, stream);
      to_free.clear();
      // admission in arrival order (a request that does not fit blocks the ones behind it)
      admit_now.clear();
      while (!stop && !waiting.empty() && !free_slots.empty()) {
        Req* r = waiting.front();
        const uint64_t charge = r->array_bytes + r->aux_bytes;
        if (used + charge > budget) break;
        waiting.pop_front();
        used += charge;
        peak_used = std::max(peak_used, used);
        r->slot = free_slots.back();
        free_slots.pop_back();
        r->admit_ns = now_ns();
        admit_now.push_back(r);
        resident.push_back(r);
        ++admitted;
      }
    }
    // set up the newly admitted requests (allocations and copies are stream-ordered)
    for (Req* r : admit_now) {
      bool ok = true;
      if (r->A == nullptr && r->n > 0) {
        r->owned = true;
        if (cudaMallocAsync(&r->A, r->array_bytes, stream) != cudaSuccess) {
          cudaGetLastError();
          r->A = nullptr;
          ok = false;
        } else {
          init_array_kernel<<<std::min<uint64_t>(4096, (r->n + 255) / 256 + 1), 256, 0, stream>>>(
              r->A, (uint32_t)r->n, r->elem_bytes);
        }
      }
      if (ok && r->n >= 2) {
        if (cudaMallocAsync(reinterpret_cast<void**>(&r->Q), (uint64_t)cta_kmax(r->F) * 4, stream) !=
            cudaSuccess) {
          cudaGetLastError();
          r->Q = nullptr;
          ok = false;
        }
      }
      ServeSlot& hs = h_slots[r->slot];
      std::memset(&hs, 0, sizeof(hs));
      hs.job.A = r->A;
      hs.job.H = nullptr;
      hs.job.seed = r->seed;
      hs.job.n = (uint32_t)r->n;
      hs.job.F = r->F;
      hs.job.slot = (uint32_t)r->slot;
      hs.elem_bytes = r->elem_bytes;
      hs.rs.Q = r->Q;
      if (!ok) {
        hs.rs.started = 1;
        hs.rs.done = 1;
        hs.rs.status = PIP_ENOMEM;
      }
      cudaMemcpyAsync(d_slots + r->slot, &hs, sizeof(ServeSlot), cudaMemcpyHostToDevice, stream);
    }
    // one tick over every resident request, the most remaining work first
    // (the largest requests set the makespan), each for a time slice that
    // spreads the tick's time budget over the requests per block
    uint32_t count = 0;
    int max_slot = -1;
    std::vector<std::pair<uint64_t, int>> order;
    order.reserve(resident.size());
    for (Req* r : resident) {
      const ServeSlot& hs = h_slots[r->slot];
      const uint64_t left = hs.rs.started ? (uint64_t)hs.rs.L + hs.rs.nl : r->n;
      order.emplace_back(left, r->slot);
      max_slot = std::max(max_slot, r->slot);
      r->ticks += 1;
    }
    std::sort(order.begin(), order.end(), [](const auto& x, const auto& y) { return x.first > y.first; });
    for (const auto& o : order) h_work[count++] = (uint32_t)o.second;
    if (count > 0) {
      cudaMemcpyAsync(d_work, h_work, count * sizeof(uint32_t), cudaMemcpyHostToDevice, stream);
      cudaMemsetAsync(d_next, 0, sizeof(uint32_t), stream);
      const uint32_t grid = std::max(1u, std::min(count, blocks));
      const uint64_t waves = (count + grid - 1) / grid;
      const uint64_t slice = std::max<uint64_t>(20000ull, tick_ns / waves);
      serve_tick_kernel<<<grid, threads, smem, stream>>>(d_slots, d_work, count, d_next, fmax, sigma,
                                                         rounds_per_tick, 120000000000ull, slice);
      cudaMemcpyAsync(h_slots, d_slots, (size_t)(max_slot + 1) * sizeof(ServeSlot), cudaMemcpyDeviceToHost, stream);
    }
    const cudaError_t e = cudaStreamSynchronize(stream);
    const int64_t t = now_ns();
    {
      std::lock_guard<std::mutex> lk(mu);
      ++ticks;
      if (e != cudaSuccess) {
        cudaGetLastError();
        loop_error = PIP_ECUDA;
      }
      std::vector<Req*> still;
      for (Req* r : resident) {
        const ServeSlot& hs = h_slots[r->slot];
        if (hs.rs.done || e != cudaSuccess) {
          r->done = true;
          r->status = e != cudaSuccess ? (uint32_t)PIP_ECUDA : hs.rs.status;
          r->rounds = hs.rs.rounds;
          r->attempts = hs.rs.attempts;
          r->losers = hs.rs.losers;
          r->done_ns = t;
          if (r->Q != nullptr) cudaFreeAsync(r->Q, stream);
          r->Q = nullptr;
          used -= r->aux_bytes;
          free_slots.push_back(r->slot);
          ++completed;
          finished.push_back(r->ticket);
          if (r->status != PIP_OK && r->owned) {
            // a failed request keeps no server-owned array; its charge goes back now
            if (r->A != nullptr) cudaFreeAsync(r->A, stream);
            r->A = nullptr;
            used -= r->array_bytes;
            r->array_bytes = 0;
          }
        } else {
          still.push_back(r);
        }
      }
      resident.swap(still);
    }
    cv_done.notify_all();
  }
  cudaStreamSynchronize(stream);
}

extern "C" {

pip_status pip_serve_create(pip_server** out, uint64_t device_budget_bytes, int device, const pip_serve_options* opt) {
  using namespace pip;
  if (out == nullptr || device_budget_bytes == 0) return PIP_EINVAL;
  pip_server* s = new (std::nothrow) pip_server();
  if (s == nullptr) return PIP_ENOMEM;
  if (opt != nullptr) s->opt = *opt;
  s->device = device;
  s->budget = device_budget_bytes;
  if (cudaSetDevice(device) != cudaSuccess) {
    cudaGetLastError();
    delete s;
    return PIP_ECUDA;
  }
  s->sigma = s->opt.slot_factor ? s->opt.slot_factor : 4u;
  s->fmax = s->opt.fresh_cap ? s->opt.fresh_cap : 1024u;
  s->threads = s->opt.block_threads ? s->opt.block_threads : 512u;
  s->max_resident = s->opt.max_resident ? s->opt.max_resident : 1024u;
  s->rounds_per_tick = s->opt.rounds_per_tick ? s->opt.rounds_per_tick : 1000000u;
  s->tick_ns = (uint64_t)(s->opt.tick_us ? s->opt.tick_us : 1000u) * 1000ull;
  if (s->sigma < 2 || s->sigma > 16 || s->threads < 128 || s->threads > 1024 || s->threads % 32 ||
      s->fmax > cta_max_fmax(s->sigma)) {
    delete s;
    return PIP_EINVAL;
  }
  s->smem = cta_smem_bytes(s->fmax, s->sigma);
  const void* k = reinterpret_cast<const void*>(&serve_tick_kernel);
  int optin = 0;
  cudaFuncAttributes fa{};
  if (cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, device) != cudaSuccess ||
      cudaFuncGetAttributes(&fa, k) != cudaSuccess ||
      cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, optin - (int)fa.sharedSizeBytes) !=
          cudaSuccess) {
    cudaGetLastError();
    delete s;
    return PIP_ECUDA;
  }
  int per_sm = 0;
  DeviceInfo di;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, (int)s->threads, s->smem) != cudaSuccess ||
      per_sm < 1 || device_info(&di) != PIP_OK) {
    cudaGetLastError();
    delete s;
    return PIP_EINVAL;
  }
  s->blocks = (uint32_t)per_sm * (uint32_t)di.sms;
  // by default a request is resident only while a tick block is free for it,
  // so every resident request advances for the whole tick (requests beyond
  // that wait in the arrival-ordered admission queue)
  if (s->opt.max_resident == 0) s->max_resident = s->blocks;
  if (cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking) != cudaSuccess ||
      cudaMalloc(&s->d_slots, sizeof(ServeSlot) * s->max_resident) != cudaSuccess ||
      cudaMallocHost(&s->h_slots, sizeof(ServeSlot) * s->max_resident) != cudaSuccess ||
      cudaMalloc(&s->d_work, sizeof(uint32_t) * s->max_resident) != cudaSuccess ||
      cudaMallocHost(&s->h_work, sizeof(uint32_t) * s->max_resident) != cudaSuccess ||
      cudaMalloc(&s->d_next, sizeof(uint32_t)) != cudaSuccess) {
    cudaGetLastError();
    if (s->stream) cudaStreamDestroy(s->stream);
    cudaFree(s->d_slots);
    cudaFreeHost(s->h_slots);
    cudaFree(s->d_work);
    cudaFreeHost(s->h_work);
    cudaFree(s->d_next);
    delete s;
    return PIP_ENOMEM;
  }
  for (int j = (int)s->max_resident - 1; j >= 0; --j) s->free_slots.push_back(j);
  s->th = std::thread([s] { s->loop(); });
  *out = s;
  return PIP_OK;
}

pip_status pip_serve_submit(pip_server* s, void* A_dev, uint64_t n, pip_dtype dtype, uint64_t seed, double eps,
                            uint64_t* ticket) {
  using namespace pip;
  if (s == nullptr || ticket == nullptr) return PIP_EINVAL;
  const uint32_t eb = elem_bytes_of(dtype);
  if (eb == 0 || !(eps > 0.0 && eps < 1.0) || n >= (1ull << 32)) return PIP_EINVAL;
  if (A_dev != nullptr && reinterpret_cast<uintptr_t>(A_dev) % eb != 0) return PIP_EINVAL;
  Req* r = new (std::nothrow) Req();
  if (r == nullptr) return PIP_ENOMEM;
  r->n = n;
  r->elem_bytes = eb;
  r->seed = seed;
  r->eps = eps;
  r->A = A_dev;
  pip_options o{};
  o.prefix_c = s->opt.prefix_c > 0.0 ? s->opt.prefix_c : 1.0;
  r->F = n >= 2 ? cta_fresh(n, eps, &o, s->sigma, s->fmax) : 1u;
  r->array_bytes = n * eb;
  r->aux_bytes = req_aux_bytes(r->F);
  if (r->array_bytes + r->aux_bytes > s->budget) {
    delete r;
    return PIP_EINVAL;  // can never be admitted
  }
  r->submit_ns = now_ns();
  {
    std::lock_guard<std::mutex> lk(s->mu);
    r->ticket = s->next_ticket++;
    s->reqs[r->ticket] = r;
    s->waiting.push_back(r);
    ++s->submitted;
    *ticket = r->ticket;
  }
  s->cv_work.notify_one();
  return PIP_OK;
}

static void fill_stats(const pip::Req* r, pip_req_stats* st) {
  if (st == nullptr) return;
  std::memset(st, 0, sizeof(*st));
  st->status = r->status;
  st->rounds = r->rounds;
  st->attempts = r->attempts;
  st->losers = r->losers;
  st->n = r->n;
  st->charged_bytes = r->array_bytes + r->aux_bytes;
  st->submit_ns = r->submit_ns;
  st->admit_ns = r->admit_ns;
  st->done_ns = r->done_ns;
  st->ticks = r->ticks;
  st->fresh_per_round = r->F;
}

pip_status pip_serve_poll(pip_server* s, uint64_t ticket, void** A_out, pip_req_stats* st) {
  if (s == nullptr) return PIP_EINVAL;
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->reqs.find(ticket);
  if (it == s->reqs.end()) return PIP_EINVAL;
  const pip::Req* r = it->second;
  if (!r->done) return PIP_EAGAIN;
  if (A_out != nullptr) *A_out = r->A;
  fill_stats(r, st);
  return static_cast<pip_status>(r->status);
}

pip_status pip_serve_wait(pip_server* s, uint64_t ticket, uint32_t timeout_ms, void** A_out, pip_req_stats* st) {
  if (s == nullptr) return PIP_EINVAL;
  std::unique_lock<std::mutex> lk(s->mu);
  auto it = s->reqs.find(ticket);
  if (it == s->reqs.end()) return PIP_EINVAL;
  const pip::Req* r = it->second;
  if (!s->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), [&] { return r->done; })) return PIP_EAGAIN;
  if (A_out != nullptr) *A_out = r->A;
  fill_stats(r, st);
  return static_cast<pip_status>(r->status);
}

pip_status pip_serve_next_done(pip_server* s, uint32_t timeout_ms, uint64_t* ticket) {
  if (s == nullptr || ticket == nullptr) return PIP_EINVAL;
  std::unique_lock<std::mutex> lk(s->mu);
  for (;;) {
    if (!s->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), [&] { return !s->finished.empty(); }))
      return PIP_EAGAIN;
    const uint64_t t = s->finished.front();
    s->finished.pop_front();
    if (s->reqs.count(t)) {  // skip requests released before they were collected here
      *ticket = t;
      return PIP_OK;
    }
  }
}

pip_status pip_serve_release(pip_server* s, uint64_t ticket) {
  if (s == nullptr) return PIP_EINVAL;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end()) return PIP_EINVAL;
    pip::Req* r = it->second;
    if (!r->done) return PIP_EAGAIN;
    if (r->owned && r->A != nullptr) s->to_free.push_back(r->A);
    s->used -= r->array_bytes;
    s->reqs.erase(it);
    delete r;
  }
  s->cv_work.notify_one();
  return PIP_OK;
}

pip_status pip_serve_info_get(pip_server* s, pip_serve_info* out) {
  if (s == nullptr || out == nullptr) return PIP_EINVAL;
  std::lock_guard<std::mutex> lk(s->mu);
  std::memset(out, 0, sizeof(*out));
  out->budget_bytes = s->budget;
  out->used_bytes = s->used;
  out->peak_used_bytes = s->peak_used;
  out->submitted = s->submitted;
  out->admitted = s->admitted;
  out->completed = s->completed;
  out->ticks = s->ticks;
  out->resident = (uint32_t)s->resident.size();
  out->waiting = (uint32_t)s->waiting.size();
  out->tick_blocks = s->blocks;
  out->fresh_cap = s->fmax;
  out->status = s->loop_error;
  return PIP_OK;
}

pip_status pip_serve_destroy(pip_server* s) {
  if (s == nullptr) return PIP_EINVAL;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
    // requests never admitted are dropped
    for (pip::Req* r : s->waiting) {
      s->reqs.erase(r->ticket);
      delete r;
    }
    s->waiting.clear();
  }
  s->cv_work.notify_all();
  if (s->th.joinable()) s->th.join();
  cudaSetDevice(s->device);
  for (auto& kv : s->reqs) {
    pip::Req* r = kv.second;
    if (r->owned && r->A != nullptr) cudaFreeAsync(r->A, s->stream);
    if (r->Q != nullptr) cudaFreeAsync(r->Q, s->stream);
    delete r;
  }
  for (void* p : s->to_free) cudaFreeAsync(p, s->stream);
  cudaStreamSynchronize(s->stream);
  cudaStreamDestroy(s->stream);
  cudaFree(s->d_slots);
  cudaFreeHost(s->h_slots);
  cudaFree(s->d_work);
  cudaFreeHost(s->h_work);
  cudaFree(s->d_next);
  const pip_status st = s->loop_error;
  delete s;
  return st;
}

}  // extern "C"
