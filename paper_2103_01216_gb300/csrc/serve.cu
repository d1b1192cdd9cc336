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
//
// Large requests take a lane instead of a tick block: one launch of the
// persistent grid driver with a few dozen blocks (about one per thousand
// fresh swaps of its prefix) on a low-priority stream of its own, next to
// the ticks.  One block would need the request's whole length in rounds of
// a ~1K prefix; the lane's prefix is the one the scratch bound allows, so a
// 2^28-element request takes tens of milliseconds instead of about a
// second.  A lane launch is not cooperative (the ticks hold SMs too), so its
// blocks first meet at a start gate: if they are not all resident in time
// they leave before touching anything, and the loop launches it again.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cmath>
#include <cstdint>
#include <cstdlib>
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

// Work counter and start time of one tick, cleared before every launch.
struct TickCtl {
  uint32_t next;
  uint32_t pad;
  unsigned long long start;  // globaltimer of the first block to start
};

// One tick: blocks take resident requests in the order of `work` and
// advance each for a time slice.  The tick ends `tick_ns` after its first
// block started, whatever the residency: a block that starts late (SMs held
// by lane launches) takes a shorter slice or no request, so one tick never
// stretches into several while the lanes run.
__global__ void __launch_bounds__(1024) serve_tick_kernel(ServeSlot* slots, const uint32_t* work, uint32_t count,
                                                          TickCtl* ctl, uint32_t fmax, uint32_t sigma,
                                                          uint32_t budget, uint64_t deadline_ns, uint64_t slice_ns,
                                                          uint64_t tick_ns) {
  extern __shared__ uint32_t smem[];
  __shared__ uint32_t s_w;
  __shared__ uint64_t s_slice;
  const uint64_t t0 = globaltimer_ns();
  if (threadIdx.x == 0) atomicCAS(&ctl->start, 0ull, (unsigned long long)t0);
  for (;;) {
    if (threadIdx.x == 0) {
      const uint64_t end = ld_relaxed_u64(&ctl->start) + tick_ns, now = globaltimer_ns();
      s_w = now + 10000ull < end ? atomicAdd(&ctl->next, 1u) : count;  // less than 10 us left: stop
      s_slice = now < end ? min(slice_ns, end - now) : 0ull;
    }
    __syncthreads();
    const uint32_t w = s_w;
    const uint64_t slice = s_slice;
    __syncthreads();
    if (w >= count) break;
    ServeSlot* sl = slots + work[w];
    const BatchJob job = sl->job;
    uint32_t st;
    if (sl->elem_bytes == 4)
      st = run_job<uint32_t>(job, smem, fmax, sigma, deadline_ns, t0, nullptr, &sl->rs, budget, false, slice);
    else if (sl->elem_bytes == 8)
      st = run_job<unsigned long long>(job, smem, fmax, sigma, deadline_ns, t0, nullptr, &sl->rs, budget, false,
                                       slice);
    else st = run_job<uint4>(job, smem, fmax, sigma, deadline_ns, t0, nullptr, &sl->rs, budget, false, slice);
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
  // lane requests: the grid plan, its scratch, the lane running it
  bool lane_ok = false;
  Plan plan;
  void* aux = nullptr;
  int lane = -1;
  uint32_t lane_retries = 0;
  bool done = false;
  bool released = false;
  uint32_t status = 0;
  uint32_t rounds = 0;
  uint64_t attempts = 0, losers = 0;
  uint32_t ticks = 0;
  int64_t submit_ns = 0, admit_ns = 0, done_ns = 0;
};

// One lane: a low-priority stream, the completion event of its current
// launch and the launch's statistics (device record and its host copy).
struct Lane {
  cudaStream_t stream = nullptr;
  cudaEvent_t done = nullptr;
  pip_stats* d_stats = nullptr;
  pip_stats* h_stats = nullptr;
  Req* req = nullptr;
};

constexpr uint64_t kLaneGateNs = 200000000ull;  // a lane's blocks must all be resident within 200 ms
constexpr uint32_t kLaneMinF = 2048;             // smaller prefixes stay on one block
constexpr uint32_t kLaneMaxRetries = 8;
constexpr uint32_t kMaxAdmitSkips = 512;         // waiting requests one admission pass may step over

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
  pip::TickCtl* d_next = nullptr;
  std::vector<int> free_slots;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<pip::Req*> waiting;
  std::vector<pip::Req*> resident;
  // lanes
  std::vector<pip::Lane> lanes;
  uint32_t lane_min_log2 = 22, lane_block_budget = 0, lane_blocks_used = 0;
  uint64_t lane_requests = 0, lane_launches = 0, tick_kernels = 0, tick_wait_ns = 0, lane_setup_ns = 0;
  std::vector<pip::Req*> lane_resident;
  uint64_t wake = 0;  // bumped by every submission and release (the loop's idle wait watches it)
  // The server's own memory pool.  The streams of the ticks and of the lanes
  // share it, and it never makes one stream wait for another to reuse memory
  // (no internal dependencies): with the default pool, an allocation on the
  // tick stream could be made to wait for a lane's long kernel.  It keeps
  // freed memory mapped up to the budget.
  cudaMemPool_t pool = nullptr;
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

namespace pip {
namespace {

// Queues a lane request's launch on its lane's stream: its array (when the
// server owns it), its scratch, the gated grid driver, the copy of its
// statistics and the completion event.  False when an allocation or a
// launch failed (the request then fails alone).
bool lane_launch(Lane& L, Req* r, bool first, cudaMemPool_t pool, uint64_t* launches) {
  if (first && r->A == nullptr && r->n > 0) {
    r->owned = true;
    if (cudaMallocFromPoolAsync(&r->A, r->array_bytes, pool, L.stream) != cudaSuccess) {
      cudaGetLastError();
      r->A = nullptr;
      r->status = PIP_ENOMEM;
      return false;
    }
    init_array_kernel<<<std::min<uint64_t>(4096, (r->n + 255) / 256 + 1), 256, 0, L.stream>>>(
        r->A, (uint32_t)r->n, r->elem_bytes);
  }
  if (first) {
    if (cudaMallocFromPoolAsync(&r->aux, r->plan.aux_bytes, pool, L.stream) != cudaSuccess) {
      cudaGetLastError();
      r->aux = nullptr;
      r->status = PIP_ENOMEM;
      return false;
    }
  }
  ++*launches;
  if (launch_grid_lane(r->plan, r->A, r->seed, r->aux, L.d_stats, kLaneGateNs, L.stream) != PIP_OK ||
      cudaMemcpyAsync(L.h_stats, L.d_stats, sizeof(pip_stats), cudaMemcpyDeviceToHost, L.stream) != cudaSuccess ||
      cudaEventRecord(L.done, L.stream) != cudaSuccess) {
    cudaGetLastError();
    r->status = PIP_ECUDA;
    return false;
  }
  return true;
}

}  // namespace
}  // namespace pip

void pip_server::loop() {
  using namespace pip;
  cudaSetDevice(device);
  std::vector<Req*> admit_now, admit_lane;
  std::vector<Req*> lane_failed;
  uint64_t seen_wake = 0;
  for (;;) {
    {
      std::unique_lock<std::mutex> lk(mu);
      cv_work.wait(lk, [&] {
        return stop || !waiting.empty() || !resident.empty() || !lane_resident.empty() || !to_free.empty();
      });
      if (stop && resident.empty() && lane_resident.empty()) break;
      seen_wake = wake;
      for (void* p : to_free) cudaFreeAsync(p, stream);
      to_free.clear();
      // Admission in arrival order: a request that does not fit the budget
      // blocks the ones behind it; a large request that only waits for a
      // lane (or a small one that waits for a tick slot) does not.
      admit_now.clear();
      admit_lane.clear();
      int free_lane = -1;
      for (size_t j = 0; j < lanes.size(); ++j)
        if (lanes[j].req == nullptr) free_lane = (int)j;
      uint32_t skipped = 0;  // bounds the scan past requests that wait for a lane or a slot
      for (auto it = waiting.begin(); !stop && it != waiting.end() && skipped < kMaxAdmitSkips;) {
        const bool slot_free = !free_slots.empty();
        if (!slot_free && free_lane < 0) break;
        Req* r = *it;
        const uint64_t charge = r->array_bytes + r->aux_bytes;
        if (used + charge > budget) break;
        if (r->lane_ok) {
          if (free_lane < 0 || lane_blocks_used + r->plan.blocks > lane_block_budget) {
            ++it;
            ++skipped;
            continue;
          }
          r->lane = free_lane;
          lanes[free_lane].req = r;
          lane_blocks_used += r->plan.blocks;
          lane_resident.push_back(r);
          admit_lane.push_back(r);
          ++lane_requests;
          free_lane = -1;
          for (size_t j = 0; j < lanes.size(); ++j)
            if (lanes[j].req == nullptr) free_lane = (int)j;
        } else {
          if (!slot_free) {
            ++it;
            ++skipped;
            continue;
          }
          r->slot = free_slots.back();
          free_slots.pop_back();
          admit_now.push_back(r);
          resident.push_back(r);
        }
        it = waiting.erase(it);
        used += charge;
        peak_used = std::max(peak_used, used);
        r->admit_ns = now_ns();
        ++admitted;
      }
    }
    // launch the newly admitted lane requests (stream-ordered on their lanes)
    lane_failed.clear();
    const int64_t t_lane = now_ns();
    for (Req* r : admit_lane)
      if (!lane_launch(lanes[r->lane], r, true, pool, &lane_launches)) lane_failed.push_back(r);
    lane_setup_ns += (uint64_t)(now_ns() - t_lane);
    // set up the newly admitted requests (allocations and copies are stream-ordered)
    for (Req* r : admit_now) {
      bool ok = true;
      if (r->A == nullptr && r->n > 0) {
        r->owned = true;
        if (cudaMallocFromPoolAsync(&r->A, r->array_bytes, pool, stream) != cudaSuccess) {
          cudaGetLastError();
          r->A = nullptr;
          ok = false;
        } else {
          init_array_kernel<<<std::min<uint64_t>(4096, (r->n + 255) / 256 + 1), 256, 0, stream>>>(
              r->A, (uint32_t)r->n, r->elem_bytes);
        }
      }
      if (ok && r->n >= 2) {
        if (cudaMallocFromPoolAsync(reinterpret_cast<void**>(&r->Q), (uint64_t)cta_kmax(r->F) * 4, pool, stream) !=
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
    // one tick over the resident requests, the least remaining work first
    // (the large requests run on lanes; among the rest, finishing the short
    // ones first keeps their latency at a tick or two), each for a time slice
    // that spreads the tick's time budget over the requests per block
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
    std::sort(order.begin(), order.end(), [](const auto& x, const auto& y) { return x.first < y.first; });
    for (const auto& o : order) h_work[count++] = (uint32_t)o.second;
    if (count > 0) {
      cudaMemcpyAsync(d_work, h_work, count * sizeof(uint32_t), cudaMemcpyHostToDevice, stream);
      cudaMemsetAsync(d_next, 0, sizeof(TickCtl), stream);
      const uint32_t grid = std::max(1u, std::min(count, blocks));
      const uint64_t waves = (count + grid - 1) / grid;
      const uint64_t slice = std::max<uint64_t>(20000ull, tick_ns / waves);
      serve_tick_kernel<<<grid, threads, smem, stream>>>(d_slots, d_work, count, d_next, fmax, sigma,
                                                         rounds_per_tick, 120000000000ull, slice, tick_ns);
      cudaMemcpyAsync(h_slots, d_slots, (size_t)(max_slot + 1) * sizeof(ServeSlot), cudaMemcpyDeviceToHost, stream);
    }
    const int64_t t_sync = now_ns();
    const cudaError_t e = cudaStreamSynchronize(stream);
    if (count > 0) {
      ++tick_kernels;
      tick_wait_ns += (uint64_t)(now_ns() - t_sync);
    }
    if (count == 0 && admit_lane.empty() && admit_now.empty()) {
      // no tick ran: wait for a lane to finish (polled), a submission or a
      // release, instead of spinning
      std::unique_lock<std::mutex> lk(mu);
      const auto limit = lane_resident.empty() ? std::chrono::microseconds(5000) : std::chrono::microseconds(100);
      cv_work.wait_for(lk, limit, [&] { return stop || wake != seen_wake; });
    }
    // lanes whose launch finished: retire the request, or launch it again
    // when its blocks could not all meet at the start gate
    std::vector<Req*> lane_done;
    for (Lane& L : lanes) {
      Req* r = L.req;
      if (r == nullptr || std::find(lane_failed.begin(), lane_failed.end(), r) != lane_failed.end()) continue;
      const cudaError_t q = cudaEventQuery(L.done);
      if (q == cudaErrorNotReady) continue;
      if (q != cudaSuccess) {
        cudaGetLastError();
        r->status = PIP_ECUDA;
      } else {
        r->status = L.h_stats->status;
        r->rounds = L.h_stats->rounds;
        r->attempts = L.h_stats->attempts;
        r->losers = L.h_stats->losers;
        if (r->status == PIP_EBUSY && r->lane_retries < kLaneMaxRetries) {
          ++r->lane_retries;
          if (lane_launch(L, r, false, pool, &lane_launches)) continue;
        }
      }
      lane_done.push_back(r);
    }
    for (Req* r : lane_failed) lane_done.push_back(r);
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
      for (Req* r : lane_done) {
        Lane& L = lanes[r->lane];
        r->done = true;
        r->done_ns = t;
        r->ticks += 1;
        if (r->aux != nullptr) cudaFreeAsync(r->aux, L.stream);
        r->aux = nullptr;
        used -= r->aux_bytes;
        lane_blocks_used -= r->plan.blocks;
        L.req = nullptr;
        ++completed;
        finished.push_back(r->ticket);
        if (r->status != PIP_OK && r->owned) {
          if (r->A != nullptr) cudaFreeAsync(r->A, L.stream);
          r->A = nullptr;
          used -= r->array_bytes;
          r->array_bytes = 0;
        }
        lane_resident.erase(std::find(lane_resident.begin(), lane_resident.end(), r));
      }
    }
    cv_done.notify_all();
  }
  cudaStreamSynchronize(stream);
  for (Lane& L : lanes) cudaStreamSynchronize(L.stream);
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
  // the tick stream has the highest priority: as SMs free up, the blocks of
  // the next tick (the small requests, each a few ticks long) are placed
  // ahead of pending lane blocks
  int prio_lo = 0, prio_hi = 0;
  cudaDeviceGetStreamPriorityRange(&prio_lo, &prio_hi);
  cudaGetLastError();
  if (cudaStreamCreateWithPriority(&s->stream, cudaStreamNonBlocking, prio_hi) != cudaSuccess ||
      cudaMalloc(&s->d_slots, sizeof(ServeSlot) * s->max_resident) != cudaSuccess ||
      cudaMallocHost(&s->h_slots, sizeof(ServeSlot) * s->max_resident) != cudaSuccess ||
      cudaMalloc(&s->d_work, sizeof(uint32_t) * s->max_resident) != cudaSuccess ||
      cudaMallocHost(&s->h_work, sizeof(uint32_t) * s->max_resident) != cudaSuccess ||
      cudaMalloc(&s->d_next, sizeof(pip::TickCtl)) != cudaSuccess) {
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
  {
    cudaMemPoolProps pp{};
    pp.allocType = cudaMemAllocationTypePinned;
    pp.handleTypes = cudaMemHandleTypeNone;
    pp.location.type = cudaMemLocationTypeDevice;
    pp.location.id = device;
    int no = 0, yes = 1;
    uint64_t keep = device_budget_bytes;
    if (cudaMemPoolCreate(&s->pool, &pp) != cudaSuccess ||
        cudaMemPoolSetAttribute(s->pool, cudaMemPoolReuseAllowInternalDependencies, &no) != cudaSuccess ||
        cudaMemPoolSetAttribute(s->pool, cudaMemPoolReuseAllowOpportunistic, &yes) != cudaSuccess ||
        cudaMemPoolSetAttribute(s->pool, cudaMemPoolAttrReleaseThreshold, &keep) != cudaSuccess) {
      cudaGetLastError();
      if (s->pool) cudaMemPoolDestroy(s->pool);
      cudaStreamDestroy(s->stream);
      cudaFree(s->d_slots);
      cudaFreeHost(s->h_slots);
      cudaFree(s->d_work);
      cudaFreeHost(s->h_work);
      cudaFree(s->d_next);
      delete s;
      return PIP_ECUDA;
    }
  }
  // lanes: streams of the lowest priority (their persistent launches take
  // what the ticks leave)
  // Each stream needs a host-to-device work queue of its own: streams that
  // share one (CUDA_DEVICE_MAX_CONNECTIONS, default 8) queue behind each
  // other's launches, and a tick would then wait for a lane's persistent
  // launch.  The default keeps the tick stream and the lanes within the
  // connections, with two to spare for the caller's streams.
  uint32_t connections = 8;
  if (const char* e = std::getenv("CUDA_DEVICE_MAX_CONNECTIONS")) {
    const long v = std::atol(e);
    if (v >= 1 && v <= 32) connections = (uint32_t)v;
  }
  const uint32_t lanes_default = connections > 3 ? std::min(16u, connections - 3) : 0u;
  const uint32_t nl = s->opt.lanes == PIP_SERVE_NO_LANES ? 0u : (s->opt.lanes ? s->opt.lanes : lanes_default);
  s->lane_min_log2 = s->opt.lane_min_log2 ? s->opt.lane_min_log2 : 22u;
  const uint32_t grid_cap = grid_driver_max_blocks(8, false, 512, 1024);
  s->lane_block_budget = s->opt.lane_blocks ? std::min(s->opt.lane_blocks, grid_cap) : grid_cap / 2;
  bool lanes_ok = true;
  for (uint32_t j = 0; j < nl && lanes_ok; ++j) {
    Lane L;
    lanes_ok = cudaStreamCreateWithPriority(&L.stream, cudaStreamNonBlocking, prio_lo) == cudaSuccess &&
               cudaEventCreateWithFlags(&L.done, cudaEventDisableTiming) == cudaSuccess &&
               cudaMalloc(&L.d_stats, sizeof(pip_stats)) == cudaSuccess &&
               cudaMallocHost(&L.h_stats, sizeof(pip_stats)) == cudaSuccess;
    s->lanes.push_back(L);
  }
  if (!lanes_ok) {
    cudaGetLastError();
    for (Lane& L : s->lanes) {
      if (L.stream) cudaStreamDestroy(L.stream);
      if (L.done) cudaEventDestroy(L.done);
      cudaFree(L.d_stats);
      cudaFreeHost(L.h_stats);
    }
    s->lanes.clear();
    cudaMemPoolDestroy(s->pool);
    cudaStreamDestroy(s->stream);
    cudaFree(s->d_slots);
    cudaFreeHost(s->h_slots);
    cudaFree(s->d_work);
    cudaFreeHost(s->h_work);
    cudaFree(s->d_next);
    delete s;
    return PIP_ENOMEM;
  }
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
  if (!s->lanes.empty() && s->lane_min_log2 < 64 && n >= (1ull << s->lane_min_log2)) {
    // a lane: the grid plan the scratch bound allows, on about one block of
    // 512 threads per thousand fresh swaps (two positions per thread)
    int cur = -1;
    const bool switch_dev = cudaGetDevice(&cur) == cudaSuccess && cur != s->device;
    if (switch_dev) cudaSetDevice(s->device);
    pip_options g{};
    g.flags = PIP_FLAG_FORCE_GRID;
    g.block_threads = 512;
    g.slot_factor = s->sigma;
    Plan p0;
    if (make_plan(n, dtype, eps, &g, &p0) == PIP_OK && p0.F >= kLaneMinF) {
      const uint64_t want = (5ull * p0.F / 4 + 1023) / 1024;
      g.grid_blocks = (uint32_t)std::min<uint64_t>(64, std::max<uint64_t>(2, want));
      Plan p1;
      if (make_plan(n, dtype, eps, &g, &p1) == PIP_OK && p1.blocks <= s->lane_block_budget) {
        r->lane_ok = true;
        r->plan = p1;
        r->F = p1.F;
        r->aux_bytes = p1.aux_bytes;
      }
    }
    cudaGetLastError();
    if (switch_dev) cudaSetDevice(cur);
  }
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
    ++s->wake;
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
  st->lane_launches = r->lane >= 0 ? r->lane_retries + 1u : 0u;
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
    ++s->wake;
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
  out->lane_requests = (uint32_t)s->lane_requests;
  out->tick_kernels = s->tick_kernels;
  out->tick_wait_ns = s->tick_wait_ns;
  out->lane_launches = s->lane_launches;
  out->lane_setup_ns = s->lane_setup_ns;
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
  for (pip::Lane& L : s->lanes) cudaStreamSynchronize(L.stream);
  for (auto& kv : s->reqs) {
    pip::Req* r = kv.second;
    if (r->owned && r->A != nullptr) cudaFreeAsync(r->A, s->stream);
    if (r->Q != nullptr) cudaFreeAsync(r->Q, s->stream);
    if (r->aux != nullptr) cudaFreeAsync(r->aux, s->stream);
    delete r;
  }
  for (pip::Lane& L : s->lanes) {
    cudaStreamDestroy(L.stream);
    cudaEventDestroy(L.done);
    cudaFree(L.d_stats);
    cudaFreeHost(L.h_stats);
  }
  for (void* p : s->to_free) cudaFreeAsync(p, s->stream);
  cudaStreamSynchronize(s->stream);
  cudaMemPoolDestroy(s->pool);
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
