// Cluster round driver: one thread-block cluster (up to 16 CTAs, one per SM)
// runs every round of one array's shuffle.  The reservation tables are spread
// over the cluster's shared memory (distributed shared memory, DSMEM) and the
// rounds are separated by the hardware cluster barrier, so a round costs two
// cluster barriers instead of a grid barrier through L2.  This is the driver
// for prefixes too large for one block's shared memory but small enough that
// a grid barrier would dominate each round (about 4K to 90K swaps).
//
// The round structure is the one of the other drivers (Algorithm 1 under the
// Decomposable Property, Section 4.1; RP-OneRes rule and RP-Final dense
// window, Appendix A.2; cleaning phase, Appendix A.1): round r commits with
// the tables of round r while its losers and the fresh block W_{r+1} reserve
// into the other buffer; after a cluster barrier each CTA clears its slice of
// round r's tables and a second barrier opens round r+1.
//
// Table slicing: slot s of a slot table lives in CTA s % CS at offset s / CS;
// window entry d of a dense window in CTA d % CS at offset d / CS.  The
// carried-loser queues stay in device memory (L2-resident); their counters
// live in CTA 0's shared memory.
#include <algorithm>
#include <cooperative_groups.h>
#include <cstdint>
#include <map>
#include <mutex>
#include <tuple>

#include "device.cuh"
#include "internal.h"

namespace cg = cooperative_groups;

namespace pip {
namespace {

constexpr unsigned kFullC = 0xffffffffu;
constexpr int kClU = 2;  // positions per thread whose loads are in flight together

struct ClusterArgs {
  void* A;
  const uint32_t* H;
  uint64_t seed;
  uint32_t n, F, kmax, ns;
  uint32_t nsr, fr;  // per-CTA slice lengths of one slot table / one dense window
  uint32_t* Q[2];
  Ctrl* ctrl;
  pip_stats* stats;
  uint32_t* latch;
  uint64_t deadline_ns;
  uint32_t prefetch;
};

template <bool kExplicit>
__device__ __forceinline__ uint32_t cl_target(const ClusterArgs& a, uint32_t i) {
  if constexpr (kExplicit) return __ldg(a.H + i);
  else return hashed_target(a.seed, i);
}

template <typename Elem, bool kExplicit>
__global__ void __launch_bounds__(1024) cluster_rounds_kernel(const ClusterArgs a) {
  extern __shared__ uint32_t smem[];
  __shared__ uint32_t s_cnt[2];
  __shared__ uint32_t s_abort;
  cg::cluster_group cl = cg::this_cluster();
  const uint32_t CS = cl.num_blocks();
  const uint32_t rank = cl.block_rank();
  const uint32_t NT = blockDim.x, tid = threadIdx.x, lane = tid & 31u;
  const uint32_t g = rank * NT + tid, T = CS * NT;
  const uint32_t nsr = a.nsr, fr = a.fr;
  Elem* A = static_cast<Elem*>(a.A);
  // local slices: S[0], S[1] (nsr words each), D[0], D[1] (fr words each)
  auto S_at = [&](uint32_t buf, uint32_t slot) -> uint32_t* {
    return cl.map_shared_rank(smem + buf * nsr + slot / CS, slot % CS);
  };
  auto D_at = [&](uint32_t buf, uint32_t d) -> uint32_t* {
    return cl.map_shared_rank(smem + 2 * nsr + buf * fr + d / CS, d % CS);
  };
  uint32_t* const cnt0 = cl.map_shared_rank(&s_cnt[0], 0);
  uint32_t* const abort0 = cl.map_shared_rank(&s_abort, 0);
  auto reserve = [&](uint32_t buf, uint32_t wlo, uint32_t whi, uint32_t h, uint32_t prio) {
    if (h >= wlo && h < whi) atomicMax(D_at(buf, h - wlo), prio);
    else atomicMax(S_at(buf, slot_of(h, a.ns)), prio);
  };

  const uint64_t t_start = globaltimer_ns();
  // an invalid explicit target sequence was reported by the validation pass
  // (every CTA reads the same word, so all leave together)
  if (block_status(&a.ctrl->status) != 0u) {
    if (rank == 0 && tid == 0) {
      atomicCAS(a.latch, 0u, ld_relaxed_u32(&a.ctrl->status));
      if (a.stats != nullptr) a.stats->status = ld_relaxed_u32(&a.ctrl->status);
    }
    return;
  }

  for (uint32_t j = tid; j < 2 * nsr + 2 * fr; j += NT) smem[j] = 0u;
  if (tid == 0) {
    s_cnt[0] = 0;
    s_cnt[1] = 0;
    s_abort = 0;
  }
  cl.sync();
  uint32_t Lprev = a.n;
  uint32_t L = a.n - min(a.F, a.n - 1u);
  uint32_t nl = 0;
  uint32_t m = Lprev - L;
  for (uint32_t i = L + g; i < Lprev; i += T) {
    const uint32_t h = cl_target<kExplicit>(a, i);
    if (h != i) reserve(0u, L, Lprev, h, i + 1u);
  }
  cl.sync();

  uint32_t rounds = 0, max_active = 0, status = 0;
  uint64_t attempts = 0, losers_total = 0;
  for (uint32_t r = 0;; ++r) {
    const uint32_t b = r & 1u, nb = b ^ 1u;
    uint32_t* const Qin = a.Q[b];
    uint32_t* const Qout = a.Q[nb];
    uint32_t fn = min(a.F, L - 1u);
    fn = min(fn, a.kmax - m + 1u);
    const uint32_t Ln = L - fn;
    // ---- commit round r
    for (uint32_t p0 = g & ~31u; p0 < m; p0 += kClU * T) {
      uint32_t ii[kClU], hh[kClU];
      bool win[kClU], lose[kClU];
#pragma unroll
      for (int j = 0; j < kClU; ++j) {
        const uint32_t p = p0 + lane + (uint32_t)j * T;
        ii[j] = 0;
        hh[j] = 0;
        win[j] = false;
        lose[j] = false;
        if (p < m) {
          const uint32_t i = (p < nl) ? ldcg(Qin + p) : L + (p - nl);
          const uint32_t h = cl_target<kExplicit>(a, i);
          ii[j] = i;
          hh[j] = h;
          if (h != i) {
            const uint32_t own = (i < Lprev) ? *D_at(b, i - L) : *S_at(b, slot_of(i, a.ns));
            const uint32_t rh = (h >= L && h < Lprev) ? *D_at(b, h - L) : *S_at(b, slot_of(h, a.ns));
            const bool own_free = (i < Lprev) ? (own == 0u) : (own <= i + 1u);
            win[j] = own_free && rh == i + 1u;
            lose[j] = !win[j];
          }
        }
      }
      Elem x[kClU], y[kClU];
#pragma unroll
      for (int j = 0; j < kClU; ++j) {
        if (win[j]) {
          x[j] = ldcg(A + ii[j]);
          y[j] = ldcg(A + hh[j]);
        }
      }
#pragma unroll
      for (int j = 0; j < kClU; ++j) {
        if (win[j]) {
          stcg(A + ii[j], y[j]);
          stcg(A + hh[j], x[j]);
        }
      }
#pragma unroll
      for (int j = 0; j < kClU; ++j) {
        if (lose[j]) reserve(nb, Ln, L, hh[j], ii[j] + 1u);
        const unsigned mask = __ballot_sync(kFullC, lose[j]);
        if (mask) {
          const int leader = __ffs(mask) - 1;
          uint32_t base = 0;
          if ((int)lane == leader) base = atomicAdd(cnt0 + nb, (uint32_t)__popc(mask));
          base = __shfl_sync(kFullC, base, leader);
          if (lose[j]) {
            const uint32_t q = base + __popc(mask & ((1u << lane) - 1u));
            if (q < a.kmax) stcg(Qout + q, ii[j]);
            else atomicOr(abort0, (uint32_t)PIP_EINTERNAL);
          }
        }
      }
    }
    // ---- fresh block W_{r+1} reserves (optionally pulling the array lines it
    // will swap into L2 one round ahead)
    for (uint32_t i = Ln + g; i < L; i += T) {
      const uint32_t h = cl_target<kExplicit>(a, i);
      if (h != i) {
        reserve(nb, Ln, L, h, i + 1u);
        if (a.prefetch) {
          asm volatile("prefetch.global.L2 [%0];" ::"l"(A + h));
          asm volatile("prefetch.global.L2 [%0];" ::"l"(A + i));
        }
      }
    }
    cl.sync();
    const uint32_t nl_next = cnt0[nb];
    // ---- clean this CTA's slices of round r's tables
    for (uint32_t j = tid; j < nsr; j += NT) smem[b * nsr + j] = 0u;
    for (uint32_t j = tid; j < fr; j += NT) smem[2 * nsr + b * fr + j] = 0u;
    if (rank == 0 && tid == 0) {
      s_cnt[b] = 0;
      if (nl_next >= m) s_abort |= PIP_EINTERNAL;  // no commit: impossible
      if (globaltimer_ns() - t_start > a.deadline_ns) s_abort |= PIP_ETIMEOUT;
    }
    cl.sync();
    rounds += 1u;
    attempts += m;
    losers_total += nl_next;
    max_active = max(max_active, m);
    const uint32_t ab = *abort0;
    if (ab != 0u) {
      status = (ab & PIP_ETIMEOUT) ? (uint32_t)PIP_ETIMEOUT : (uint32_t)PIP_EINTERNAL;
      break;
    }
    Lprev = L;
    L = Ln;
    nl = nl_next;
    m = nl_next + fn;
    if (m == 0u) break;
    if (m > a.kmax || rounds > a.n + 8u) {
      status = PIP_EINTERNAL;
      break;
    }
  }
  if (rank == 0 && tid == 0) {
    if (status != 0u) {
      set_status(&a.ctrl->status, status);
      atomicCAS(a.latch, 0u, status);
    }
    if (a.stats != nullptr) {
      a.stats->status = status;
      a.stats->rounds = rounds;
      a.stats->attempts = attempts;
      a.stats->losers = losers_total;
      a.stats->max_active = max_active;
      a.stats->grid_blocks = CS;
    }
  }
  cl.sync();  // no CTA leaves while another may still address its shared memory
}

__global__ void validate_cluster_kernel(const uint32_t* __restrict__ H, uint32_t n, Ctrl* ctrl) {
  bool bad = false;
  for (uint32_t i = 1u + blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    bad |= (H[i] > i);
  if (__syncthreads_or(bad) && threadIdx.x == 0) set_status(&ctrl->status, PIP_EINVAL);
}

template <typename Elem, bool kExplicit>
const void* cl_ptr() {
  return reinterpret_cast<const void*>(&cluster_rounds_kernel<Elem, kExplicit>);
}

const void* select_cluster_kernel(uint32_t elem_bytes, bool explicit_h) {
  switch (elem_bytes) {
    case 4: return explicit_h ? cl_ptr<uint32_t, true>() : cl_ptr<uint32_t, false>();
    case 8: return explicit_h ? cl_ptr<unsigned long long, true>() : cl_ptr<unsigned long long, false>();
    case 16: return explicit_h ? cl_ptr<uint4, true>() : cl_ptr<uint4, false>();
    default: return nullptr;
  }
}

std::mutex g_cl_mu;
std::map<std::tuple<int, const void*, uint32_t, uint32_t, uint64_t>, int> g_cl_ok;

// Sets the kernel attributes for a cluster launch of `cs` CTAs and checks that
// one such cluster can be resident; cached per device and shape.
bool prepare_cluster(const void* k, uint32_t cs, uint32_t threads, uint64_t smem) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  std::lock_guard<std::mutex> lk(g_cl_mu);
  const auto key = std::make_tuple(dev, k, cs, threads, smem);
  auto it = g_cl_ok.find(key);
  if (it != g_cl_ok.end()) return it->second != 0;
  int optin = 0;
  cudaFuncAttributes fa{};
  bool ok = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) == cudaSuccess &&
            cudaFuncGetAttributes(&fa, k) == cudaSuccess &&
            (uint64_t)(optin - (int)fa.sharedSizeBytes) >= smem &&
            cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, optin - (int)fa.sharedSizeBytes) ==
                cudaSuccess;
  if (ok && cs > 8) ok = cudaFuncSetAttribute(k, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) == cudaSuccess;
  if (ok) {
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3(cs);
    cfg.blockDim = dim3(threads);
    cfg.dynamicSmemBytes = smem;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = cs;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int clusters = 0;
    ok = cudaOccupancyMaxActiveClusters(&clusters, k, &cfg) == cudaSuccess && clusters >= 1;
  }
  if (!ok) cudaGetLastError();
  g_cl_ok[key] = ok ? 1 : 0;
  return ok;
}

}  // namespace

uint64_t cluster_cta_smem(uint32_t F, uint32_t sigma, uint32_t cs) {
  const uint64_t ns = (uint64_t)sigma * F + 32;
  const uint64_t nsr = (ns + cs - 1) / cs;
  const uint64_t fr = ((uint64_t)F + cs - 1) / cs;
  return 4ull * (2 * nsr + 2 * fr);
}

pip_status launch_cluster_driver(const Plan& plan, void* A, const uint32_t* H, uint64_t seed, void* aux,
                                 pip_stats* stats, cudaStream_t stream) {
  const void* k = select_cluster_kernel(plan.elem_bytes, H != nullptr);
  if (k == nullptr) return PIP_EINVAL;
  const uint32_t cs = plan.blocks;
  const uint64_t smem = cluster_cta_smem(plan.F, plan.sigma, cs);
  if (!prepare_cluster(k, cs, plan.threads, smem)) return PIP_EINVAL;
  char* base = static_cast<char*>(aux);
  ClusterArgs a{};
  a.A = A;
  a.H = H;
  a.seed = seed;
  a.n = plan.n;
  a.F = plan.F;
  a.kmax = plan.kmax;
  a.ns = plan.nslots;
  a.nsr = (plan.nslots + cs - 1) / cs;
  a.fr = (plan.F + cs - 1) / cs;
  a.Q[0] = reinterpret_cast<uint32_t*>(base + plan.off_Q[0]);
  a.Q[1] = reinterpret_cast<uint32_t*>(base + plan.off_Q[1]);
  a.ctrl = reinterpret_cast<Ctrl*>(base);
  a.stats = stats;
  a.latch = error_latch_ptr();
  a.deadline_ns = plan.deadline_ns;
  a.prefetch = (plan.flags & PIP_FLAG_PREFETCH) ? 1u : 0u;
  if (a.latch == nullptr) return PIP_ECUDA;
  if (cudaMemsetAsync(aux, 0, sizeof(Ctrl), stream) != cudaSuccess) return PIP_ECUDA;
  if (H != nullptr) {
    const uint32_t vb = (uint32_t)std::min<uint64_t>(1024, (plan.n + 255) / 256);
    validate_cluster_kernel<<<vb, 256, 0, stream>>>(H, plan.n, a.ctrl);
    if (cudaGetLastError() != cudaSuccess) return PIP_ECUDA;
  }
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = dim3(cs);
  cfg.blockDim = dim3(plan.threads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = cs;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  void* args[] = {&a};
  if (cudaLaunchKernelExC(&cfg, k, args) != cudaSuccess) {
    cudaGetLastError();
    return PIP_ECUDA;
  }
  return PIP_OK;
}

bool cluster_supported(uint32_t elem_bytes, uint32_t cs, uint32_t threads, uint64_t smem) {
  const void* k = select_cluster_kernel(elem_bytes, false);
  return k != nullptr && prepare_cluster(k, cs, threads, smem);
}

}  // namespace pip
