// Host planner: turns (n, dtype, eps, overrides) into the prefix size, table
// sizes, grid shape and the exact scratch layout of one shuffle.
//
// The relaxed PIP model (Section 3.2) allows O(n^(1-eps)) auxiliary space,
// and Theorem 4.1 / 4.2 process a prefix of n^(1-eps) swaps per round.  The
// library fixes the constant: every plan's scratch is at most
// PIP_AUX_C * n^(1-eps) + 4096 bytes, and the prefix F is the largest
// multiple of n^(1-eps) (capped by the option prefix_c, and by what keeps the
// hot reservation tables inside L2) that fits.
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <mutex>

#include "internal.h"

namespace pip {

namespace {

constexpr uint64_t kAlign = 256;
// Default C in F = C * n^(1-eps) for a single array: large enough that the
// scratch bound (or the L2 / shared-memory caps) decides, since fewer, larger
// rounds are faster whenever the tables still fit.
constexpr double kDefaultPrefixC = 4.0;
constexpr uint32_t kDefaultSlotFactor = 4;
constexpr uint32_t kDefaultThreads = 512;
constexpr uint64_t kDefaultTimeoutNs = 2000000000ull;
constexpr uint32_t kItemsPerThread = 2;  // target positions per thread per round when sizing the grid

uint64_t align_up(uint64_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

// Grid driver limits from the barrier word's fields: losers per round (at
// most kmax = 2.5 F + 2) fit 22 bits, arriving blocks 10 bits.
constexpr uint32_t kGridMaxF = 1600000;
constexpr uint32_t kGridMaxBlocks = 1023;

// Cap on the grid driver's active set: 2.5 F.  The driver fixes the next
// fresh block before the current round's losers are known, so it assumes
// that all but one of the m active swaps lose: F stays untouched while
// m - 1 + F <= kmax, i.e. with losers up to 1.5 F (they are 10-25 % of F at
// slot factors 3-4).  A cap of 1.5 F measured 40 % more rounds at
// n = 10^9, eps = 0.5.  Only the used part of the loser queues is touched.
#ifndef PIP_KMAX_NUM
#define PIP_KMAX_NUM 5
#endif
uint32_t kmax_of(uint32_t F) {
  return (uint32_t)std::min<uint64_t>(0xFFFFFFF0ull, (uint64_t)F * PIP_KMAX_NUM / 2 + 2);
}

// Words of the grid driver's window bitmap over F locations.
uint64_t window_words(uint32_t F) { return ((uint64_t)F + 31) / 32; }

// Fills the layout fields for a given F and slot factor; returns aux bytes.
uint64_t layout(Plan* p, uint32_t F, uint32_t slot_factor) {
  p->F = F;
  p->kmax = kmax_of(F);
  const uint64_t ns = (uint64_t)slot_factor * p->F + 32;
  p->nslots = (uint32_t)std::min<uint64_t>(ns, 0xFFFFFFF0ull);
  uint64_t off = align_up(sizeof(Ctrl));
  for (int j = 0; j < 3; ++j) {
    p->off_S[j] = off;
    off += align_up(4ull * p->nslots);
  }
  for (int j = 0; j < 3; ++j) {
    p->off_D[j] = off;
    off += align_up(4ull * window_words(p->F));
  }
  for (int j = 0; j < 2; ++j) {
    p->off_Q[j] = off;
    off += align_up(4ull * p->kmax);
  }
  p->aux_bytes = off;
  return off;
}

std::mutex g_dev_mu;
DeviceInfo g_dev[64];
bool g_dev_ok[64] = {};

}  // namespace

pip_status device_info(DeviceInfo* out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return PIP_ECUDA;
  }
  if (dev < 0 || dev >= 64) return PIP_ECUDA;
  std::lock_guard<std::mutex> lk(g_dev_mu);
  if (!g_dev_ok[dev]) {
    DeviceInfo d;
    int l2 = 0;
    if (cudaDeviceGetAttribute(&d.sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&d.max_threads_per_sm, cudaDevAttrMaxThreadsPerMultiProcessor, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, dev) != cudaSuccess) {
      cudaGetLastError();
      return PIP_ECUDA;
    }
    d.l2_bytes = (size_t)l2;
    g_dev[dev] = d;
    g_dev_ok[dev] = true;
  }
  *out = g_dev[dev];
  return PIP_OK;
}

uint32_t elem_bytes_of(pip_dtype dtype) {
  switch (dtype) {
    case PIP_U32: return 4;
    case PIP_U64: return 8;
    case PIP_REC128: return 16;
    default: return 0;
  }
}

uint64_t cta_job_bytes(uint32_t F, uint32_t sigma) { return cta_smem_bytes(F, sigma); }

uint32_t cta_fresh(uint64_t n, double eps, const pip_options* opt, uint32_t sigma, uint32_t fcap) {
  if (n < 2) return 1;
  pip_options o{};
  if (opt != nullptr) o = *opt;
  const double x = std::pow((double)n, 1.0 - eps);
  const uint64_t bound = (uint64_t)std::floor(PIP_AUX_C * x) + 4096;
  double want;
  if (o.fresh_per_round) want = (double)o.fresh_per_round;
  else want = (o.prefix_c > 0.0 ? o.prefix_c : kDefaultPrefixC) * x;
  uint64_t F = (uint64_t)std::max(1.0, std::ceil(want));
  F = std::min<uint64_t>({F, n - 1, (uint64_t)std::max(1u, fcap)});
  // device bytes (the 256-byte control block) plus shared memory stay in the
  // bound: largest such F by bisection (the cost grows with F)
  if (sizeof(Ctrl) + cta_job_bytes((uint32_t)F, sigma) > bound) {
    uint64_t lo = 1, hi = F;
    while (lo < hi) {
      const uint64_t mid = (lo + hi + 1) / 2;
      if (sizeof(Ctrl) + cta_job_bytes((uint32_t)mid, sigma) <= bound) lo = mid;
      else hi = mid - 1;
    }
    F = lo;
  }
  return (uint32_t)F;
}

namespace {
pip_status make_plan_sigma(uint64_t n, pip_dtype dtype, double eps, const pip_options* opt, Plan* out);
}  // namespace

// The plan with the default slot factor, except where the grid or cluster
// driver's prefix is small and set by the scratch bound (the latency-bound
// regime): there a slot factor of 3 leaves room for a larger prefix, so
// fewer rounds, at the cost of more spurious losers (measured at n = 10^9,
// eps = 0.5: F 67.7K instead of 55.8K, 104.3-104.7 against 110.9-114.1 ms;
// 2^30 records 124.1-125.3 against 136.6-138.4 ms; n = 2^20 on the cluster
// 1.43 against 1.54 ms; a slot factor of 2 was slower, 150 ms).  Where the
// prefix is capped by L2 (large prefixes) 3 was slower (71.1 against
// 62.4 ms at eps = 0.25), and the one-block driver at eps = 0.75 gained
// nothing (4.74 against 4.57 s), so 4 stays there.
pip_status make_plan(uint64_t n, pip_dtype dtype, double eps, const pip_options* opt, Plan* out) {
  pip_status st = make_plan_sigma(n, dtype, eps, opt, out);
  if (st != PIP_OK || (opt != nullptr && opt->slot_factor != 0)) return st;
  if (out->driver == kDriverCta || out->F > 131072u) return st;
  pip_options o{};
  if (opt != nullptr) o = *opt;
  o.slot_factor = 3;
  o.flags |= out->driver == kDriverGrid ? PIP_FLAG_FORCE_GRID : PIP_FLAG_FORCE_CLUSTER;
  Plan p3;
  if (make_plan_sigma(n, dtype, eps, &o, &p3) == PIP_OK && p3.driver == out->driver &&
      (uint64_t)p3.F * 10 > (uint64_t)out->F * 11) {
    p3.flags = (p3.flags & ~(PIP_FLAG_FORCE_GRID | PIP_FLAG_FORCE_CLUSTER)) |
               (out->flags & (PIP_FLAG_FORCE_GRID | PIP_FLAG_FORCE_CLUSTER));
    *out = p3;
  }
  return PIP_OK;
}

namespace {
pip_status make_plan_sigma(uint64_t n, pip_dtype dtype, double eps, const pip_options* opt, Plan* out) {
  const uint32_t eb = elem_bytes_of(dtype);
  if (eb == 0 || !(eps > 0.0 && eps < 1.0) || n >= (1ull << 32) || n < 2) return PIP_EINVAL;
  pip_options o{};
  if (opt != nullptr) o = *opt;
  Plan p;
  p.n = (uint32_t)n;
  p.elem_bytes = eb;
  p.eps = eps;
  p.flags = o.flags;

  const double x = std::pow((double)n, 1.0 - eps);  // n^(1-eps)
  p.aux_bound = (uint64_t)std::floor(PIP_AUX_C * x) + 4096;

  uint32_t slot_factor = o.slot_factor ? o.slot_factor : kDefaultSlotFactor;
  if (slot_factor < 2 || slot_factor > 16) return PIP_EINVAL;
  uint32_t threads = o.block_threads ? o.block_threads : kDefaultThreads;
  if (threads < 128 || threads > 1024 || threads % 32 != 0) return PIP_EINVAL;
  p.threads = threads;

  // requested prefix
  double want;
  if (o.fresh_per_round) {
    want = (double)o.fresh_per_round;
  } else {
    const double c = o.prefix_c > 0.0 ? o.prefix_c : kDefaultPrefixC;
    want = c * x;
  }
  uint64_t F = (uint64_t)std::max(1.0, std::ceil(want));
  F = std::min<uint64_t>(F, n - 1);
  // the three slot tables (read, reserved into, being cleared) stay within
  // a quarter of L2 unless the caller fixed F explicitly: the array's random
  // traffic shares L2 with them (n = 10^9 u64, eps = 0.25, slot factor 4:
  // F = 600K / 700K / 900K / 1.0M / 1.13M measured 59.2-59.5 / 59.2 / 59.7 /
  // 60.6 / 61.5 ms on one box; 2/5 of L2 gave the 1.13M)
  DeviceInfo di;
  const bool have_dev = device_info(&di) == PIP_OK;
  if (!o.fresh_per_round && !(o.prefix_c > 0.0) && have_dev && di.l2_bytes > 0) {
    const uint64_t hot_cap = di.l2_bytes / 4;
    const uint64_t per_F = 3ull * 4ull * slot_factor;  // 3 slot tables * 4 B * slots per F
    F = std::max<uint64_t>(1, std::min<uint64_t>(F, hot_cap / per_F));
  }
  // shrink until the scratch obeys the bound
  while (layout(&p, (uint32_t)F, slot_factor) > p.aux_bound && F > 1) {
    const double ratio = (double)p.aux_bound / (double)p.aux_bytes;
    uint64_t nf = (uint64_t)std::floor((double)F * std::min(ratio, 0.999));
    F = std::max<uint64_t>(1, std::min<uint64_t>(nf, F - 1));
  }
  if (p.aux_bytes > p.aux_bound) return PIP_EINVAL;  // cannot happen for n >= 2: F=1 needs ~2.3 KB

  p.sigma = slot_factor;
  // Driver choice.  Each driver has its own scratch cost per fresh swap; the
  // cheapest one whose own memory cap does not cut the (bound-limited)
  // prefix wins: one block, then one cluster, then the persistent grid.
  // The flags force a driver.
  const uint32_t fcap = cta_max_fmax(slot_factor);
  const uint64_t F_req = std::min<uint64_t>(
      n - 1, (uint64_t)std::max(1.0, std::ceil(o.fresh_per_round ? (double)o.fresh_per_round
                                                                   : (o.prefix_c > 0.0 ? o.prefix_c : kDefaultPrefixC) * x)));
  // Measured on GB300 (prefix sweep over the three drivers, n = 2^26): one
  // block costs 2.3-2.6 us per round up to F ~ 512 and degrades beyond ~1K
  // (one SM); a 16-CTA cluster costs 3.1-4.0 us per round for F in 1K-4K;
  // the grid costs 4.5-5 us per round at small F and wins from F ~ 6-8K on
  // (its throughput scales with the whole GPU).
  constexpr uint32_t kCtaMaxF = 768, kGridMinF = 6000;
  const uint32_t F_cta_nocap = cta_fresh(n, eps, opt, slot_factor, 0xFFFFFFFFu);
  const bool forced = (o.flags & (PIP_FLAG_FORCE_GRID | PIP_FLAG_FORCE_CTA | PIP_FLAG_FORCE_CLUSTER)) != 0;
  bool want_cta = (o.flags & PIP_FLAG_FORCE_CTA) || (!forced && F_cta_nocap <= std::min(fcap, kCtaMaxF));
  const bool grid_large = F >= kGridMinF;  // F here is the grid plan's (bound- and L2-limited) prefix
  // cluster: 16 CTAs when the device allows that many, else 8
  const uint32_t cl_threads = o.block_threads ? threads : 256u;
  uint32_t cl_cs = 0, F_cl = 0;
  if (!want_cta && !(o.flags & PIP_FLAG_FORCE_GRID) && have_dev &&
      ((o.flags & PIP_FLAG_FORCE_CLUSTER) || !grid_large)) {
    for (uint32_t cs : {16u, 8u}) {
      // largest F within the bound: shared memory of all CTAs + control block + two loser queues
      uint64_t lo = 1, hi = F_req;
      auto cost = [&](uint64_t f) {
        const uint64_t km = f * 5 / 2 + 2;
        return cluster_cta_smem((uint32_t)f, slot_factor, cs) * cs + sizeof(Ctrl) + 2 * align_up(4 * km);
      };
      while (lo < hi) {
        const uint64_t mid = (lo + hi + 1) / 2;
        if (cost(mid) <= p.aux_bound) lo = mid;
        else hi = mid - 1;
      }
      const uint64_t F_b = lo;
      if (cluster_supported(eb, cs, cl_threads, cluster_cta_smem((uint32_t)F_b, slot_factor, cs))) {
        cl_cs = cs;
        F_cl = (uint32_t)F_b;
        break;
      }
    }
  }
  const bool want_cluster = cl_cs != 0 && !(o.flags & PIP_FLAG_TWO_RES) &&
                            ((o.flags & PIP_FLAG_FORCE_CLUSTER) || (!forced && !want_cta && !grid_large));
  if (o.flags & PIP_FLAG_FORCE_CLUSTER && cl_cs == 0) return PIP_EINVAL;
  // the cluster driver implements the one-reservation rule only
  if ((o.flags & PIP_FLAG_TWO_RES) && (o.flags & PIP_FLAG_FORCE_CLUSTER)) return PIP_EINVAL;
  if (want_cluster) {
    p.driver = kDriverCluster;
    p.F = F_cl;
    p.kmax = p.F * 5 / 2 + 2;
    p.nslots = slot_factor * p.F + 32;
    p.blocks = cl_cs;
    p.threads = cl_threads;
    p.smem_bytes = cluster_cta_smem(p.F, slot_factor, cl_cs) * cl_cs;
    p.off_Q[0] = align_up(sizeof(Ctrl));
    p.off_Q[1] = p.off_Q[0] + align_up(4ull * p.kmax);
    p.aux_bytes = p.off_Q[1] + align_up(4ull * p.kmax);
    p.timeout_ns = o.wait_timeout_ns ? o.wait_timeout_ns : kDefaultTimeoutNs;
    p.deadline_ns = 60000000000ull + 5000ull * (p.n / p.F + 1) + 20ull * p.n;
    if (const char* e = std::getenv("PIP_DEADLINE_MS")) {
      const long long ms = std::atoll(e);
      if (ms > 0) p.deadline_ns = (uint64_t)ms * 1000000ull;
    }
    *out = p;
    return PIP_OK;
  }
  if (want_cta) {
    p.driver = kDriverCta;
    p.F = cta_fresh(n, eps, opt, slot_factor, fcap);
    p.kmax = cta_kmax(p.F);
    p.nslots = slot_factor * p.F + 32;
    p.smem_bytes = cta_job_bytes(p.F, slot_factor);
    p.aux_bytes = sizeof(Ctrl);
    p.blocks = 1;
    // one thread per fresh swap up to 1024, so that every fresh swap gets
    // the one-round-ahead loads (PIP_FLAG_PREFETCH turns them on)
    p.threads = o.block_threads ? threads : (p.F > 512u ? 1024u : 512u);
    p.flags |= PIP_FLAG_PREFETCH;
    uint64_t tmo = o.wait_timeout_ns ? o.wait_timeout_ns : kDefaultTimeoutNs;
    p.timeout_ns = tmo;
    p.deadline_ns = 60000000000ull + 5000ull * (p.n / p.F + 1) + 20ull * p.n;
    if (const char* e = std::getenv("PIP_DEADLINE_MS")) {
      const long long ms = std::atoll(e);
      if (ms > 0) p.deadline_ns = (uint64_t)ms * 1000000ull;
    }
    *out = p;
    return PIP_OK;
  }

  // the grid kernel is built for at most 512 threads per block
  if (o.block_threads > 512) return PIP_EINVAL;
  // grid: the per-round counts travel in 22-bit fields of the barrier word
  // (at most kmax losers), and the arrivals in a 10-bit field
  if (p.F > kGridMaxF) {
    layout(&p, kGridMaxF, slot_factor);
  }
  // Block size: 256 threads for small prefixes, where more and smaller
  // blocks shorten a latency-bound round (measured 107 against 116 ms at
  // n = 10^9, eps = 0.5), 512 for large ones (68.7 against 70.0 ms at
  // eps = 0.25).
  if (!o.block_threads) {
    threads = p.F <= 131072u ? 256u : 512u;
    p.threads = threads;
  }
  // Shape: enough threads for ~kItemsPerThread active swaps each (F plus a
  // quarter for carried losers) and at least two blocks per SM while each
  // still gets a warp's worth of items (measured: spreading a round over the
  // whole GPU shortens it even when blocks have little work), at most what
  // can be co-resident (a cooperative launch needs every block resident).
  // Each block keeps its losers in an on-chip list sized for a generous
  // share of them (overflow goes to the queue in device memory); that shared
  // memory counts against the aux bound, so F shrinks until everything fits.
  for (;;) {
    const uint64_t active_est = (uint64_t)p.F + p.F / 4 + 1;
    uint64_t want = (active_est + (uint64_t)threads * kItemsPerThread - 1) / ((uint64_t)threads * kItemsPerThread);
    // at least two blocks per SM while each still gets a warp's worth of
    // items, and at most two: a third block per SM measured slower with the
    // exchange commit (n = 10^9 u64, eps = 0.25, F = 706K: 304 blocks of 512
    // threads 58.8 ms, 456 of 512 61.1 ms, 608 of 256 59.5 ms, 152 of 512
    // 64.0 ms), its barrier arrivals and L2 traffic costing more than its
    // extra memory parallelism brings
    if (have_dev) {
      want = std::max<uint64_t>(want, std::min<uint64_t>(2ull * di.sms, (active_est + 31) / 32));
      want = std::min<uint64_t>(want, 2ull * di.sms);
    }
    if (o.grid_blocks) want = o.grid_blocks;
    want = std::max<uint64_t>(1, std::min<uint64_t>(want, kGridMaxBlocks));
    // blocks that fit with the largest list first, then the list for them
    const uint32_t maxb = have_dev ? grid_driver_max_blocks(eb, false, threads, 4096) : 0;
    if (maxb) want = std::min<uint64_t>(want, maxb);
    const uint64_t share = ((uint64_t)p.F * 3 / 8 + want - 1) / want;
    p.kloc = (uint32_t)std::min<uint64_t>(4096, std::max<uint64_t>(32, (share + 31) / 32 * 32));
    p.blocks = (uint32_t)want;
    p.smem_bytes = (uint64_t)p.blocks * grid_block_smem(p.kloc);
    if (p.aux_bytes + p.smem_bytes <= p.aux_bound || p.F <= 1) break;
    const double ratio = (double)p.aux_bound / (double)(p.aux_bytes + p.smem_bytes);
    const uint64_t nf = (uint64_t)std::floor((double)p.F * std::min(ratio, 0.999));
    layout(&p, (uint32_t)std::max<uint64_t>(1, std::min<uint64_t>(nf, p.F - 1)), slot_factor);
  }
  if (p.aux_bytes + p.smem_bytes > p.aux_bound) return PIP_EINVAL;

  uint64_t tmo = o.wait_timeout_ns ? o.wait_timeout_ns : kDefaultTimeoutNs;
  if (const char* e = std::getenv("PIP_WAIT_TIMEOUT_MS")) {
    const long long ms = std::atoll(e);
    if (ms > 0 && !o.wait_timeout_ns) tmo = (uint64_t)ms * 1000000ull;
  }
  p.timeout_ns = tmo;
  // Commit mode.  Small prefixes are latency-bound: issue both array loads
  // with the checks (measured 2-7 % faster up to F ~ 50K, 27 % slower at
  // F ~ 1.1M).  Large ones are bound by the rate of random accesses: the
  // exchange commit does one random L2 transaction per swap instead of two.
  // PIP_FLAG_SWAP_LOADSTORE / PIP_FLAG_SWAP_EXCHANGE force a mode.
  if (o.flags & PIP_FLAG_SWAP_LOADSTORE) {
    p.flags &= ~PIP_FLAG_SWAP_EXCHANGE;
    if (p.F <= 131072u) p.flags |= PIP_FLAG_SPECULATE;
  } else if (!(o.flags & PIP_FLAG_SWAP_EXCHANGE)) {
    if (p.F <= 131072u) p.flags |= PIP_FLAG_SPECULATE;
    else p.flags |= PIP_FLAG_SWAP_EXCHANGE;
  }
  // Phase order: small prefixes issue the next round's reservations and the
  // cleaning before the commit (n = 10^9 u64, eps = 0.5: 98.1 against
  // 99.8 ms; 2^30 records 109.1 against 111.2 ms; at eps = 0.25, F = 706K,
  // 60.1 against 58.1 ms, so large prefixes keep them after it).
  if (p.F <= 131072u) p.flags |= PIP_FLAG_EARLY_RESERVE;
  // whole-run limit: far above any legitimate run (about 1 us per round plus
  // 1 ns per element would already be slow), so only a defect can reach it
  uint64_t deadline = 60000000000ull + 2000ull * (p.n / p.F + 1) + 20ull * p.n;
  if (const char* e = std::getenv("PIP_DEADLINE_MS")) {
    const long long ms = std::atoll(e);
    if (ms > 0) deadline = (uint64_t)ms * 1000000ull;
  }
  p.deadline_ns = deadline;
  *out = p;
  return PIP_OK;
}
}  // namespace

}  // namespace pip
