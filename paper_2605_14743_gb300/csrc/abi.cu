// abi.cu -- host side of the C ABI declared in include/afc.h: argument validation, launch
// configuration (shared-memory layout, thread groups, bucket width), the stream-ordered
// end-to-end query path and the bucket-width / group-size autotuner.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <stdexcept>
#include <string>
#include <thread>
#include <vector>

#include <cuda_runtime.h>

#include "afc.h"
#include "abi_util.h"
#include "afc_internal.h"

using namespace afc;

namespace afc {

std::string &abi_error_text() {
  thread_local std::string text;
  return text;
}

int fail(int code, const char *fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  abi_error_text() = buf;
  return code;
}

int cuda_fail(cudaError_t e, const char *what) {
  return fail(AFC_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

DevInfo dev_info() {
  DevInfo d;
  int dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&d.sms, cudaDevAttrMultiProcessorCount, dev);
  cudaDeviceGetAttribute(&d.smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  return d;
}

}  // namespace afc

namespace {

// Requested bucket width; the kernels round it up to a power of two (and to the ring bound).
uint32_t auto_delta(const afc_mc_problem &p) {
  if (p.bucket_width) return p.bucket_width;
  const double lo = p.w_lo ? 1.0 : (double)p.w_lo_all;
  const double hi = p.w_hi ? 100.0 : (double)p.w_hi_all;
  const double mean = 0.5 * (lo + hi);
  // measured: on the 1000-node Watts-Strogatz workload (lengths 1..100) the best width is about
  // the mean length (fewer buckets outweigh the extra in-bucket relaxation passes); on the
  // 20,000-node one (lengths 1..1000) about a quarter of it, as buckets hold more members
  const double shrink = std::min(1.0, std::sqrt(1000.0 / std::max(1, p.n)));
  return (uint32_t)std::max(1.0, std::floor(0.95 * mean * shrink));
}

int auto_block(const afc_mc_problem &p) {
  // measured: 1024-thread CTAs with one-warp teams are the fastest shape for small graphs too
  // (n = 64: 1.7x the former 256-thread CTAs)
  return p.block_threads ? p.block_threads : 1024;
}

int validate(const afc_mc_problem *p) {
  if (!p) return fail(AFC_EINVAL, "null problem");
  if (p->n < 1 || p->n > 65535) return fail(AFC_EUNSUPPORTED, "n = %d outside [1, 65535]", p->n);
  {
    // every distance, (n - 1) * max length at most, and one more arc must stay below 2^31
    const uint64_t wmax = p->w_hi ? 65535u : p->w_hi_all;
    if ((uint64_t)p->n * wmax >= 0x7FFFFFFFull)
      return fail(AFC_EUNSUPPORTED, "n * max length = %llu reaches 2^31 (distance range)",
                  (unsigned long long)((uint64_t)p->n * wmax));
  }
  if (p->memory_path < AFC_PATH_AUTO || p->memory_path > AFC_PATH_GLOBAL)
    return fail(AFC_EINVAL, "memory_path must be AFC_PATH_AUTO, _SHARED or _GLOBAL");
  if (p->reward_k || p->report_rank > 1) {
    if (p->precision != AFC_FP64 || p->in_w || p->top_k)
      return fail(AFC_EINVAL, "rewards and rank-r reports need FP64, no candidate pool and no rank cutoff");
    if (p->reward_k > 256 || p->report_rank > 256)
      return fail(AFC_EUNSUPPORTED, "at most 256 ranks per component");
    if (p->reward_k && !p->psi_sum) return fail(AFC_EINVAL, "reward_k needs psi_sum");
  }
  if (p->use_fallback != 0 && p->use_fallback != 1) return fail(AFC_EINVAL, "use_fallback must be 0 or 1");
  if (p->tie_random != 0 && p->tie_random != 1) return fail(AFC_EINVAL, "tie_random must be 0 or 1");
  if (p->wtab_ptr && !p->wtab) return fail(AFC_EINVAL, "wtab_ptr without wtab");
  if (p->per_row != 0 && p->per_row != 1) return fail(AFC_EINVAL, "per_row must be 0 or 1");
  if (p->hop_radius && !p->per_row) return fail(AFC_EINVAL, "hop_radius needs the row-wise mode (per_row = 1)");
  if (p->per_row && (p->reward_k || p->report_rank > 1))
    return fail(AFC_EINVAL, "the row-wise mode does not combine with rewards or rank-r reports");
  if (p->tie_random && (p->reward_k || p->report_rank > 1))
    return fail(AFC_EINVAL, "the randomised tie-break does not combine with rewards or rank-r reports");
  if (p->use_fallback) {
    if (p->fallback_node < 0 || p->fallback_node >= p->n)
      return fail(AFC_EINVAL, "fallback_node %d outside [0, n)", p->fallback_node);
    if (p->reward_k || p->report_rank > 1)
      return fail(AFC_EINVAL, "the fallback selector does not combine with rewards or rank-r reports");
  }
  if (p->m < 0 || p->m > 0x3FFFFFFF) return fail(AFC_EINVAL, "m = %lld out of range", (long long)p->m);
  if (!p->row_ptr || (p->m > 0 && (!p->col || !p->eid)))
    return fail(AFC_EINVAL, "CSR pointers missing");
  if (!p->w_lo && (p->w_lo_all < 1 || p->w_lo_all > 65535)) return fail(AFC_EINVAL, "w_lo_all must be in [1, 65535]");
  if (!p->w_hi && (p->w_hi_all < 1 || p->w_hi_all > 65535)) return fail(AFC_EINVAL, "w_hi_all must be in [1, 65535]");
  if (!p->w_lo && !p->w_hi && p->w_hi_all < p->w_lo_all) return fail(AFC_EINVAL, "w_hi_all < w_lo_all");
  if (!p->thresh && p->thresh_all > (1ull << 32)) return fail(AFC_EINVAL, "thresh_all > 2^32");
  if (p->k_min < 1) return fail(AFC_EINVAL, "k_min must be >= 1");
  if (!(p->tie_rel >= 0.0) || p->tie_rel >= 1.0) return fail(AFC_EINVAL, "tie_rel must be in [0, 1)");
  if (p->precision != AFC_FP64 && p->precision != AFC_FP32_RECHECK) return fail(AFC_EINVAL, "bad precision");
  if (p->precision == AFC_FP32_RECHECK && !(p->recheck_margin >= 0.0)) return fail(AFC_EINVAL, "bad recheck_margin");
  const int B = auto_block(*p);
  if (B != 256 && B != 512 && B != 1024) return fail(AFC_EINVAL, "block_threads must be 256, 512 or 1024");
  if (p->team_threads && !big_config_supported(B, p->team_threads))
    return fail(AFC_EINVAL, "team_threads %d not supported with block_threads %d", p->team_threads, B);
  if (p->slots_per_team < 0 || p->slots_per_team > kMaxSlotsPerTeam)
    return fail(AFC_EINVAL, "slots_per_team must be in [0, %d]", kMaxSlotsPerTeam);
  if (p->bucket_width > 0x7FFFFFFF) return fail(AFC_EINVAL, "bucket_width too large");
  return AFC_OK;
}

McDev to_dev(const afc_mc_problem &p, uint32_t r_begin, uint32_t *counts, afc_mc_stats *stats,
             double *dump_bc, int32_t *dump_next) {
  McDev d{};
  d.n = p.n;
  d.m = p.m;
  d.row_ptr = p.row_ptr;
  d.col = p.col;
  d.eid = p.eid;
  d.key_lo = (uint32_t)p.seed;
  d.key_hi = (uint32_t)(p.seed >> 32);
  d.graph_tag = p.graph_tag;
  d.thresh = p.thresh;
  d.thresh_all = p.thresh_all;
  d.w_lo = p.w_lo;
  d.w_hi = p.w_hi;
  d.w_lo_all = p.w_lo_all;
  d.w_hi_all = p.w_hi_all;
  d.k_min = p.k_min;
  d.in_w = p.in_w;
  d.top_k = p.top_k;
  d.tie_rel = p.tie_rel;
  d.precision = p.precision;
  d.recheck_margin = p.recheck_margin;
  d.delta = auto_delta(p);
  d.reward_k = p.reward_k;
  d.reward_gamma = p.reward_gamma;
  d.reward_pool = p.reward_pool;
  d.psi = p.psi_sum;
  d.report_rank = p.report_rank;
  d.fb_node = p.use_fallback ? (uint32_t)p.fallback_node : 0xFFFFFFFFu;
  d.fb_count = p.use_fallback ? p.fallback_count : nullptr;
  d.tie_random = p.tie_random ? 1u : 0u;
  d.wtab_ptr = p.wtab_ptr;
  d.wtab = p.wtab_ptr ? p.wtab : nullptr;
  d.per_row = p.per_row ? 1u : 0u;
  d.hop_radius = p.per_row ? p.hop_radius : 0u;
  d.r_begin = r_begin;
  d.counts = counts;
  d.stats = stats;
  d.dump_bc = dump_bc;
  d.dump_next = dump_next;
  return d;
}

// Launch plan of the shared-memory counting kernel for a set of problems: block size, source
// warps (one source slot each: as many of the CTA's warps as shared memory holds slots for,
// the other warps help with the per-realization steps only) and grid.
struct McPlan {
  int block = 1024;
  uint32_t nsw = 1, smem = 0, grid = 1;
  bool fits = true;
};

// Source slots (compact: 12 bytes per node) that fit next to the realization of an (n, arcs)
// graph within `bytes` of shared memory, with room for at least one wide slot.
uint32_t slots_within(uint32_t n, uint64_t arcs, uint32_t bytes) {
  return mc_slots_within(n, arcs, bytes);
}

// want_warps: source warps the launch should offer (0: as many as fit for the largest graph;
// a batched launch passes the most that any of its problems can use).
McPlan plan_for(const afc_mc_problem &p0, uint32_t nmax, uint64_t amax, uint64_t total_items,
                uint32_t want_warps = 0) {
  const DevInfo d = dev_info();
  McPlan pl;
  const uint32_t cap = (uint32_t)std::max(0, d.smem_optin - 1024);
  // node ids share their 16-bit settle-order entries with a step mark: below 2^15 nodes
  const uint32_t fit = nmax < 32768u ? slots_within(nmax, amax, cap) : 0u;
  if (p0.block_threads) {
    pl.block = p0.block_threads;
  } else {
    // the smallest CTA that holds a warp for every slot that fits (fewer threads per CTA leave
    // each thread more registers for the source warps' caches)
    const uint32_t want = 32u * std::min<uint32_t>(std::max(fit, want_warps), 32u);
    pl.block = want <= 256u ? 256 : want <= 512u ? 512 : 1024;
  }
  pl.nsw = std::min<uint32_t>(fit, (uint32_t)pl.block / 32u);
  pl.fits = pl.nsw >= 1;
  if (pl.fits) {
    pl.smem = mc_layout_bytes(nmax, amax, pl.nsw);
    const uint32_t smem_sm = 228u * 1024u;
    const uint32_t per_sm = std::max<uint32_t>(1u, std::min<uint32_t>(smem_sm / (pl.smem + 1024u),
                                                                      2048u / (uint32_t)pl.block));
    pl.grid = (uint32_t)std::min<uint64_t>(total_items, (uint64_t)d.sms * per_sm);
  }
  if (pl.grid == 0) pl.grid = 1;
  return pl;
}

// The global path's settle-step kernel when shared memory holds the distance arrays of at
// least this many warps (about 14,000 nodes) and steps_beat_buckets; otherwise the bucketed
// kernel.
constexpr uint32_t kMinStepWarps = 4;

// Whether the settle-step kernel outruns the bucketed one on this graph.  Its cost grows with
// the range of lengths (a wider range settles fewer nodes per step against a pending list of
// about the same length), the bucketed kernel's does not.  Measured on WS graphs of mean
// degree 8 (k = 8, beta = 0.2, survival 0.9), lengths uniform in 1..W, realizations/s of the
// settle-step kernel over the better bucketed team size: n = 2,500: W = 25 2.43x, 50 1.91x,
// 100 1.51x, 400 1.29x; n = 3,200: 2.07x, 1.59x, 1.19x, 0.98x; n = 3,818: 1.89x, 1.45x, 1.07x,
// 0.85x; n = 4,000: 1.73x, 1.31x, 0.96x, 0.75x; W = 100: n = 5,000 0.75x, 7,000 0.53x, 10,000
// 0.30x.  The ratio goes about as n^-1.17 and min(W, 200)^-0.35, which puts the crossover at
// n min(W, 200)^0.35 = 19,500 (n = 6,400 for W = 25, 5,000 for W = 50, 3,900 for W = 100,
// 3,050 for W >= 200).  Per-edge length ranges and length laws count as W = 65,535.
bool steps_beat_buckets(const afc_mc_problem &p) {
  const double w = (p.w_hi || p.wtab_ptr) ? 65535.0 : (double)std::max<uint32_t>(p.w_hi_all, 1u);
  return (double)p.n * std::pow(std::min(w, 200.0), 0.35) <= 19500.0;
}

// Launch plan of the global-memory path for one problem.
struct BigPlan {
  int block = 1024, team = 256;
  uint32_t spt = 1, grid = 1, ngroups = 1;
  uint32_t smem = 0;        // dynamic shared memory per Brandes CTA (0: control block only)
  int on_chip = 0;          // 0: slots in the arena, 1: their distances on chip, 2: whole slots
  size_t slot_stride = 0, group_bytes = 0;
  size_t off_groups = 0, off_garr = 0, off_arena = 0, total = 0;   // relative to its base
};

BigPlan plan_big(const afc_mc_problem &p, uint64_t r_count) {
  const DevInfo d = dev_info();
  BigPlan b;
  const uint32_t n = (uint32_t)p.n;
  const uint64_t arcs = 2ull * (uint64_t)p.m;
  const uint32_t per_warp = (4u * n + 15u) & ~15u;   // one distance array
  const uint32_t fit = (uint32_t)std::max(0, d.smem_optin - 1024) / per_warp;
  if (p.team_threads == 0 && fit >= kMinStepWarps && steps_beat_buckets(p)) {
    // settle-step kernel: one source per warp, its distances on chip (16 warps per CTA at most:
    // 1024-thread CTAs would cap the registers below what the routine needs)
    b.team = 0;
    b.block = p.block_threads ? std::min(p.block_threads, 512) : 512;
    b.spt = std::min<uint32_t>(fit, (uint32_t)b.block / 32u);
    b.on_chip = 1;
    if (!p.block_threads && b.spt <= 8) b.block = 256;
    b.smem = b.on_chip ? b.spt * per_warp : 0u;
    b.slot_stride = big_step_slot_bytes(n, !b.on_chip);
    const uint32_t per_sm = std::max<uint32_t>(
        1u, std::min<uint32_t>(2048u / (uint32_t)b.block, (228u * 1024u) / (b.smem + 1024u)));
    b.grid = (uint32_t)std::max(1, d.sms) * per_sm;
    // realizations in flight: enough for about 64 sources per warp of the grid (at most 128),
    // since warps that run out of sources idle until the batch ends; measured on the mix's
    // 2,306 / 3,164 / 3,818-node graphs (realizations/s): about 4 sources per warp 863 / 394 /
    // 252, 8: 894 / 423 / 271, 16: 928 / 439 / 282, 32: 947 / 448 / 289, 64: 954 / 452 / 293,
    // 128 (at most 256 groups): 960 / 456 / 294
    const uint64_t want = ((uint64_t)64 * b.grid * b.spt + n - 1) / n;
    b.ngroups = (uint32_t)std::max<uint64_t>(
        1, std::min<uint64_t>({std::max<uint64_t>(want, 2), 128, std::max<uint64_t>(r_count, 1)}));
    b.group_bytes = big_group_bytes(n, arcs);
    size_t o = 0;
    b.off_groups = o; o += (sizeof(BigGroup) * b.ngroups + 255) & ~size_t(255);
    b.off_garr = o;   o += b.group_bytes * b.ngroups;
    b.off_arena = o;  o += b.slot_stride * (size_t)b.grid * b.spt;
    b.total = o;
    return b;
  }
  b.block = p.block_threads ? p.block_threads : 1024;
  b.slot_stride = big_slot_bytes(n);
  if (p.team_threads) {
    b.team = p.team_threads;
  } else {
    // measured on ER and WS graphs of mean degree 8 (n = 1,000 .. 10,000) and on the
    // 20,000-node workload: up to about 4,000 nodes, teams of 128 threads (8 sources in flight
    // per CTA), except where only four whole slots fit in shared memory: then four teams of 256
    // with their slots on chip (+7% at n = 1,800, +10-14% at n = 3,200 over teams of 128 with
    // only their distances on chip); teams of 128 up to 6,000 nodes (realizations/s, 128 / 256
    // threads: n = 4,600 156 / 143, n = 5,000 132 / 124); then teams of 256 while four distance
    // arrays fit on chip (n = 7,000: 67 against 58 with 128 and 58 with 512; n = 10,000: 36
    // against 28 and 30); beyond, teams of 512 whose two slots keep at least their distance
    // arrays in shared memory (7.1 realizations/s on the 20,000-node workload, against 6.2 with
    // four teams of 256 and distances in device memory), or 256 when two such arrays do not fit
    if (n <= 4096) {
      const bool eight = (int)big_slots_smem_bytes(n, 8u) + 1024 <= d.smem_optin;
      const bool four = (int)big_slots_smem_bytes(n, 4u) + 1024 <= d.smem_optin;
      b.team = (b.block == 1024 && !eight && four) ? 256 : 128;
    } else if (n <= 6000) {
      b.team = 128;
    } else {
      const bool four_fit = (int)big_dist_smem_bytes(n, 4u) + 1024 <= d.smem_optin;
      const bool two_fit = (int)big_dist_smem_bytes(n, 2u) + 1024 <= d.smem_optin;
      b.team = (b.block >= 1024 && !four_fit && two_fit) ? 512 : 256;
    }
    b.team = std::min(b.block, b.team);
    if (!big_config_supported(b.block, b.team)) b.team = b.block;
  }
  const uint32_t nt = (uint32_t)(b.block / b.team);
  b.spt = p.slots_per_team ? (uint32_t)p.slots_per_team : 1u;
  b.spt = std::min<uint32_t>(b.spt, std::max<uint32_t>(1u, (uint32_t)kMaxSlots / nt));
  // the CTA's source slots in shared memory when they fit, else their distance arrays (every
  // arc reads them and the relaxations update them atomically: on chip instead of L2 round
  // trips), else nothing
  const uint32_t whole = big_slots_smem_bytes(n, nt * b.spt);
  const uint32_t ds = big_dist_smem_bytes(n, nt * b.spt);
  if ((int)whole + 1024 <= d.smem_optin) {
    b.smem = whole;
    b.on_chip = 2;
  } else if ((int)ds + 1024 <= d.smem_optin) {
    b.smem = ds;
    b.on_chip = 1;
  }
  const uint32_t smem_cta = b.on_chip ? b.smem : (uint32_t)sizeof(CtaCtl);
  const uint32_t per_sm = std::max<uint32_t>(
      1u, std::min<uint32_t>((uint32_t)std::max(1, 1024 / b.block), (228u * 1024u) / (smem_cta + 1024u)));
  b.grid = (uint32_t)std::max(1, d.sms) * per_sm;
  // realizations in flight: about 64 sources for every team (at most 64 realizations), since
  // teams that run out of sources idle until the batch ends; measured with lengths 1..100
  // (realizations/s, about 4 / 16 / 64 sources per team): n = 5,000 131 / 141 / 148, n = 7,000
  // 67 / 67 / 69, n = 10,000 35.9 / 35.9 / 36.6
  const uint64_t want = ((uint64_t)64 * b.grid * nt * b.spt + n - 1) / n;
  b.ngroups = (uint32_t)std::max<uint64_t>(1, std::min<uint64_t>({std::max<uint64_t>(want, 2), 64,
                                                                   std::max<uint64_t>(r_count, 1)}));
  b.group_bytes = big_group_bytes(n, arcs);
  size_t o = 0;
  b.off_groups = o; o += (sizeof(BigGroup) * b.ngroups + 255) & ~size_t(255);
  b.off_garr = o;   o += b.group_bytes * b.ngroups;
  b.off_arena = o;  o += b.on_chip == 2 ? 0 : b.slot_stride * (size_t)b.grid * nt * b.spt;
  b.total = o;
  return b;
}

// Items of a counting call: r_count realizations, or in the row-wise mode r_count draws for
// each of the n rows (one item per draw and row).
uint64_t items_of(const afc_mc_problem &p, uint32_t r_count) {
  return p.per_row ? (uint64_t)r_count * (uint64_t)p.n : (uint64_t)r_count;
}

bool smem_fits(const afc_mc_problem &p) {
  return plan_for(p, (uint32_t)p.n, 2ull * (uint64_t)p.m, 1).fits;
}

// AFC_PATH_AUTO: the shared-memory path when shared memory holds at least this many compact
// source slots.  Measured on mix graphs (mean degree 8, FP64): with 7 slots (1,771 nodes) it
// is 7% faster than the global path's settle-step kernel, with 6 slots (2,014 nodes) 3%
// faster, with 5 slots (2,161-2,340 nodes) 7-8% slower.
constexpr uint32_t kMinSharedSlots = 6;

bool wants_global(const afc_mc_problem &p) {
  if (p.memory_path == AFC_PATH_GLOBAL) return true;
  if (p.memory_path == AFC_PATH_SHARED) return false;
  const McPlan pl = plan_for(p, (uint32_t)p.n, 2ull * (uint64_t)p.m, 1);
  return !pl.fits || pl.nsw < kMinSharedSlots;
}

size_t meta_bytes(int nprob) {
  return ((sizeof(McDev) * (size_t)nprob + sizeof(uint64_t) * (size_t)(nprob + 1)) + 255) &
         ~size_t(255);
}

// The shared-memory problems of a call, in launch order, and their launch: one persistent
// kernel sized for the largest graph, each CTA with its region of device scratch.
struct SharedBatch {
  std::vector<int> order;
  uint32_t nmax = 1;
  uint64_t amax = 1, items = 0;
  uint32_t want_warps = 0;
  McPlan pl;
  size_t scratch_stride = 0, scratch_bytes = 0;
};

SharedBatch shared_batch(int nprob, const afc_mc_problem *probs, const uint32_t *r_count) {
  SharedBatch sb;
  for (int g = 0; g < nprob; ++g)
    if (!wants_global(probs[g])) sb.order.push_back(g);
  if (sb.order.empty()) return sb;
  const DevInfo di = dev_info();
  const uint32_t cap = (uint32_t)std::max(0, di.smem_optin - 1024);
  for (int g : sb.order) {
    const afc_mc_problem &p = probs[g];
    sb.nmax = std::max<uint32_t>(sb.nmax, (uint32_t)p.n);
    sb.amax = std::max<uint64_t>(sb.amax, 2ull * (uint64_t)p.m);
    // no count given: size for a launch that fills the GPU
    sb.items += r_count ? items_of(p, r_count[g]) : (uint64_t)1 << 40;
    if (sb.order.size() > 1)
      sb.want_warps = std::max(sb.want_warps, slots_within((uint32_t)p.n, 2ull * (uint64_t)p.m, cap));
  }
  sb.pl = plan_for(probs[sb.order[0]], sb.nmax, sb.amax, std::max<uint64_t>(sb.items, 1),
                   sb.want_warps);
  sb.scratch_stride = (mc_cta_scratch_bytes(sb.nmax) + 255) & ~size_t(255);
  sb.scratch_bytes = sb.pl.fits ? sb.scratch_stride * sb.pl.grid : 0;
  return sb;
}

// Workspace: [McDev x nprob][item prefix of the shared-path problems], the shared path's CTA
// scratch, then the global path's groups, group arrays and slot arena (reused by the
// global-path problems one after another).
size_t counts_ws_total(int nprob, const afc_mc_problem *probs, const uint32_t *r_count) {
  size_t big = 0;
  for (int g = 0; g < nprob; ++g)
    if (wants_global(probs[g]))
      big = std::max(big, plan_big(probs[g], r_count ? items_of(probs[g], r_count[g]) : 1u << 20).total);
  return meta_bytes(nprob) + shared_batch(nprob, probs, r_count).scratch_bytes + big;
}

int run_counts(int nprob, const afc_mc_problem *probs, const uint32_t *r_begin,
               const uint32_t *r_count, uint32_t *const *counts, afc_mc_stats *const *stats,
               double *dump_bc, int32_t *dump_next, void *workspace, size_t ws_bytes,
               cudaStream_t stream) {
  for (int g = 0; g < nprob; ++g) {
    int st = validate(&probs[g]);
    if (st) return st;
    if (!counts[g]) return fail(AFC_EINVAL, "counts[%d] is null", g);
    if (probs[g].memory_path == AFC_PATH_SHARED && !smem_fits(probs[g]))
      return fail(AFC_EUNSUPPORTED, "problem %d does not fit the shared-memory counting path", g);
    if (probs[g].per_row) {
      const uint64_t rb = r_begin ? r_begin[g] : 0u;
      if ((rb + r_count[g]) * (uint64_t)probs[g].n > 0xFFFFFFFFull)
        return fail(AFC_EUNSUPPORTED, "row-wise mode: (r_begin + r_count) x n must stay below 2^32");
      if (dump_bc || dump_next)
        return fail(AFC_EINVAL, "the row-wise mode writes no per-realization dumps");
    }
  }
  // problems on the shared-memory path first (one persistent launch), then the others
  const SharedBatch sb = shared_batch(nprob, probs, r_count);
  std::vector<int> order = sb.order, big;
  for (int g = 0; g < nprob; ++g)
    if (wants_global(probs[g])) big.push_back(g);
  const int ns = (int)order.size();
  for (int g : order)
    if (auto_block(probs[g]) != auto_block(probs[order[0]]))
      return fail(AFC_EINVAL, "all shared-path problems of a batch must use the same block_threads");
  order.insert(order.end(), big.begin(), big.end());
  std::vector<McDev> devs(nprob);
  std::vector<uint64_t> prefix(ns + 1, 0);
  for (int k = 0; k < nprob; ++k) {
    const int g = order[k];
    devs[k] = to_dev(probs[g], r_begin ? r_begin[g] : 0u, counts[g], stats ? stats[g] : nullptr,
                     nprob == 1 ? dump_bc : nullptr, nprob == 1 ? dump_next : nullptr);
    if (k < ns) prefix[k + 1] = prefix[k] + items_of(probs[g], r_count[g]);
  }
  const size_t need = counts_ws_total(nprob, probs, r_count);
  if (!workspace || ws_bytes < need)
    return fail(AFC_ENOMEM, "workspace of %zu bytes given, %zu needed", ws_bytes, need);
  unsigned char *ws = static_cast<unsigned char *>(workspace);
  McDev *devs_d = reinterpret_cast<McDev *>(ws);
  uint64_t *prefix_d = reinterpret_cast<uint64_t *>(ws + sizeof(McDev) * (size_t)nprob);
  AFC_CUDA(cudaMemcpyAsync(devs_d, devs.data(), sizeof(McDev) * (size_t)nprob, cudaMemcpyHostToDevice, stream));
  AFC_CUDA(cudaMemcpyAsync(prefix_d, prefix.data(), sizeof(uint64_t) * (size_t)(ns + 1), cudaMemcpyHostToDevice, stream));
  if (ns > 0 && prefix[ns] > 0) {
    const McPlan &pl = sb.pl;
    if (!pl.fits)
      return fail(AFC_EUNSUPPORTED, "batch too large for the shared-memory counting kernel");
    if (ns > 1) {
      // every problem of a batched launch takes as many source warps as the launch's shared
      // memory holds slots for at its own size (the launch is sized for the largest graph)
      for (int k = 0; k < ns; ++k) {
        const afc_mc_problem &p = probs[order[k]];
        const uint32_t fit = slots_within((uint32_t)p.n, 2ull * (uint64_t)p.m, pl.smem);
        devs[k].spt = std::max<uint32_t>(1u, std::min<uint32_t>(fit, (uint32_t)pl.block / 32u));
      }
      AFC_CUDA(cudaMemcpyAsync(devs_d, devs.data(), sizeof(McDev) * (size_t)ns, cudaMemcpyHostToDevice, stream));
    }
    // the shared batch's grid was sized for all its items: the launch may use fewer CTAs
    const uint32_t grid = (uint32_t)std::min<uint64_t>(pl.grid, prefix[ns]);
    cudaError_t e = launch_mc_counts(pl.block, devs_d, ns, prefix_d, prefix[ns], pl.nsw, pl.smem,
                                     std::max<uint32_t>(grid, 1u), ws + meta_bytes(nprob),
                                     sb.scratch_stride, stream);
    if (e != cudaSuccess) return cuda_fail(e, "counting kernel launch");
  }
  unsigned char *bigbase = ws + meta_bytes(nprob) + sb.scratch_bytes;
  for (int k = ns; k < nprob; ++k) {
    const afc_mc_problem &p = probs[order[k]];
    const uint32_t rc = (uint32_t)items_of(p, r_count[order[k]]);
    if (rc == 0) continue;
    const BigPlan b = plan_big(p, rc);
    std::vector<BigGroup> groups(b.ngroups);
    for (uint32_t i = 0; i < b.ngroups; ++i)
      big_group_carve(groups[i], bigbase + b.off_garr + b.group_bytes * i, (uint32_t)p.n,
                      2ull * (uint64_t)p.m);
    BigGroup *groups_d = reinterpret_cast<BigGroup *>(bigbase + b.off_groups);
    AFC_CUDA(cudaMemcpyAsync(groups_d, groups.data(), sizeof(BigGroup) * b.ngroups,
                             cudaMemcpyHostToDevice, stream));
    cudaError_t e = launch_mc_global(b.block, b.team, devs_d + k, p.precision, groups_d, b.ngroups,
                                     rc, bigbase + b.off_arena, b.slot_stride, b.spt, b.smem, b.on_chip,
                                     b.grid, stream);
    if (e != cudaSuccess) return cuda_fail(e, "global-path counting launch");
  }
  return AFC_OK;
}

}  // namespace

namespace afc {

int report_error(int code, const char *msg) { return fail(code, "%s", msg); }

int counts_ranges(int nprob, const afc_mc_problem *probs, const uint32_t *r_begin,
                  const uint32_t *r_count, uint32_t *const *counts, afc_mc_stats *const *stats,
                  void *workspace, size_t ws_bytes, cudaStream_t stream) {
  if (nprob <= 0 || !probs || !r_count || !counts) return fail(AFC_EINVAL, "bad batch arguments");
  return run_counts(nprob, probs, r_begin, r_count, counts, stats, nullptr, nullptr, workspace,
                    ws_bytes, stream);
}

size_t counts_ranges_workspace(int nprob, const afc_mc_problem *probs, const uint32_t *r_count) {
  return counts_ws_total(nprob, probs, r_count);
}

}  // namespace afc

extern "C" {

const char *afc_last_error(void) { return abi_error_text().c_str(); }

int afc_version(void) { return 10000; }

int afc_csr_from_edges(int32_t n, int64_t m, const int32_t *eu, const int32_t *ev, int32_t *row_ptr,
                       int32_t *col, int32_t *eid) {
  return guarded("afc_csr_from_edges", [&]() -> int {
    if (n < 0 || m < 0 || !row_ptr || (m > 0 && (!eu || !ev || !col || !eid)))
      return fail(AFC_EINVAL, "bad arguments");
    if (2 * m > 0x7FFFFFFF) return fail(AFC_EUNSUPPORTED, "too many edges");
    for (int64_t e = 0; e < m; ++e)
      if (eu[e] < 0 || eu[e] >= n || ev[e] < 0 || ev[e] >= n || eu[e] == ev[e])
        return fail(AFC_EINVAL, "edge %lld = (%d, %d) invalid", (long long)e, eu[e], ev[e]);
    std::vector<int32_t> deg((size_t)n + 1, 0);
    for (int64_t e = 0; e < m; ++e) { deg[eu[e]]++; deg[ev[e]]++; }
    row_ptr[0] = 0;
    for (int32_t v = 0; v < n; ++v) row_ptr[v + 1] = row_ptr[v] + deg[v];
    std::vector<int32_t> fill(row_ptr, row_ptr + n);
    for (int64_t e = 0; e < m; ++e) {
      const int32_t a = eu[e], b = ev[e];
      col[fill[a]] = b; eid[fill[a]++] = (int32_t)e;
      col[fill[b]] = a; eid[fill[b]++] = (int32_t)e;
    }
    std::vector<std::pair<int32_t, int32_t>> row;
    for (int32_t v = 0; v < n; ++v) {
      row.clear();
      for (int32_t a = row_ptr[v]; a < row_ptr[v + 1]; ++a) row.emplace_back(col[a], eid[a]);
      std::sort(row.begin(), row.end());
      for (size_t k = 0; k < row.size(); ++k) {
        if (k > 0 && row[k].first == row[k - 1].first)
          return fail(AFC_EINVAL, "duplicate edge (%d, %d)", v, row[k].first);
        col[row_ptr[v] + k] = row[k].first;
        eid[row_ptr[v] + k] = row[k].second;
      }
    }
    return AFC_OK;
  });
}

uint64_t afc_survival_threshold(double p) {
  if (!(p > 0.0)) return 0;
  if (p >= 1.0) return 1ull << 32;
  return (uint64_t)std::floor(p * 4294967296.0);
}

int afc_counts_path(const afc_mc_problem *prob) {
  const int st = validate(prob);
  if (st) return -st;
  return wants_global(*prob) ? AFC_PATH_GLOBAL : AFC_PATH_SHARED;
}

size_t afc_transition_counts_workspace(const afc_mc_problem *prob) {
  if (validate(prob)) return 0;
  return counts_ws_total(1, prob, nullptr);
}

int afc_transition_counts(const afc_mc_problem *prob, uint32_t r_begin, uint32_t r_count,
                          uint32_t *counts, afc_mc_stats *stats, double *dump_bc,
                          int32_t *dump_next, void *workspace, size_t workspace_bytes,
                          void *stream) {
  NvtxRange nvtx_range("afc.transition_counts");
  if (!prob) return fail(AFC_EINVAL, "null problem");
  uint32_t *cs[1] = {counts};
  afc_mc_stats *sl[1] = {stats};
  return run_counts(1, prob, &r_begin, &r_count, cs, stats ? sl : nullptr, dump_bc, dump_next,
                    workspace, workspace_bytes, (cudaStream_t)stream);
}

size_t afc_transition_counts_batched_workspace(int32_t nprob, const afc_mc_problem *probs,
                                               const uint32_t *r_count) {
  if (nprob <= 0 || !probs || !r_count) return 0;
  for (int g = 0; g < nprob; ++g)
    if (validate(&probs[g])) return 0;
  uint64_t total = 0;
  for (int g = 0; g < nprob; ++g) total += r_count[g];
  (void)total;
  return counts_ws_total(nprob, probs, r_count);
}

int afc_transition_counts_batched(int32_t nprob, const afc_mc_problem *probs,
                                  const uint32_t *r_count, uint32_t *const *counts,
                                  afc_mc_stats *stats, void *workspace, size_t workspace_bytes,
                                  void *stream) {
  NvtxRange nvtx_range("afc.transition_counts_batched");
  if (nprob <= 0 || !probs || !r_count || !counts) return fail(AFC_EINVAL, "bad batch arguments");
  std::vector<afc_mc_stats *> sl;
  if (stats)
    for (int g = 0; g < nprob; ++g) sl.push_back(stats + g);
  return run_counts(nprob, probs, nullptr, r_count, counts, stats ? sl.data() : nullptr, nullptr,
                    nullptr, workspace, workspace_bytes, (cudaStream_t)stream);
}

int afc_autotune(afc_mc_problem *prob, uint32_t r_begin, uint32_t sample, void *stream,
                 afc_tune_result *out) {
  NvtxRange nvtx_range("afc.autotune");
  int st = validate(prob);
  if (st) return st;
  cudaStream_t s = (cudaStream_t)stream;
  const DevInfo d = dev_info();
  const afc_mc_problem base = *prob;
  const bool global = wants_global(base);
  if (sample == 0)
    sample = (uint32_t)std::min<uint64_t>(2ull * d.sms,
                                          std::max<uint64_t>(2, (2000ull * d.sms + base.n - 1) / base.n));
  // bucket widths: the power of two the kernels would use for the automatic request, half and
  // double (the kernels raise a width below ceil(wmax / 14) to that bound; those duplicates go)
  const uint32_t wmax = base.w_hi ? 0u : (uint32_t)base.w_hi_all;
  const uint32_t dmin = wmax ? (wmax + (kRing - 2) - 1) / (kRing - 2) : 1u;
  auto eff = [&](uint32_t w) {
    const uint32_t want = std::max(std::max(w, 1u), dmin);
    uint32_t p2 = 1;
    while (p2 < want && p2 < (1u << 30)) p2 <<= 1;
    return p2;
  };
  const uint32_t w0 = eff(auto_delta(base));
  std::vector<uint32_t> widths;
  for (uint32_t w : {w0, w0 > 1 ? w0 / 2 : 1u, w0 * 2})
    if (std::find(widths.begin(), widths.end(), eff(w)) == widths.end()) widths.push_back(eff(w));
  // shared-memory path: the CTA size (its warps are the source warps where slots fit; bucket
  // widths do not apply); global path: (block, team) pairs and bucket widths
  static const int kShared[] = {1024, 512, 256};
  static const std::pair<int, int> kGlobal[] = {{1024, 128}, {1024, 256}, {1024, 512}};
  // the automatic configuration first (it is also the warm-up), then the grid; a problem on
  // AFC_PATH_AUTO whose state fits in shared memory also tries the global-memory path
  std::vector<afc_mc_problem> cands;
  cands.push_back(base);
  cands.back().bucket_width = w0;
  auto add = [&](int path, int block, int team, uint32_t w) {
    afc_mc_problem c = base;
    c.block_threads = block;
    c.team_threads = team;
    c.bucket_width = w;
    c.memory_path = path;
    if (validate(&c) != AFC_OK) return;
    if (path == AFC_PATH_SHARED && !smem_fits(c)) return;
    cands.push_back(c);
  };
  if (!global)
    for (int blk : kShared) add(AFC_PATH_SHARED, blk, 0, w0);
  for (uint32_t w : widths)
    if (global || base.memory_path == AFC_PATH_AUTO)
      for (const auto &sh : kGlobal) add(AFC_PATH_GLOBAL, sh.first, sh.second, w);
  abi_error_text().clear();
  size_t ws = 0;
  for (const auto &c : cands) ws = std::max(ws, counts_ws_total(1, &c, &sample));
  const size_t counts_bytes = sizeof(uint32_t) * (size_t)base.n * (size_t)(base.n + 1);
  const size_t psi_bytes = base.reward_k ? sizeof(double) * (size_t)base.n : 0;
  const size_t off_psi = (counts_bytes + 255) & ~size_t(255);
  const size_t off_ws = off_psi + ((psi_bytes + 255) & ~size_t(255));
  void *buf = nullptr;
  AFC_CUDA(cudaMallocAsync(&buf, off_ws + ws, s));
  unsigned char *b = static_cast<unsigned char *>(buf);
  uint32_t *counts = reinterpret_cast<uint32_t *>(b);
  double *psi = psi_bytes ? reinterpret_cast<double *>(b + off_psi) : nullptr;
  void *wsp = b + off_ws;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  double best_t = 0.0, default_t = 0.0;
  size_t best = 0;
  int timed = 0;
  for (size_t k = 0; k < cands.size() + 1 && st == AFC_OK; ++k) {
    // k = 0 warms up with the automatic configuration; k >= 1 times candidate k - 1
    afc_mc_problem c = cands[k == 0 ? 0 : k - 1];
    if (psi) c.psi_sum = psi;   // the caller's accumulators are never touched
    c.fallback_count = nullptr;
    uint32_t *cs[1] = {counts};
    cudaEventRecord(e0, s);
    st = run_counts(1, &c, &r_begin, &sample, cs, nullptr, nullptr, nullptr, wsp, ws, s);
    cudaEventRecord(e1, s);
    if (st != AFC_OK) break;
    cudaError_t e = cudaEventSynchronize(e1);
    if (e != cudaSuccess) { st = cuda_fail(e, "autotune launch"); break; }
    if (k == 0) continue;
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    ++timed;
    if (k == 1) default_t = ms;
    if (k == 1 || ms < best_t) { best_t = ms; best = k - 1; }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFreeAsync(buf, s);
  cudaError_t e = cudaStreamSynchronize(s);
  if (st != AFC_OK) return st;
  if (e != cudaSuccess) return cuda_fail(e, "autotune");
  const afc_mc_problem &w = cands[best];
  if (best == 0) {
    // the automatic configuration won: pin what it resolves to
    if (global) {
      const BigPlan bp = plan_big(base, sample);
      prob->block_threads = bp.block;
      prob->team_threads = bp.team;
    } else {
      const McPlan pl = plan_for(base, (uint32_t)base.n, 2ull * (uint64_t)base.m, sample);
      prob->block_threads = pl.block;
    }
  } else {
    prob->block_threads = w.block_threads;
    prob->team_threads = w.team_threads;
    if (base.memory_path == AFC_PATH_AUTO) prob->memory_path = w.memory_path;
  }
  prob->bucket_width = w.bucket_width;
  if (out) {
    out->block_threads = prob->block_threads;
    out->team_threads = prob->team_threads;
    out->bucket_width = prob->bucket_width;
    out->realizations_per_s = best_t > 0 ? 1e3 * sample / best_t : 0.0;
    out->default_per_s = default_t > 0 ? 1e3 * sample / default_t : 0.0;
    out->candidates = timed;
  }
  return AFC_OK;
}

int afc_debug_realize(const afc_mc_problem *prob, uint32_t r_begin, uint32_t r_count, uint8_t *alive,
                      uint32_t *w, void *stream) {
  int st = validate(prob);
  if (st) return st;
  if (!alive || !w) return fail(AFC_EINVAL, "null output");
  McDev d = to_dev(*prob, r_begin, nullptr, nullptr, nullptr, nullptr);
  cudaError_t e = launch_debug_realize(d, r_count, alive, w, (cudaStream_t)stream);
  return e == cudaSuccess ? AFC_OK : cuda_fail(e, "debug_realize");
}

int afc_debug_components(const afc_mc_problem *prob, uint32_t r_begin, uint32_t r_count,
                         int32_t *comp, int32_t *csize, void *stream) {
  int st = validate(prob);
  if (st) return st;
  if (!comp || !csize) return fail(AFC_EINVAL, "null output");
  const DevInfo di = dev_info();
  if ((int)mc_layout_bytes(prob->n, 2 * prob->m, 0) > di.smem_optin)
    return fail(AFC_EUNSUPPORTED, "graph too large for the shared-memory component kernel");
  if (r_count == 0) return AFC_OK;
  McDev d = to_dev(*prob, r_begin, nullptr, nullptr, nullptr, nullptr);
  cudaError_t e = launch_debug_components(d, r_count, comp, csize, (cudaStream_t)stream);
  return e == cudaSuccess ? AFC_OK : cuda_fail(e, "debug_components");
}

int afc_debug_sssp(const afc_mc_problem *prob, uint32_t r, const int32_t *sources, int32_t nsrc,
                   uint32_t *dist, uint64_t *sigma, afc_mc_stats *stats, void *stream) {
  int st = validate(prob);
  if (st) return st;
  if (nsrc < 0 || (nsrc > 0 && (!sources || !dist || !sigma))) return fail(AFC_EINVAL, "bad outputs");
  if (nsrc == 0) return AFC_OK;
  const McPlan pl = plan_for(*prob, (uint32_t)prob->n, 2ull * (uint64_t)prob->m, (uint64_t)nsrc);
  if (!pl.fits) return fail(AFC_EUNSUPPORTED, "graph too large for the shared-memory SSSP kernel");
  McDev d = to_dev(*prob, 0, nullptr, stats, nullptr, nullptr);
  cudaError_t e = launch_debug_sssp(pl.block, d, r, sources, nsrc, pl.nsw, pl.smem, dist, sigma,
                                    (cudaStream_t)stream);
  return e == cudaSuccess ? AFC_OK : cuda_fail(e, "debug_sssp");
}

// ---- A8 / A9 ---------------------------------------------------------------------------------

int afc_observed_states(int32_t n, const uint32_t *counts, int32_t *c_index, int32_t *c_list,
                        int32_t *c_host, void *stream) {
  NvtxRange nvtx_range("afc.observed_states");
  if (n < 1 || !counts || !c_index || !c_list || !c_host) return fail(AFC_EINVAL, "bad arguments");
  cudaStream_t s = (cudaStream_t)stream;
  int32_t *c_dev = nullptr;
  AFC_CUDA(cudaMallocAsync(&c_dev, sizeof(int32_t), s));
  cudaError_t e = launch_observed_states(n, counts, c_index, c_list, c_dev, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(c_host, c_dev, sizeof(int32_t), cudaMemcpyDeviceToHost, s);
  cudaFreeAsync(c_dev, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  return e == cudaSuccess ? AFC_OK : cuda_fail(e, "observed_states");
}

// Perturbation slabs (one per resident perturbation CTA): two per SM while they take at most
// 8 GB together, else one per SM.
static uint32_t perturb_slabs(const DevInfo &d, size_t slab) {
  const uint32_t sms = (uint32_t)std::max(1, d.sms);
  return (size_t)2 * sms * slab <= (8ull << 30) ? 2 * sms : sms;
}

static SolveWs ws_layout_for(int32_t n, int32_t c) {
  const DevInfo d = dev_info();
  // nonzeros of the kernel: at most the transient columns in C plus the absorbing column
  const size_t nnz_cap = (size_t)n * ((size_t)std::min<int32_t>(c, n) + 1);
  const size_t slab = std::max<size_t>(perturb_slab_bytes(n, c) + nnz_cap * 8, 8 * (size_t)(c + 1) * 64 / (size_t)std::max(1, d.sms) + 256);
  // the large-c sweep's column-wise pattern of Q_CC (at most c entries per column)
  const size_t csc = perturb_on_chip(c, d.smem_optin) ? 0 : (size_t)c * (size_t)c;
  return solve_ws_layout(n, c, nnz_cap, perturb_slabs(d, slab), slab, csc);
}

static size_t solve_ws_bytes(int32_t n, int32_t c) { return ws_layout_for(n, c).total; }

size_t afc_solve_workspace(int32_t n, int32_t c) {
  if (n < 1 || c < 0 || c > n) return 0;
  return solve_ws_bytes(n, c);
}

static int chain_checks(const afc_chain *ch, const uint32_t *counts, const int32_t *c_index,
                        const int32_t *c_list, int32_t c) {
  if (!ch || !counts || !c_index || !c_list) return fail(AFC_EINVAL, "null argument");
  if (const int st = chain_params_check(ch)) return st;
  if (c < 0 || c > ch->n) return fail(AFC_EINVAL, "bad n or c");
  return AFC_OK;
}

static ChainDev chain_dev(const afc_chain *ch, const uint32_t *counts, const int32_t *c_index,
                          const int32_t *c_list, int32_t c) {
  ChainDev C{};
  C.n = ch->n;
  C.R = ch->realizations;
  C.alpha = ch->alpha;
  C.eta = ch->absorb_floor;
  C.s = ch->s_init;
  C.f = ch->reward;
  C.counts = counts;
  C.c_index = c_index;
  C.c_list = c_list;
  C.c = c;
  return C;
}

int afc_absorbing_solve(const afc_chain *chain, const uint32_t *counts, const int32_t *c_index,
                        const int32_t *c_list, int32_t c, double *mu, double *b, double *scalars,
                        double *lu, int32_t *piv, void *workspace, size_t workspace_bytes,
                        void *stream) {
  NvtxRange nvtx_range("afc.absorbing_solve");
  int st = chain_checks(chain, counts, c_index, c_list, c);
  if (st) return st;
  if (!mu || !b || !scalars || (c > 0 && (!lu || !piv))) return fail(AFC_EINVAL, "null output");
  const SolveWs L = ws_layout_for(chain->n, c);
  if (!workspace || workspace_bytes < L.total)
    return fail(AFC_ENOMEM, "workspace of %zu bytes given, %zu needed", workspace_bytes, L.total);
  cudaStream_t s = (cudaStream_t)stream;
  unsigned char *ws = static_cast<unsigned char *>(workspace);
  uint32_t *status = reinterpret_cast<uint32_t *>(ws + L.off_tmp + 256);
  AFC_CUDA(cudaMemsetAsync(status, 0, sizeof(uint32_t), s));
  ChainDev C = chain_dev(chain, counts, c_index, c_list, c);
  cudaError_t e = launch_solve(C, mu, b, scalars, lu, piv, ws, L, status, s);
  if (e != cudaSuccess) return cuda_fail(e, "solve launch");
  uint32_t st_host = 0;
  AFC_CUDA(cudaMemcpyAsync(&st_host, status, sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
  AFC_CUDA(cudaStreamSynchronize(s));
  if (st_host & kErrSolve) return fail(AFC_ESINGULAR, "zero pivot in the LU of I - Q_CC");
  return AFC_OK;
}

int afc_perturb_sweep(const afc_chain *chain, const afc_perturb_params *pp, const uint32_t *counts,
                      const int32_t *c_index, const int32_t *c_list, int32_t c, const double *mu0,
                      const double *b0, const double *lu0, const int32_t *piv0, uint64_t *counters,
                      uint64_t *pair_flips, uint64_t *shift_hist, double *maxima, double *b_out,
                      void *workspace, size_t workspace_bytes, void *stream) {
  NvtxRange nvtx_range("afc.perturb_sweep");
  int st = chain_checks(chain, counts, c_index, c_list, c);
  if (st) return st;
  if (!pp || !mu0 || !b0 || (c > 0 && (!lu0 || !piv0)) || !counters || !pair_flips || !shift_hist || !maxima)
    return fail(AFC_EINVAL, "null argument");
  if (pp->k2 < 1 || pp->k2 > 32 || pp->top_k < 1 || pp->top_k > pp->k2 || pp->hist_bins < 1 || pp->hist_bins > 64)
    return fail(AFC_EINVAL, "need 1 <= top_k <= k2 <= 32 and 1 <= hist_bins <= 64");
  if (!(pp->l1_radius >= 0.0) || !(pp->r_min >= 0.0 && pp->r_min < 1.0) || !(pp->tie_rel >= 0.0))
    return fail(AFC_EINVAL, "bad perturbation parameters");
  if ((pp->model != 0 && pp->model != 1) || (pp->model == 1 && !(pp->rel_radius >= 0.0)))
    return fail(AFC_EINVAL, "model must be 0 (l1) or 1 (multiplicative, rel_radius >= 0)");
  const SolveWs L = ws_layout_for(chain->n, c);
  if (!workspace || workspace_bytes < L.total)
    return fail(AFC_ENOMEM, "workspace of %zu bytes given, %zu needed", workspace_bytes, L.total);
  cudaStream_t s = (cudaStream_t)stream;
  unsigned char *ws = static_cast<unsigned char *>(workspace);
  uint32_t *status = reinterpret_cast<uint32_t *>(ws + L.off_tmp + 256);
  AFC_CUDA(cudaMemsetAsync(status, 0, sizeof(uint32_t), s));
  ChainDev C = chain_dev(chain, counts, c_index, c_list, c);
  const DevInfo d = dev_info();
  cudaError_t e = launch_perturb(C, *pp, mu0, b0, lu0, piv0, counters, pair_flips, shift_hist, maxima,
                                 b_out, ws, L, status, d.sms, s);
  if (e != cudaSuccess) return cuda_fail(e, "perturb launch");
  return AFC_OK;
}

int afc_certificates(const afc_chain *chain, const uint32_t *counts, const int32_t *c_index,
                     const int32_t *c_list, int32_t c, const double *mu0, const double *lu0,
                     const int32_t *piv0, double eps_bar, double r_min, int32_t npairs,
                     const int32_t *pu, const int32_t *pv, double *gap, double *sharp,
                     void *workspace, size_t workspace_bytes, void *stream) {
  NvtxRange nvtx_range("afc.certificates");
  int st = chain_checks(chain, counts, c_index, c_list, c);
  if (st) return st;
  if (npairs < 0 || (npairs > 0 && (!pu || !pv || !gap || !sharp)) || !mu0 || (c > 0 && (!lu0 || !piv0)))
    return fail(AFC_EINVAL, "null argument");
  if (!(r_min > 0.0) || !(eps_bar >= 0.0)) return fail(AFC_EINVAL, "need r_min > 0 and eps_bar >= 0");
  const SolveWs L = ws_layout_for(chain->n, c);
  if (!workspace || workspace_bytes < L.total)
    return fail(AFC_ENOMEM, "workspace of %zu bytes given, %zu needed", workspace_bytes, L.total);
  ChainDev C = chain_dev(chain, counts, c_index, c_list, c);
  cudaError_t e = launch_certificates(C, mu0, lu0, piv0, eps_bar, r_min, npairs, pu, pv, gap, sharp,
                                      static_cast<unsigned char *>(workspace), L, (cudaStream_t)stream);
  return e == cudaSuccess ? AFC_OK : cuda_fail(e, "certificates launch");
}

int afc_reward_afc(const afc_chain *chain, const uint32_t *counts, const double *b,
                   const double *psi_sum, double *out, void *stream) {
  if (!chain || !counts || !b || !out || chain->n < 1 || chain->realizations == 0)
    return fail(AFC_EINVAL, "bad arguments");
  cudaError_t e = launch_reward_afc(chain->n, chain->realizations, chain->alpha,
                                    chain->absorb_floor, counts, b, psi_sum, out,
                                    (cudaStream_t)stream);
  return e == cudaSuccess ? AFC_OK : cuda_fail(e, "reward_afc");
}

int afc_absorbing_solve_noalloc(const afc_chain *chain, const uint32_t *counts, double *mu,
                                double *b, double *scalars, void *stream) {
  if (!chain || !counts || !mu || !b || !scalars) return fail(AFC_EINVAL, "null argument");
  if (const int st = chain_params_check(chain)) return st;
  if (chain->n > 4096)
    return fail(AFC_EUNSUPPORTED, "the allocation-free solve supports n <= 4096 (got %d)", chain->n);
  uint32_t status = 0;
  int32_t c = 0;
  cudaError_t e = launch_solve_static(chain->n, chain->realizations, chain->alpha,
                                      chain->absorb_floor, chain->s_init, chain->reward, counts, mu,
                                      b, scalars, &status, &c, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "allocation-free solve");
  if (status == 1u)
    return fail(AFC_EUNSUPPORTED, "the allocation-free solve supports at most 256 observed states (got %d)", c);
  if (status == 2u) return fail(AFC_ESINGULAR, "zero pivot in the LU of I - Q_CC");
  return AFC_OK;
}

// ---- end to end from host memory ----------------------------------------------------------------

int afc_run_host(const afc_host_query *q, afc_host_result *res, void *stream) {
  NvtxRange nvtx_range("afc.run_host");
  if (!q || !res) return fail(AFC_EINVAL, "null query or result");
  if (!res->b) return fail(AFC_EINVAL, "result.b (host output [n]) is null");
  const int32_t n = q->n;
  const int64_t m = q->m;
  if (n < 1 || m < 0) return fail(AFC_EINVAL, "bad n/m");
  cudaStream_t s = (cudaStream_t)stream;
  std::vector<int32_t> rp((size_t)n + 1), col((size_t)std::max<int64_t>(2 * m, 1)), eid(col.size());
  int st = afc_csr_from_edges(n, m, q->eu, q->ev, rp.data(), col.data(), eid.data());
  if (st) return st;
  std::vector<uint64_t> th;
  if (q->p_survive) {
    th.resize((size_t)m);
    for (int64_t e = 0; e < m; ++e) th[e] = afc_survival_threshold(q->p_survive[e]);
  }
  std::vector<uint8_t> inw;
  if (q->candidates) {
    inw.assign((size_t)n, 0);
    for (int32_t k = 0; k < q->n_candidates; ++k) {
      if (q->candidates[k] < 0 || q->candidates[k] >= n) return fail(AFC_EINVAL, "candidate out of range");
      inw[q->candidates[k]] = 1;
    }
  }
  // device buffers (stream ordered)
  std::vector<void *> allocs;
  auto dalloc = [&](size_t bytes) -> void * {
    void *p = nullptr;
    if (cudaMallocAsync(&p, std::max<size_t>(bytes, 16), s) != cudaSuccess) return nullptr;
    allocs.push_back(p);
    return p;
  };
  auto cleanup = [&]() {
    for (void *p : allocs) cudaFreeAsync(p, s);
    cudaStreamSynchronize(s);
  };
  int rc = AFC_OK;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  cudaEventCreate(&ev0);
  cudaEventCreate(&ev1);
  do {
    int32_t *d_rp = (int32_t *)dalloc(4 * rp.size());
    int32_t *d_col = (int32_t *)dalloc(4 * col.size());
    int32_t *d_eid = (int32_t *)dalloc(4 * eid.size());
    uint64_t *d_th = th.empty() ? nullptr : (uint64_t *)dalloc(8 * th.size());
    uint32_t *d_wlo = q->w_lo ? (uint32_t *)dalloc(4 * (size_t)m) : nullptr;
    uint32_t *d_whi = q->w_hi ? (uint32_t *)dalloc(4 * (size_t)m) : nullptr;
    uint8_t *d_inw = inw.empty() ? nullptr : (uint8_t *)dalloc(inw.size());
    double *d_s = q->s_init ? (double *)dalloc(8 * (size_t)n) : nullptr;
    double *d_f = q->reward ? (double *)dalloc(8 * (size_t)n) : nullptr;
    uint32_t *d_counts = (uint32_t *)dalloc(4 * (size_t)n * ((size_t)n + 1));
    afc_mc_stats *d_stats = (afc_mc_stats *)dalloc(sizeof(afc_mc_stats));
    if (!d_rp || !d_col || !d_eid || !d_counts || !d_stats) { rc = fail(AFC_ENOMEM, "device allocation"); break; }
    cudaEventRecord(ev0, s);
    cudaMemcpyAsync(d_rp, rp.data(), 4 * rp.size(), cudaMemcpyHostToDevice, s);
    cudaMemcpyAsync(d_col, col.data(), 4 * col.size(), cudaMemcpyHostToDevice, s);
    cudaMemcpyAsync(d_eid, eid.data(), 4 * eid.size(), cudaMemcpyHostToDevice, s);
    if (d_th) cudaMemcpyAsync(d_th, th.data(), 8 * th.size(), cudaMemcpyHostToDevice, s);
    if (d_wlo) cudaMemcpyAsync(d_wlo, q->w_lo, 4 * (size_t)m, cudaMemcpyHostToDevice, s);
    if (d_whi) cudaMemcpyAsync(d_whi, q->w_hi, 4 * (size_t)m, cudaMemcpyHostToDevice, s);
    if (d_inw) cudaMemcpyAsync(d_inw, inw.data(), inw.size(), cudaMemcpyHostToDevice, s);
    if (d_s) cudaMemcpyAsync(d_s, q->s_init, 8 * (size_t)n, cudaMemcpyHostToDevice, s);
    if (d_f) cudaMemcpyAsync(d_f, q->reward, 8 * (size_t)n, cudaMemcpyHostToDevice, s);
    cudaMemsetAsync(d_counts, 0, 4 * (size_t)n * ((size_t)n + 1), s);
    cudaMemsetAsync(d_stats, 0, sizeof(afc_mc_stats), s);
    afc_mc_problem p{};
    p.n = n; p.m = m; p.row_ptr = d_rp; p.col = d_col; p.eid = d_eid;
    p.seed = q->seed; p.graph_tag = q->graph_tag;
    p.thresh = d_th; p.thresh_all = afc_survival_threshold(q->p_survive_all);
    p.w_lo = d_wlo; p.w_hi = d_whi; p.w_lo_all = q->w_lo_all; p.w_hi_all = q->w_hi_all;
    p.k_min = q->k_min; p.in_w = d_inw; p.top_k = q->top_k; p.tie_rel = q->tie_rel;
    p.precision = q->precision; p.recheck_margin = q->recheck_margin;
    const size_t wsc = afc_transition_counts_workspace(&p);
    if (wsc == 0) { rc = validate(&p); if (!rc) rc = fail(AFC_EINVAL, "problem rejected"); break; }
    void *d_wsc = dalloc(wsc);
    if (!d_wsc) { rc = fail(AFC_ENOMEM, "device allocation"); break; }
    rc = afc_transition_counts(&p, q->r_begin, q->realizations, d_counts, d_stats, nullptr, nullptr,
                               d_wsc, wsc, s);
    if (rc) break;
    int32_t *d_cidx = (int32_t *)dalloc(4 * (size_t)n);
    int32_t *d_clist = (int32_t *)dalloc(4 * (size_t)n);
    int32_t c = 0;
    rc = afc_observed_states(n, d_counts, d_cidx, d_clist, &c, s);
    if (rc) break;
    afc_chain ch{n, q->realizations, q->alpha, q->absorb_floor, d_s, d_f};
    const size_t wss = afc_solve_workspace(n, c);
    void *d_wss = dalloc(wss);
    double *d_mu = (double *)dalloc(8 * (size_t)n);
    double *d_b = (double *)dalloc(8 * (size_t)n);
    double *d_sc = (double *)dalloc(8 * 4);
    double *d_lu = (double *)dalloc(8 * (size_t)std::max(c, 1) * (size_t)std::max(c, 1));
    int32_t *d_piv = (int32_t *)dalloc(4 * (size_t)std::max(c, 1));
    if (!d_wss || !d_mu || !d_b || !d_sc || !d_lu || !d_piv) { rc = fail(AFC_ENOMEM, "device allocation"); break; }
    rc = afc_absorbing_solve(&ch, d_counts, d_cidx, d_clist, c, d_mu, d_b, d_sc, d_lu, d_piv, d_wss, wss, s);
    if (rc) break;
    uint64_t *d_pc = (uint64_t *)dalloc(8 * (3 + 100 + 16));
    double *d_pm = (double *)dalloc(8 * 3);
    if (q->n_perturb > 0) {
      if (!d_pc || !d_pm) { rc = fail(AFC_ENOMEM, "device allocation"); break; }
      cudaMemsetAsync(d_pc, 0, 8 * (3 + 100 + 16), s);
      cudaMemsetAsync(d_pm, 0, 8 * 3, s);
      afc_perturb_params pp{0, q->n_perturb, q->l1_radius, q->r_min, q->perturb_seed, 5, 10, 16, q->tie_rel};
      rc = afc_perturb_sweep(&ch, &pp, d_counts, d_cidx, d_clist, c, d_mu, d_b, d_lu, d_piv, d_pc,
                             d_pc + 3, d_pc + 103, d_pm, nullptr, d_wss, wss, s);
      if (rc) break;
    }
    double sc[4] = {0, 0, 0, 0};
    cudaMemcpyAsync(sc, d_sc, sizeof(sc), cudaMemcpyDeviceToHost, s);
    cudaMemcpyAsync(res->b, d_b, 8 * (size_t)n, cudaMemcpyDeviceToHost, s);
    if (res->mu) cudaMemcpyAsync(res->mu, d_mu, 8 * (size_t)n, cudaMemcpyDeviceToHost, s);
    if (res->counts) cudaMemcpyAsync(res->counts, d_counts, 4 * (size_t)n * ((size_t)n + 1), cudaMemcpyDeviceToHost, s);
    cudaMemcpyAsync(&res->stats, d_stats, sizeof(afc_mc_stats), cudaMemcpyDeviceToHost, s);
    if (q->n_perturb > 0) {
      cudaMemcpyAsync(res->perturb_counters, d_pc, 8 * 3, cudaMemcpyDeviceToHost, s);
      cudaMemcpyAsync(res->perturb_maxima, d_pm, 8 * 3, cudaMemcpyDeviceToHost, s);
    } else {
      memset(res->perturb_counters, 0, sizeof(res->perturb_counters));
      memset(res->perturb_maxima, 0, sizeof(res->perturb_maxima));
    }
    cudaEventRecord(ev1, s);
    cudaError_t e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) { rc = cuda_fail(e, "run_host"); break; }
    float ms = 0.f;
    cudaEventElapsedTime(&ms, ev0, ev1);
    res->device_ms = ms;
    res->expected_T = sc[0];
    res->b_f = sc[1];
    res->max_rowsum_N = sc[2];
    res->c = c;
    if (res->stats.device_error) { rc = fail(AFC_EDEVICE, "device consistency check failed (bits %llu)", (unsigned long long)res->stats.device_error); break; }
    if (res->stats.overflow) { rc = fail(AFC_EOVERFLOW, "path count overflow in %llu realizations", (unsigned long long)res->stats.overflow); break; }
  } while (false);
  cleanup();
  cudaEventDestroy(ev0);
  cudaEventDestroy(ev1);
  return rc;
}

}  // extern "C"
