// mc_types.h -- the structures and constants of the counting kernels (both paths): the
// problem as the kernels see it, the per-CTA control blocks and the global path's groups.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "afc.h"

namespace afc {

constexpr uint32_t kSizeMask = 0x00FFFFFFu;  // component size in cinfo
constexpr uint32_t kHasCand = 0x80000000u;   // component holds a candidate

// device_error bits
constexpr uint32_t kErrInput = 1u;       // malformed CSR / weight seen on the device
constexpr uint32_t kErrCapacity = 2u;    // a per-source list would have overflowed
constexpr uint32_t kErrPassLimit = 4u;   // an iteration bound was hit
constexpr uint32_t kErrSolve = 8u;       // zero pivot in a device LU

// One problem as seen by the counting kernel (all pointers device).
struct McDev {
  int32_t n;
  int64_t m;
  const int32_t *row_ptr, *col, *eid;
  uint32_t key_lo, key_hi, graph_tag;
  const uint64_t *thresh;
  uint64_t thresh_all;
  const uint32_t *w_lo, *w_hi;
  uint32_t w_lo_all, w_hi_all;
  uint32_t k_min;
  const uint8_t *in_w;
  uint32_t top_k;
  double tie_rel;
  int32_t precision;
  double recheck_margin;
  uint32_t delta;
  uint32_t spt;          // shared path: source warps for this problem (0: the launch's value)
  uint32_t r_begin;
  uint32_t reward_k;             // valued Top-k step reward (0: off)
  const double *reward_gamma;    // [n] or null (1)
  const uint8_t *reward_pool;    // [n] or null (every node)
  double *psi;                   // [n] step-reward accumulator
  uint32_t report_rank;          // 0 / 1: the centre; r > 1: the r-th node of the ordering
  uint32_t fb_node;              // fallback node v_fb, or 0xFFFFFFFF (infeasible draws absorb)
  uint32_t *fb_count;            // [n] redirected draws per anchor, or null
  uint32_t tie_random;           // 1: uniformly drawn tie-break instead of the smallest id
  const uint32_t *wtab_ptr;      // [m+1] per-edge threshold ranges of a discrete length law, or null
  const uint32_t *wtab;          // thresholds
  uint32_t per_row;              // 1: independent draws per row (items = draws x n)
  uint32_t hop_radius;           // row-wise mode: r of the r-hop neighbourhood (0 = whole graph)
  uint32_t *counts;
  afc_mc_stats *stats;
  double *dump_bc;
  int32_t *dump_next;
};

constexpr int kMaxSlots = 64;          // sources in flight per CTA
constexpr int kMaxTeams = 32;          // independent thread teams per CTA
constexpr int kMaxSlotsPerTeam = 16;   // sources a team advances in lockstep
constexpr int kRing = 16;              // bucket bitmaps per source (ring over pending distances)

struct SlotCtl {
  uint32_t s, nm, mstart, hi, lo, ring_mask, pad[2];
};

struct TeamCtl {
  uint32_t bucket, claim, nslots, base;
  uint32_t red[4];
  uint32_t pref[kMaxSlotsPerTeam + 1];
  uint32_t pad[3];
};

// Per-warp scratch of the warp-cooperative arc loops: accumulators of the current chunk of
// 32 items (one per lane), the floating contributions of the current window of 32 arc
// positions (summed by their owners in arc order, so sums never depend on the schedule) and
// the rank -> lane table of the chunk's items that have arcs.
struct WarpScratch {
  unsigned long long acc[32];
  double buf[32];
  uint32_t acci[32];
  uint32_t flags[32];
  uint8_t table[32];
};

// Control fields of a CTA that works on one realization (realization, components, selection).
struct CtaHead {
  uint32_t err, ovf, nsrc, cursor;
  unsigned long long edges, verts;
  uint32_t need_recheck, delta, dsh, wmax;
  uint32_t scan[32];
  uint32_t scan_total, wide_redo, pad2, pad3;   // wide_redo: a path count needs 64-bit slots
};

// The bucketed kernel's control block: the head plus its slot, team and warp tables.
struct CtaCtl : CtaHead {
  SlotCtl slot[kMaxSlots];
  TeamCtl team[kMaxTeams];
  WarpScratch warp[32];
};

// One realization in flight on the global-memory counting path.  The arrays are carved from
// the caller's workspace by the host; the counters are (re)set by the preparation kernel.
struct BigGroup {
  uint32_t r_local;      // realization offset from the problem's r_begin
  uint32_t active;       // 1 while the group holds a realization of the current batch
  uint32_t nsrc, cursor, dsh, err, ovf, redo;
  unsigned long long edges, verts;
  uint32_t *rp, *arc, *comp, *cinfo, *centre, *rank;
  uint16_t *src;
  // betweenness: exact fixed point accumulated in (bc's bits, a1, a2), B 2^64 = bc 2^64 +
  // a1 2^32 + a2, converted to doubles in place (bc) before the selection
  double *bc;
  unsigned long long *a1, *a2;
  unsigned long long *best;
  uint16_t *mw;           // smallest alive incident length per node
};

}  // namespace afc
