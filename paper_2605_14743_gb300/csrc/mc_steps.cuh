// mc_steps.cuh -- Brandes from one source by one warp, by settle steps (Dijkstra with the IN
// and OUT finality criteria), used by both counting paths: source slots in shared memory
// (mc_kernel.cu) or split between shared memory (distances) and device memory (mc_global.cu).
//
// Every step settles, at once, all pending nodes v whose tentative distance d(v) is below
// d_min + mw(v) (mw: v's smallest incident length; the "IN" criterion) or below the smallest
// d(u) + mw(u) over the pending nodes u (the "OUT" criterion).  Such a distance is final, and
// no pending node can precede v on a shortest path, so every predecessor of a step's nodes was
// settled in an earlier step: path counts are pulled from them in the same arc scan that
// relaxes the step's other arcs, and dependencies take one reverse scan per arc, step by step
// in reverse.  Per-source results do not depend on which warp runs the source, and the exact
// betweenness sum does not depend on the order in which sources finish.
#pragma once
#include "mc_common.cuh"

namespace afc {

// One source slot, wide form (16 bytes per node): dist[n] (u32 | kFlag once settled), sig[n]
// (sigma, then rho in place), ord[n] (settle order; bit 15 marks the first node of a step) and
// plist[n] (the pending nodes: discovered, not yet settled, each once).
//
// Compact form (COMPACT = true, 12 bytes per node): dist[n] and n 8-byte words, word[k] =
// sigma of node k (low 32 bits) | pending-list entry k (16 bits) | settle-order entry k (top
// 16 bits); the separate ord and plist arrays are not used.  The backward pass no longer needs
// sigma of a node once its rho is known, nor the pending list, nor 32-bit distances: when the
// forward pass ends, node v's distance mod 2^16 moves into the pending-list half of word[v],
// and rho(v) (64 bits) takes dist[v] (high half) and the sigma half of word[v] (low half).
// Distances mod 2^16 identify successors exactly when every length is below 2^15 (adjacent
// nodes' distances differ by at most the arc's length), and sigma must stay below 2^32: a
// realization outside either limit runs on wide slots (the routine reports a path count above
// 2^32 - 1 as ovf bit 1 and the caller redoes the realization).
struct StepSlot {
  uint32_t *dist;
  uint64_t *sig;
  uint16_t *ord, *plist;
};

constexpr uint32_t kOvfWide = 2u;          // ovf bit: a path count does not fit a compact slot
constexpr uint32_t kCompactMaxLen = 32767;  // longest length a compact slot supports

template <bool COMPACT>
__device__ __forceinline__ uint16_t *pend_at(const StepSlot &sl, uint32_t j) {
  if constexpr (COMPACT)
    return reinterpret_cast<uint16_t *>(sl.sig) + 4u * j + 2u;
  else
    return sl.plist + j;
}

template <bool COMPACT>
__device__ __forceinline__ uint16_t *ord_at(const StepSlot &sl, uint32_t k) {
  if constexpr (COMPACT)
    return reinterpret_cast<uint16_t *>(sl.sig) + 4u * k + 3u;
  else
    return sl.ord + k;
}

// sigma(v) during the forward pass (and of a node not yet given its rho in the backward pass)
template <bool COMPACT>
__device__ __forceinline__ uint64_t sig_get(const StepSlot &sl, uint32_t v) {
  if constexpr (COMPACT)
    return (uint64_t)reinterpret_cast<const uint32_t *>(sl.sig)[2u * v];
  else
    return sl.sig[v];
}

template <bool COMPACT>
__device__ __forceinline__ void sig_put(const StepSlot &sl, uint32_t v, uint64_t x) {
  if constexpr (COMPACT)
    reinterpret_cast<uint32_t *>(sl.sig)[2u * v] = (uint32_t)x;
  else
    sl.sig[v] = x;
}

// rho(v) in the backward pass (kIntTag | integer, or the bits of a DT)
template <bool COMPACT>
__device__ __forceinline__ uint64_t rho_get(const StepSlot &sl, uint32_t v) {
  if constexpr (COMPACT)
    return ((uint64_t)sl.dist[v] << 32) | reinterpret_cast<const uint32_t *>(sl.sig)[2u * v];
  else
    return sl.sig[v];
}

template <bool COMPACT>
__device__ __forceinline__ void rho_put(const StepSlot &sl, uint32_t v, uint64_t x) {
  if constexpr (COMPACT) {
    sl.dist[v] = (uint32_t)(x >> 32);
    reinterpret_cast<uint32_t *>(sl.sig)[2u * v] = (uint32_t)x;
  } else {
    sl.sig[v] = x;
  }
}

// Distance of a settled node in the backward pass: exact (wide) or mod 2^16 (compact).
template <bool COMPACT>
__device__ __forceinline__ uint32_t bdist(const StepSlot &sl, uint32_t v) {
  if constexpr (COMPACT)
    return reinterpret_cast<const uint16_t *>(sl.sig)[4u * v + 2u];
  else
    return sl.dist[v] & kMask;
}

constexpr uint16_t kStepStart = 0x8000u;   // ord entry opens a step (node ids stay below 2^15)

// Smallest alive incident length of every node (0xFFFF for a node without alive arcs).
__device__ inline void min_lengths(const Realized &H, uint16_t *mw) {
  for (uint32_t v = threadIdx.x; v < H.n; v += blockDim.x) {
    uint32_t m = 0xFFFFu;
    for (uint32_t e = H.rp[v]; e < H.rp[v + 1]; ++e) m = min(m, H.arc[e] >> 16);
    mw[v] = (uint16_t)m;
  }
}

// Exclusive prefix of x over the warp's lanes; total = the sum over all lanes.
__device__ __forceinline__ uint32_t warp_excl(uint32_t x, uint32_t &total) {
  const uint32_t lane = lane_id();
  uint32_t incl = x;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(kFull, incl, o);
    if (lane >= (uint32_t)o) incl += y;
  }
  total = __shfl_sync(kFull, incl, 31);
  return incl - x;
}

// Issue widths of the routine, by where the source slot lives (measured on ws1000 for slots in
// shared memory, on the batched mix's 2,300-3,800-node graphs for slots in the device arena):
// pend: pending-list windows (32 nodes each) loaded together at the start of a step's
// selection; fwd / bwd: arcs of a lane's node whose loads (and relaxations) are issued
// together in the forward / backward pass.
template <bool ONCHIP> struct StepTune;
template <> struct StepTune<true> { static constexpr int pend = 6, fwd = 4, bwd = 2; };
template <> struct StepTune<false> { static constexpr int pend = 16, fwd = 4, bwd = 8; };

// ---------------------------------------------------------------------------------------
// Brandes from source s by one warp (Sec. 3.1 definitions: d_H, sigma_st, ordered-pair
// betweenness).  Forward: settle steps (see the file comment), sigma pulled from the
// predecessors while the step's arcs are relaxed; the next step's bounds d_min and
// min (d + mw) come from the pending nodes that stay and from the relaxations (every pending
// node's current distance is one of those values, and no recorded value is below the node's
// current distance), so no separate pass over the pending list is needed.  Backward
// (want_delta): the steps in reverse; rho(v) = (1 + delta(v)) / sigma(v) replaces sigma in
// place, delta(v) =
// sigma(v) * sum over successors w of rho(w) in arc order; unique-path subtrees (sigma = 1
// throughout) stay exact integers.  delta_s(v) for v != s goes to the exact accumulators of
// the CTA scratch (fx_red).  Every lane of the warp must call it; err / ovf collect
// device-error bits and path-count overflow per lane (bit 0: above 2^64 - 1; bit 1, compact
// slots only: above 2^32 - 1, after which the backward pass is skipped).  Compact slots need
// every length below 2^15 (kCompactMaxLen).
// ---------------------------------------------------------------------------------------
template <typename DT, bool COMPACT, bool ONCHIP>
__device__ bool source_steps(const Realized &H, const uint16_t *mw, const StepSlot &sl,
                             uint32_t s, bool want_delta, const BcAcc &cs, uint32_t &err,
                             uint32_t &ovf) {
  constexpr int kPendCache = StepTune<ONCHIP>::pend, kArcsFwd = StepTune<ONCHIP>::fwd,
                kArcsBwd = StepTune<ONCHIP>::bwd;
  static_assert(!COMPACT || ONCHIP, "compact slots live in shared memory");
  const uint32_t n = H.n, lane = lane_id();
  for (uint32_t v = lane; v < n; v += 32) sl.dist[v] = kInf;
  __syncwarp();
  if (lane == 0) {
    sl.dist[s] = 0u;
    sig_put<COMPACT>(sl, s, 1ull);
    *pend_at<COMPACT>(sl, 0) = (uint16_t)s;
  }
  __syncwarp();

  // ---- forward
  uint32_t nord = 0, pc = 1;                   // settled nodes, pending nodes (warp-uniform)
  uint32_t dmin = 0u, lout = (uint32_t)mw[s];   // d_min and min (d + mw) over the pending nodes
  for (uint32_t step = 0;; ++step) {
    if (step > n) { err |= kErrPassLimit; return false; }
    if (pc == 0) break;   // nothing pending: the source's component is done
    // (1) settle every pending v with d(v) < d_min + mw(v) (IN) or d(v) < lout (OUT; the node
    // at d_min always qualifies): append it to ord, flag it settled; the others stay,
    // compacted in order, and give the next step's bounds together with the relaxations below
    const uint32_t g0 = nord;
    const uint32_t below = lanemask_lt();
    uint32_t kept = 0, ndmin = kInf, nlout = 0xFFFFFFFFu;
    auto place = [&](bool sel, bool keep, uint32_t sm, uint32_t km, uint32_t v, uint32_t d,
                     uint32_t m) {
      if (sel) {
        const uint32_t pos = nord + (uint32_t)__popc(sm & below);
        if (pos < n) {
          *ord_at<COMPACT>(sl, pos) = (uint16_t)(v | (pos == g0 ? kStepStart : 0u));
          sl.dist[v] = d | kFlag;
        } else {
          err |= kErrCapacity;
        }
      } else if (keep) {
        *pend_at<COMPACT>(sl, kept + (uint32_t)__popc(km & below)) = (uint16_t)v;
        ndmin = min(ndmin, d);
        nlout = min(nlout, d + m);
      }
      nord += (uint32_t)__popc(sm);
      kept += (uint32_t)__popc(km);
    };
    {
      // the first kPendCache windows: every load first, then the decisions, then the stores
      uint32_t cv[kPendCache], cm[kPendCache], cd[kPendCache];
#pragma unroll
      for (int c = 0; c < kPendCache; ++c) {
        const uint32_t j = (uint32_t)c * 32u + lane;
        cv[c] = j < pc ? (uint32_t)*pend_at<COMPACT>(sl, j) : 0u;
      }
#pragma unroll
      for (int c = 0; c < kPendCache; ++c) {
        const bool valid = (uint32_t)c * 32u + lane < pc;
        cm[c] = valid ? (uint32_t)mw[cv[c]] : 0u;
        cd[c] = valid ? (uint32_t)sl.dist[cv[c]] : 0u;
      }
#pragma unroll
      for (int c = 0; c < kPendCache; ++c) {
        if ((uint32_t)c * 32u >= pc) break;   // warp-uniform
        const bool valid = (uint32_t)c * 32u + lane < pc;
        const bool sel = valid && (cd[c] < dmin + cm[c] || cd[c] < lout);
        const uint32_t sm = __ballot_sync(kFull, sel), km = __ballot_sync(kFull, valid && !sel);
        place(sel, valid && !sel, sm, km, cv[c], cd[c], cm[c]);
      }
    }
    // the other windows: each is read before its kept nodes move down (to lower positions)
    for (uint32_t j0 = kPendCache * 32u; j0 < pc; j0 += 32u) {
      const uint32_t j = j0 + lane;
      uint32_t v = 0, d = 0, m = 0;
      if (j < pc) {
        v = *pend_at<COMPACT>(sl, j);
        d = sl.dist[v];
        m = mw[v];
      }
      const bool sel = j < pc && (d < dmin + m || d < lout);
      const uint32_t smw = __ballot_sync(kFull, sel);
      const uint32_t kmw = __ballot_sync(kFull, j < pc && !sel);
      place(sel, j < pc && !sel, smw, kmw, v, d, m);
    }
    pc = kept;
    __syncwarp();
    // (3) the step's arcs, one member per lane: sigma from the (settled) predecessors and
    // relaxation of the rest; each group of kArcsFwd arcs issues its loads and atomics together
    const uint32_t g1 = min(nord, n);
    for (uint32_t c0 = g0; c0 < g1; c0 += 32) {
      const uint32_t k = c0 + lane;
      const bool mine = k < g1;
      uint32_t v = 0, dv = 0, e = 0, e1 = 0;
      if (mine) {
        v = *ord_at<COMPACT>(sl, k) & 0x7FFFu;
        dv = sl.dist[v] & kMask;
        e = H.rp[v];
        e1 = H.rp[v + 1];
      }
      unsigned long long sg = 0;
      while (__any_sync(kFull, e < e1)) {
        uint32_t pk[kArcsFwd], du[kArcsFwd], old[kArcsFwd];
        unsigned long long x[kArcsFwd];
#pragma unroll
        for (int t = 0; t < kArcsFwd; ++t) pk[t] = e + t < e1 ? H.arc[e + t] : 0u;
#pragma unroll
        for (int t = 0; t < kArcsFwd; ++t) du[t] = e + t < e1 ? sl.dist[pk[t] & 0xFFFFu] : kFlag;
#pragma unroll
        for (int t = 0; t < kArcsFwd; ++t) {
          const uint32_t u = pk[t] & 0xFFFFu, len = pk[t] >> 16;
          // a predecessor: settled in an earlier step
          const bool pred = (du[t] & kFlag) && (du[t] & kMask) + len == dv && e + t < e1;
          x[t] = pred ? sig_get<COMPACT>(sl, u) : 0ull;
          const uint32_t nd = dv + len;
          const bool relax = !(du[t] & kFlag) && nd < du[t];
          old[t] = relax ? atomicMin(&sl.dist[u], nd) : 0u;
          if (relax) {   // a pending node's new distance: the next step's bounds
            ndmin = min(ndmin, nd);
            nlout = min(nlout, nd + (uint32_t)mw[u]);
          }
        }
        // discovered now (each node once): onto the pending list
        uint32_t dm[kArcsFwd];
#pragma unroll
        for (int t = 0; t < kArcsFwd; ++t) dm[t] = __ballot_sync(kFull, old[t] == kInf);
#pragma unroll
        for (int t = 0; t < kArcsFwd; ++t) {
          const unsigned long long nx = sg + x[t];
          if (!COMPACT && nx < sg) ovf |= 1u;   // compact addends are below 2^32: no wrap
          sg = nx;
          if ((dm[t] >> lane) & 1u)
            *pend_at<COMPACT>(sl, pc + (uint32_t)__popc(dm[t] & lanemask_lt())) =
                (uint16_t)(pk[t] & 0xFFFFu);
          pc += (uint32_t)__popc(dm[t]);
        }
        e += kArcsFwd;
      }
      if (COMPACT && (sg >> 32)) ovf |= kOvfWide;
      if (mine && v != s) sig_put<COMPACT>(sl, v, sg);
    }
    dmin = __reduce_min_sync(kFull, ndmin);
    lout = __reduce_min_sync(kFull, nlout);
    __syncwarp();
  }
  if (!want_delta) return true;
  if constexpr (COMPACT) {
    // a path count that a compact slot cannot hold: the caller redoes the realization
    if (__any_sync(kFull, ovf & kOvfWide)) return true;
    // distances mod 2^16 into the (now empty) pending-list halves; every node the backward
    // pass reads was reached (settled nodes and their neighbours)
    uint16_t *w16 = reinterpret_cast<uint16_t *>(sl.sig);
    for (uint32_t v = lane; v < n; v += 32) w16[4u * v + 2u] = (uint16_t)sl.dist[v];
    __syncwarp();
  }

  // ---- backward: the steps in reverse order of settlement, one member per lane
  uint32_t hi = min(nord, n);
  while (hi > 0) {
    // the step holding position hi - 1 starts at the nearest step mark at or below it
    uint32_t lo = 0;
    for (int32_t top = (int32_t)hi - 1; top >= 0; top -= 32) {
      const int32_t p = top - (int32_t)lane;
      const bool mark = p >= 0 && (*ord_at<COMPACT>(sl, (uint32_t)p) & kStepStart);
      const uint32_t mm = __ballot_sync(kFull, mark);
      if (mm) {
        lo = (uint32_t)(top - (__ffs(mm) - 1));
        break;
      }
    }
    for (uint32_t c0 = lo; c0 < hi; c0 += 32) {
      const uint32_t k = c0 + lane;
      const bool mine = k < hi;
      uint32_t v = 0, dv = 0, e = 0, e1 = 0;
      uint64_t sg = 0;
      if (mine) {
        v = *ord_at<COMPACT>(sl, k) & 0x7FFFu;
        dv = bdist<COMPACT>(sl, v);
        e = H.rp[v];
        e1 = H.rp[v + 1];
        sg = sig_get<COMPACT>(sl, v);
      }
      // the successors' rho in arc order: integral ones exactly, the others in DT
      uint32_t acc_i = 0;
      DT acc_f = 0;
      bool any_f = false;
      while (__any_sync(kFull, e < e1)) {
        uint32_t pk[kArcsBwd];
        uint64_t rw[kArcsBwd];
#pragma unroll
        for (int t = 0; t < kArcsBwd; ++t) pk[t] = e + t < e1 ? H.arc[e + t] : 0u;
#pragma unroll
        for (int t = 0; t < kArcsBwd; ++t) {
          const uint32_t w = pk[t] & 0xFFFFu, want = dv + (pk[t] >> 16);
          const bool suc = e + t < e1 && bdist<COMPACT>(sl, w) == (COMPACT ? want & 0xFFFFu : want);
          rw[t] = suc ? rho_get<COMPACT>(sl, w) : kIntTag;   // kIntTag alone adds 0
        }
#pragma unroll
        for (int t = 0; t < kArcsBwd; ++t) {
          if (rw[t] & kIntTag) {
            acc_i += (uint32_t)rw[t];
          } else {
            acc_f += *reinterpret_cast<const DT *>(&rw[t]);
            any_f = true;
          }
        }
        e += kArcsBwd;
      }
      if (mine) {
        if (sg == 1ull && !any_f) {
          // delta(v) = sum of the successors' subtree sizes: exact in integers
          rho_put<COMPACT>(sl, v, kIntTag | (uint64_t)(1u + acc_i));
          if (v != s && acc_i) atomicAdd(&cs.a0[v], (unsigned long long)acc_i);
        } else {
          DT dep, rho;
          dependency<DT>(sg, (DT)acc_i + acc_f, dep, rho);
          uint64_t bits = 0;
          *reinterpret_cast<DT *>(&bits) = rho;
          rho_put<COMPACT>(sl, v, bits);
          if (v != s) fx_red(cs.a0, cs.a1, cs.a2, v, (double)dep);
        }
      }
    }
    __syncwarp();
    hi = lo;
  }
  return true;
}

}  // namespace afc
