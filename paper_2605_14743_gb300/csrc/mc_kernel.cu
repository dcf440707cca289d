// mc_kernel.cu -- Monte Carlo transition counts on GB300 (sm_103a), shared-memory path.
//
// One CTA owns one network realization at a time (persistent over realizations) and keeps
// it in shared memory:
//   A1  Philox4x32-10 edge draws -> alive-compacted CSR with packed (neighbour, length) arcs,
//       and the smallest alive length at every node
//   A2  components by lock-free union-find (root = smallest id), sizes, candidate flags
//   A3  one warp per source: Dijkstra by settle steps.  Every step settles, at once, all
//       pending nodes v whose tentative distance d(v) is below d_min + mw(v) (mw: v's smallest
//       incident length; the "IN" criterion) or below the smallest d(u) + mw(u) over the
//       pending nodes u (the "OUT" criterion).  Such a distance is final, and no pending node
//       can precede v on a shortest path, so every predecessor of a step's nodes was settled
//       in an earlier step.
//   A4  path counts sigma (exact 64-bit) pulled from those predecessors in the same arc scan
//       that relaxes the step's outgoing arcs: one scan per arc in the forward direction
//   A5  dependencies delta step by step in reverse (a successor is always settled in a later
//       step), one scan per arc; betweenness accumulated exactly in 128-bit fixed point
//   A6  tie-ruled argmax per valid component (Sec. 3.2 eq. local-center, Sec. 7.1 Sel_W)
//       and the transition-count update of every anchor (Alg. 1 / Alg. 2)
//   A7  FP32 mode: a realization whose top-two gap is under the margin is redone in FP64
// Per-source results do not depend on which warp or CTA runs the source, and the exact
// betweenness sum does not depend on the order in which sources finish, so B and every count
// are the same bit for bit for any launch shape.
#include "mc_common.cuh"

namespace afc {

// One source slot: dist[n] (u32 | kFlag once settled), sig[n] (sigma, then rho in place),
// ord[n] (settle order; bit 15 marks the first node of a step) and plist[n] (the pending nodes:
// discovered, not yet settled, each once).
struct StepSlot {
  uint32_t *dist;
  uint64_t *sig;
  uint16_t *ord, *plist;
};

constexpr uint16_t kStepStart = 0x8000u;   // ord entry opens a step (node ids stay below 2^15)

// Shared-memory layout of a counting CTA: control head, the realization (rp, arcs, smallest
// incident length) and one slot per source warp.  What the source warps do not touch while
// they run (components, the source list, selection scratch, betweenness accumulators) lives
// in the CTA's region of device memory (CtaScratch), so that more source slots fit on chip.
struct StepLayout {
  uint32_t off_rp, off_arc, off_mw, off_slots;
  uint32_t slot_bytes, total;
  __host__ __device__ static uint32_t al(uint32_t x) { return al16(x); }
  __host__ __device__ void make(uint32_t n, uint32_t arcs, uint32_t nsw) {
    uint32_t o = al(sizeof(CtaHead));
    off_rp = o;     o = al(o + 4u * (n + 1));
    off_arc = o;    o = al(o + 4u * (arcs > 0 ? arcs : 1));
    off_mw = o;     o = al(o + 2u * n);
    off_slots = o;
    slot_bytes = al(4u * n) + al(8u * n) + 2u * al(2u * n);
    total = o + nsw * slot_bytes;
  }
  __device__ StepSlot slot(unsigned char *smem, uint32_t i, uint32_t n) const {
    unsigned char *p = smem + off_slots + i * slot_bytes;
    StepSlot s;
    s.dist = reinterpret_cast<uint32_t *>(p);  p += al(4u * n);
    s.sig = reinterpret_cast<uint64_t *>(p);   p += al(8u * n);
    s.ord = reinterpret_cast<uint16_t *>(p);   p += al(2u * n);
    s.plist = reinterpret_cast<uint16_t *>(p);
    return s;
  }
};

// A counting CTA's region of device memory, for graphs of up to n nodes: comp[n], cinfo[n],
// sel[n], src[n] and the betweenness accumulators a0, a1, a2 [n] (B_v 2^64 = a0 2^64 +
// a1 2^32 + a2, see fx_red).
struct CtaScratch {
  uint32_t *comp, *cinfo, *sel;
  uint16_t *src;
  unsigned long long *a0, *a1, *a2;
  __host__ __device__ static size_t al(size_t x) { return (x + 255u) & ~size_t(255); }
  __host__ __device__ static size_t bytes(uint32_t n) {
    return 3 * al(4ull * n) + al(2ull * n) + 3 * al(8ull * n);
  }
  __device__ void carve(unsigned char *p, uint32_t n) {
    comp = reinterpret_cast<uint32_t *>(p);   p += al(4ull * n);
    cinfo = reinterpret_cast<uint32_t *>(p);  p += al(4ull * n);
    sel = reinterpret_cast<uint32_t *>(p);    p += al(4ull * n);
    src = reinterpret_cast<uint16_t *>(p);    p += al(2ull * n);
    a0 = reinterpret_cast<unsigned long long *>(p);  p += al(8ull * n);
    a1 = reinterpret_cast<unsigned long long *>(p);  p += al(8ull * n);
    a2 = reinterpret_cast<unsigned long long *>(p);
  }
};

// Betweenness accumulation without return values (device-memory reductions): the addend x
// (0 <= x < 2^64) is split exactly, from its bits, into x 2^64 = xi 2^64 + xf (xf < 2^64,
// truncated below 2^-64 as in fx_add), and xi, the top and the bottom 32 bits of xf go to three
// 64-bit sums (each far from overflow for fewer than 2^31 addends).  Integer additions are
// associative, so the total is exact and independent of the order.
__device__ __forceinline__ void fx_red(unsigned long long *a0, unsigned long long *a1,
                                       unsigned long long *a2, uint32_t v, double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const int ex = (int)((b >> 52) & 0x7FFu);
  if (ex == 0 || (b >> 63)) return;
  const unsigned long long m = (b & 0xFFFFFFFFFFFFFull) | (1ull << 52);
  const int sh = ex - 1075 + 64;
  unsigned long long xi, xf;
  if (sh >= 64) {
    xi = m << (sh - 64);
    xf = 0ull;
  } else if (sh > 0) {
    xi = m >> (64 - sh);
    xf = m << sh;
  } else if (sh > -53) {
    xi = 0ull;
    xf = m >> (-sh);
  } else {
    return;
  }
  if (xi) atomicAdd(&a0[v], xi);
  if (xf >> 32) atomicAdd(&a1[v], xf >> 32);
  if (xf & 0xFFFFFFFFull) atomicAdd(&a2[v], xf & 0xFFFFFFFFull);
}

// B_v as a double, written over a0 (each thread converts its own entries).
__device__ __forceinline__ void fx_finalize3(unsigned long long *a0, const unsigned long long *a1,
                                             const unsigned long long *a2, uint32_t n) {
  for (uint32_t v = threadIdx.x; v < n; v += blockDim.x) {
    const unsigned long long t = a1[v];
    const unsigned long long lo = a2[v] + (t << 32);
    const unsigned long long hi = a0[v] + (t >> 32) + (lo < (t << 32) ? 1ull : 0ull);
    reinterpret_cast<double *>(a0)[v] = (double)hi + __ull2double_rn(lo) * 0x1p-64;
  }
}

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

// Pending-list windows (32 nodes each) loaded together at the start of a step's selection.
constexpr int kPendCache = 8;

// ---------------------------------------------------------------------------------------
// Brandes from source s by one warp (Sec. 3.1 definitions: d_H, sigma_st, ordered-pair
// betweenness).  Forward: settle steps (see the file comment), sigma pulled from the
// predecessors while the step's arcs are relaxed; the next step's bounds d_min and
// min (d + mw) come from the pending nodes that stay and from the relaxations (every pending
// node's current distance is one of those values, and no recorded value is below the node's
// current distance), so no separate pass over the pending list is needed.  Backward (want_delta): the steps in
// reverse; rho(v) = (1 + delta(v)) / sigma(v) replaces sigma in place, delta(v) =
// sigma(v) * sum over successors w of rho(w) in arc order; unique-path subtrees (sigma = 1
// throughout) stay exact integers.  delta_s(v) for v != s goes to the exact accumulators of
// the CTA scratch (fx_red).  Every lane of the warp must call it; err / ovf collect
// device-error bits and path-count overflow per lane.
// ---------------------------------------------------------------------------------------
template <typename DT>
__device__ bool source_steps(const Realized &H, const uint16_t *mw, const StepSlot &sl,
                             uint32_t s, bool want_delta, const CtaScratch &cs, uint32_t &err,
                             uint32_t &ovf) {
  const uint32_t n = H.n, lane = lane_id();
  for (uint32_t v = lane; v < n; v += 32) sl.dist[v] = kInf;
  __syncwarp();
  if (lane == 0) {
    sl.dist[s] = 0u;
    sl.sig[s] = 1ull;
    sl.plist[0] = (uint16_t)s;
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
          sl.ord[pos] = (uint16_t)(v | (pos == g0 ? kStepStart : 0u));
          sl.dist[v] = d | kFlag;
        } else {
          err |= kErrCapacity;
        }
      } else if (keep) {
        sl.plist[kept + (uint32_t)__popc(km & below)] = (uint16_t)v;
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
        cv[c] = j < pc ? (uint32_t)sl.plist[j] : 0u;
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
        v = sl.plist[j];
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
    // relaxation of the rest; each group of four arcs issues its loads and atomics together
    const uint32_t g1 = min(nord, n);
    for (uint32_t c0 = g0; c0 < g1; c0 += 32) {
      const uint32_t k = c0 + lane;
      const bool mine = k < g1;
      uint32_t v = 0, dv = 0, e = 0, e1 = 0;
      if (mine) {
        v = sl.ord[k] & 0x7FFFu;
        dv = sl.dist[v] & kMask;
        e = H.rp[v];
        e1 = H.rp[v + 1];
      }
      unsigned long long sg = 0;
      while (__any_sync(kFull, e < e1)) {
        uint32_t pk[4], du[4], old[4];
        unsigned long long x[4];
#pragma unroll
        for (int t = 0; t < 4; ++t) pk[t] = e + t < e1 ? H.arc[e + t] : 0u;
#pragma unroll
        for (int t = 0; t < 4; ++t) du[t] = e + t < e1 ? sl.dist[pk[t] & 0xFFFFu] : kFlag;
#pragma unroll
        for (int t = 0; t < 4; ++t) {
          const uint32_t u = pk[t] & 0xFFFFu, len = pk[t] >> 16;
          // a predecessor: settled in an earlier step
          const bool pred = (du[t] & kFlag) && (du[t] & kMask) + len == dv && e + t < e1;
          x[t] = pred ? sl.sig[u] : 0ull;
          const uint32_t nd = dv + len;
          const bool relax = !(du[t] & kFlag) && nd < du[t];
          old[t] = relax ? atomicMin(&sl.dist[u], nd) : 0u;
          if (relax) {   // a pending node's new distance: the next step's bounds
            ndmin = min(ndmin, nd);
            nlout = min(nlout, nd + (uint32_t)mw[u]);
          }
        }
        // discovered now (each node once): onto the pending list
        uint32_t dm[4];
#pragma unroll
        for (int t = 0; t < 4; ++t) dm[t] = __ballot_sync(kFull, old[t] == kInf);
#pragma unroll
        for (int t = 0; t < 4; ++t) {
          const unsigned long long nx = sg + x[t];
          if (nx < sg) ovf = 1u;
          sg = nx;
          if ((dm[t] >> lane) & 1u)
            sl.plist[pc + (uint32_t)__popc(dm[t] & lanemask_lt())] = (uint16_t)(pk[t] & 0xFFFFu);
          pc += (uint32_t)__popc(dm[t]);
        }
        e += 4;
      }
      if (mine && v != s) sl.sig[v] = sg;
    }
    dmin = __reduce_min_sync(kFull, ndmin);
    lout = __reduce_min_sync(kFull, nlout);
    __syncwarp();
  }
  if (!want_delta) return true;

  // ---- backward: the steps in reverse order of settlement, one member per lane
  uint32_t hi = min(nord, n);
  while (hi > 0) {
    // the step holding position hi - 1 starts at the nearest step mark at or below it
    uint32_t lo = 0;
    for (int32_t top = (int32_t)hi - 1; top >= 0; top -= 32) {
      const int32_t p = top - (int32_t)lane;
      const bool mark = p >= 0 && (sl.ord[p] & kStepStart);
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
        v = sl.ord[k] & 0x7FFFu;
        dv = sl.dist[v] & kMask;
        e = H.rp[v];
        e1 = H.rp[v + 1];
        sg = sl.sig[v];
      }
      // the successors' rho in arc order: integral ones exactly, the others in DT
      uint32_t acc_i = 0;
      DT acc_f = 0;
      bool any_f = false;
      while (__any_sync(kFull, e < e1)) {
        uint32_t pk[4];
        uint64_t rw[4];
#pragma unroll
        for (int t = 0; t < 4; ++t) pk[t] = e + t < e1 ? H.arc[e + t] : 0u;
#pragma unroll
        for (int t = 0; t < 4; ++t) {
          const bool suc = e + t < e1 && (sl.dist[pk[t] & 0xFFFFu] & kMask) == dv + (pk[t] >> 16);
          rw[t] = suc ? sl.sig[pk[t] & 0xFFFFu] : kIntTag;   // kIntTag alone adds 0
        }
#pragma unroll
        for (int t = 0; t < 4; ++t) {
          if (rw[t] & kIntTag) {
            acc_i += (uint32_t)rw[t];
          } else {
            acc_f += *reinterpret_cast<const DT *>(&rw[t]);
            any_f = true;
          }
        }
        e += 4;
      }
      if (mine) {
        if (sg == 1ull && !any_f) {
          // delta(v) = sum of the successors' subtree sizes: exact in integers
          sl.sig[v] = kIntTag | (uint64_t)(1u + acc_i);
          if (v != s && acc_i) atomicAdd(&cs.a0[v], (unsigned long long)acc_i);
        } else {
          DT dep, rho;
          dependency<DT>(sg, (DT)acc_i + acc_f, dep, rho);
          uint64_t bits = 0;
          *reinterpret_cast<DT *>(&bits) = rho;
          sl.sig[v] = bits;
          if (v != s) fx_red(cs.a0, cs.a1, cs.a2, v, (double)dep);
        }
      }
    }
    __syncwarp();
    hi = lo;
  }
  return true;
}

// ---------------------------------------------------------------------------------------
// The persistent kernel.  Work item w enumerates (problem, realization) pairs of all
// problems; items are visited in strided order by the CTAs.  Inside a realization the source
// warps claim sources one at a time.
// ---------------------------------------------------------------------------------------
template <int BLOCK>
__global__ void __launch_bounds__(BLOCK, 1)
mc_counts_kernel(const McDev *__restrict__ probs, int nprob, const uint64_t *item_prefix,
                 uint64_t total_items, uint32_t nsw_launch, unsigned char *scratch,
                 size_t scratch_stride) {
  extern __shared__ __align__(16) unsigned char smem[];
  CtaHead *ctl = reinterpret_cast<CtaHead *>(smem);
  const uint32_t warp = threadIdx.x >> 5, lane = threadIdx.x & 31u;
  unsigned char *const my_scratch = scratch + (size_t)blockIdx.x * scratch_stride;
  for (uint64_t item = blockIdx.x; item < total_items; item += gridDim.x) {
    int g = 0;
    while (g + 1 < nprob && item_prefix[g + 1] <= item) ++g;
    const McDev &P = probs[g];
    // source warps: per problem in a batched launch (small graphs use more of the CTA's
    // warps), else the launch's value
    const uint32_t nsw = P.spt ? P.spt : nsw_launch;
    const uint32_t r_local = (uint32_t)(item - item_prefix[g]);
    uint32_t anchor;
    const uint32_t r = item_rho(P, r_local, anchor);
    const uint32_t n = P.n;
    StepLayout L;
    L.make(n, (uint32_t)(2 * P.m), nsw);
    uint32_t *rp = reinterpret_cast<uint32_t *>(smem + L.off_rp);
    uint32_t *arc = reinterpret_cast<uint32_t *>(smem + L.off_arc);
    uint16_t *mw = reinterpret_cast<uint16_t *>(smem + L.off_mw);
    CtaScratch cs;
    cs.carve(my_scratch, n);
    uint32_t *comp = cs.comp, *cinfo = cs.cinfo, *sel = cs.sel;
    uint16_t *src = cs.src;
    if (threadIdx.x == 0) {
      ctl->err = 0; ctl->ovf = 0; ctl->nsrc = 0; ctl->cursor = 0;
      ctl->edges = 0; ctl->verts = 0; ctl->wmax = 1;
    }
    __syncthreads();

    const bool ball = P.per_row && P.hop_radius;
    if (ball) hop_ball(P, anchor, cinfo);   // cinfo is free until the components
    realize_csr(P, r, rp, arc, ctl, ball ? cinfo : nullptr);
    Realized H{n, rp, arc};
    components(P, H, comp, cinfo);
    if (P.per_row) keep_anchor_component(n, anchor, comp, cinfo);
    min_lengths(H, mw);

    // sources: every node of a valid component (ascending), alive edges per root for TEPS
    uint32_t *cedges = sel;
    for (uint32_t v = threadIdx.x; v < n; v += blockDim.x) {
      cedges[v] = 0; cs.a0[v] = 0ull; cs.a1[v] = 0ull; cs.a2[v] = 0ull;
    }
    __syncthreads();
    for (uint32_t v = threadIdx.x; v < n; v += blockDim.x) {
      const uint32_t root = comp[v];
      if (!comp_valid(cinfo[root], P.k_min)) continue;
      uint32_t up = 0;
      for (uint32_t e = rp[v]; e < rp[v + 1]; ++e) up += ((arc[e] & 0xFFFFu) > v) ? 1u : 0u;
      if (up) atomicAdd(&cedges[root], up);
    }
    {
      const uint32_t per = (n + blockDim.x - 1) / blockDim.x;
      const uint32_t v0 = min(n, threadIdx.x * per), v1 = min(n, v0 + per);
      uint32_t cnt = 0;
      for (uint32_t v = v0; v < v1; ++v) cnt += comp_valid(cinfo[comp[v]], P.k_min) ? 1u : 0u;
      uint32_t off = block_exclusive_scan(cnt, ctl->scan, &ctl->scan_total);
      for (uint32_t v = v0; v < v1; ++v)
        if (comp_valid(cinfo[comp[v]], P.k_min)) src[off++] = (uint16_t)v;
      if (threadIdx.x == 0) ctl->nsrc = ctl->scan_total;
    }
    __syncthreads();
    {
      unsigned long long local = 0, lv = 0;
      for (uint32_t v = threadIdx.x; v < n; v += blockDim.x)
        if (comp[v] == v && comp_valid(cinfo[v], P.k_min)) {
          const unsigned long long sz = cinfo[v] & kSizeMask;
          local += sz * cedges[v];
          lv += sz * sz;
        }
      if (local) atomicAdd(&ctl->edges, local);
      if (lv) atomicAdd(&ctl->verts, lv);
    }
    __syncthreads();
    const uint32_t nsrc = ctl->nsrc;

    const bool fp32 = (P.precision == 1);
    const StepSlot s0 = L.slot(smem, 0, n);
    for (int attempt = 0; attempt < 2; ++attempt) {
      const bool use32 = fp32 && attempt == 0;
      if (attempt == 1) {
        for (uint32_t v = threadIdx.x; v < n; v += blockDim.x) {
          cs.a0[v] = 0ull; cs.a1[v] = 0ull; cs.a2[v] = 0ull;
        }
        if (threadIdx.x == 0) ctl->cursor = 0;
        __syncthreads();
      }
      if (warp < nsw) {
        const StepSlot sl = L.slot(smem, warp, n);
        uint32_t err = 0, ovf = 0;
        for (;;) {
          uint32_t k = 0;
          if (lane == 0) k = atomicAdd(&ctl->cursor, 1u);
          k = __shfl_sync(kFull, k, 0);
          if (k >= nsrc) break;
          const uint32_t s = src[k];
          const bool ok = use32 ? source_steps<float>(H, mw, sl, s, true, cs, err, ovf)
                                : source_steps<double>(H, mw, sl, s, true, cs, err, ovf);
          if (!ok) break;
        }
        err = __reduce_or_sync(kFull, err);
        ovf = __reduce_or_sync(kFull, ovf);
        if (lane == 0) {
          if (err) atomicOr(&ctl->err, err);
          if (ovf) atomicOr(&ctl->ovf, 1u);
        }
      }
      __syncthreads();
      fx_finalize3(cs.a0, cs.a1, cs.a2, n);   // betweenness as doubles, in a0's storage
      __syncthreads();
      SlotArrays scratch{};
      scratch.dist = s0.dist;
      scratch.sig = s0.sig;
      const bool recheck = select_and_count(P, r_local, comp, cinfo,
                                            reinterpret_cast<const double *>(cs.a0), scratch, sel,
                                            src, use32, ctl);
      __syncthreads();
      if (!recheck) break;
      if (threadIdx.x == 0 && P.stats) atomicAdd(u64p(&P.stats->rechecked), 1ull);
    }
    if (threadIdx.x == 0 && P.stats) {
      if (ctl->err) atomicOr(u64p(&P.stats->device_error), (unsigned long long)ctl->err);
      atomicAdd(u64p(&P.stats->realizations), 1ull);
      atomicAdd(u64p(&P.stats->sources), (unsigned long long)nsrc);
      atomicAdd(u64p(&P.stats->edge_visits), (unsigned long long)ctl->edges);
      atomicAdd(u64p(&P.stats->vertex_visits), (unsigned long long)ctl->verts);
      if (ctl->ovf) atomicAdd(u64p(&P.stats->overflow), 1ull);
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------------------
// Parity kernels
// ---------------------------------------------------------------------------------------
__global__ void debug_realize_kernel(McDev P, uint32_t r_count, uint8_t *alive, uint32_t *w) {
  const uint64_t total = (uint64_t)r_count * P.m;
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < total;
       i += (uint64_t)gridDim.x * blockDim.x) {
    const uint32_t k = (uint32_t)(i / P.m), e = (uint32_t)(i % P.m);
    bool al; uint32_t ww;
    edge_draw(P, P.r_begin + k, e, al, ww);
    alive[i] = al ? 1 : 0;
    w[i] = ww;
  }
}

// Shared memory of the component parity kernel: head, rp, arcs, comp, cinfo.
__host__ __device__ inline uint32_t components_smem_bytes(uint32_t n, uint32_t arcs) {
  return al16((uint32_t)sizeof(CtaHead)) + al16(4u * (n + 1)) + al16(4u * (arcs > 0 ? arcs : 1)) +
         2u * al16(4u * n);
}

__global__ void debug_components_kernel(McDev P, int32_t *comp_out, int32_t *csize_out) {
  extern __shared__ __align__(16) unsigned char smem[];
  CtaHead *ctl = reinterpret_cast<CtaHead *>(smem);
  const uint32_t n0 = (uint32_t)P.n, arcs = (uint32_t)(2 * P.m);
  unsigned char *p = smem + al16((uint32_t)sizeof(CtaHead));
  uint32_t *rp = reinterpret_cast<uint32_t *>(p);     p += al16(4u * (n0 + 1));
  uint32_t *arc = reinterpret_cast<uint32_t *>(p);    p += al16(4u * (arcs > 0 ? arcs : 1));
  uint32_t *comp = reinterpret_cast<uint32_t *>(p);   p += al16(4u * n0);
  uint32_t *cinfo = reinterpret_cast<uint32_t *>(p);
  const uint32_t k = blockIdx.x;
  if (threadIdx.x == 0) { ctl->err = 0; ctl->wmax = 1; }
  __syncthreads();
  realize_csr(P, P.r_begin + k, rp, arc, ctl);
  Realized H{(uint32_t)P.n, rp, arc};
  components(P, H, comp, cinfo);
  for (uint32_t v = threadIdx.x; v < (uint32_t)P.n; v += blockDim.x) {
    comp_out[(size_t)k * P.n + v] = (int32_t)comp[v];
    csize_out[(size_t)k * P.n + v] = (int32_t)(cinfo[comp[v]] & kSizeMask);
  }
}

// Distances and path counts of given sources from the production forward routine: warp w of
// CTA b handles source b * nsw + w of the list on realization r.
template <int BLOCK>
__global__ void __launch_bounds__(BLOCK, 1)
debug_sssp_kernel(McDev P, uint32_t r, const int32_t *sources, int32_t nsrc, uint32_t nsw,
                  uint32_t *dist_out, uint64_t *sigma_out) {
  extern __shared__ __align__(16) unsigned char smem[];
  CtaHead *ctl = reinterpret_cast<CtaHead *>(smem);
  const uint32_t n = P.n, warp = threadIdx.x >> 5, lane = threadIdx.x & 31u;
  StepLayout L;
  L.make(n, (uint32_t)(2 * P.m), nsw);
  uint32_t *rp = reinterpret_cast<uint32_t *>(smem + L.off_rp);
  uint32_t *arc = reinterpret_cast<uint32_t *>(smem + L.off_arc);
  uint16_t *mw = reinterpret_cast<uint16_t *>(smem + L.off_mw);
  if (threadIdx.x == 0) { ctl->err = 0; ctl->ovf = 0; ctl->wmax = 1; }
  __syncthreads();
  realize_csr(P, r, rp, arc, ctl);
  Realized H{n, rp, arc};
  min_lengths(H, mw);
  __syncthreads();
  const uint32_t k = blockIdx.x * nsw + warp;
  if (warp < nsw && k < (uint32_t)nsrc) {
    const int32_t sv = sources[k];
    const uint32_t s = (sv >= 0 && (uint32_t)sv < n) ? (uint32_t)sv : 0u;
    const StepSlot sl = L.slot(smem, warp, n);
    uint32_t err = 0, ovf = 0;
    source_steps<double>(H, mw, sl, s, false, CtaScratch{}, err, ovf);
    err = __reduce_or_sync(kFull, err);
    ovf = __reduce_or_sync(kFull, ovf);
    if (lane == 0) {
      if (err) atomicOr(&ctl->err, err);
      if (ovf) atomicOr(&ctl->ovf, 1u);
    }
    for (uint32_t v = lane; v < n; v += 32) {
      const uint32_t d = sl.dist[v] & kMask;
      const bool reached = d < kInf;
      dist_out[(size_t)k * n + v] = reached ? d : 0xFFFFFFFFu;
      sigma_out[(size_t)k * n + v] = reached ? sl.sig[v] : 0ull;
    }
  }
  __syncthreads();
  if (threadIdx.x == 0 && P.stats) {
    if (ctl->err) atomicOr(u64p(&P.stats->device_error), (unsigned long long)ctl->err);
    if (ctl->ovf) atomicAdd(u64p(&P.stats->overflow), 1ull);
  }
}

// ---------------------------------------------------------------------------------------
// Host-side launch helpers (called from the C ABI)
// ---------------------------------------------------------------------------------------
uint32_t mc_layout_bytes(uint32_t n, uint64_t arcs, uint32_t nsw) {
  StepLayout L;
  L.make(n, (uint32_t)arcs, nsw);
  return L.total;
}

size_t mc_cta_scratch_bytes(uint32_t n) { return CtaScratch::bytes(n); }

#define AFC_MC_BLOCKS(X) X(256) X(512) X(1024)

template <int BLOCK>
static cudaError_t launch_counts_t(const McDev *probs_dev, int nprob, const uint64_t *prefix_dev,
                                   uint64_t total_items, uint32_t nsw, uint32_t smem,
                                   uint32_t grid, unsigned char *scratch, size_t stride,
                                   cudaStream_t stream) {
  cudaFuncSetAttribute(mc_counts_kernel<BLOCK>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  mc_counts_kernel<BLOCK><<<grid, BLOCK, smem, stream>>>(probs_dev, nprob, prefix_dev,
                                                         total_items, nsw, scratch, stride);
  return cudaGetLastError();
}

cudaError_t launch_mc_counts(int block, const McDev *probs_dev, int nprob,
                             const uint64_t *prefix_dev, uint64_t total_items,
                             uint32_t source_warps, uint32_t smem_bytes, uint32_t grid,
                             unsigned char *scratch, size_t scratch_stride, cudaStream_t stream) {
  if (source_warps < 1 || source_warps > (uint32_t)block / 32u) return cudaErrorInvalidValue;
#define AFC_X(B)                                                                       \
  if (block == B)                                                                      \
    return launch_counts_t<B>(probs_dev, nprob, prefix_dev, total_items, source_warps, \
                              smem_bytes, grid, scratch, scratch_stride, stream);
  AFC_MC_BLOCKS(AFC_X)
#undef AFC_X
  return cudaErrorInvalidValue;
}

cudaError_t launch_debug_realize(const McDev &P, uint32_t r_count, uint8_t *alive, uint32_t *w,
                                 cudaStream_t stream) {
  const uint64_t total = (uint64_t)r_count * P.m;
  if (total == 0) return cudaSuccess;
  const uint64_t want = (total + 255) / 256;
  const uint32_t grid = (uint32_t)(want < 4096 ? want : 4096);
  debug_realize_kernel<<<grid, 256, 0, stream>>>(P, r_count, alive, w);
  return cudaGetLastError();
}

cudaError_t launch_debug_components(const McDev &P, uint32_t r_count, int32_t *comp, int32_t *csize,
                                    cudaStream_t stream) {
  const uint32_t smem = components_smem_bytes(P.n, (uint32_t)(2 * P.m));
  cudaFuncSetAttribute(debug_components_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  debug_components_kernel<<<r_count, 256, smem, stream>>>(P, comp, csize);
  return cudaGetLastError();
}

template <int BLOCK>
static cudaError_t launch_sssp_t(const McDev &P, uint32_t r, const int32_t *sources, int32_t nsrc,
                                 uint32_t nsw, uint32_t smem, uint32_t *dist, uint64_t *sigma,
                                 cudaStream_t stream) {
  const uint32_t grid = (uint32_t)((nsrc + (int32_t)nsw - 1) / (int32_t)nsw);
  cudaFuncSetAttribute(debug_sssp_kernel<BLOCK>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  debug_sssp_kernel<BLOCK><<<grid, BLOCK, smem, stream>>>(P, r, sources, nsrc, nsw, dist, sigma);
  return cudaGetLastError();
}

cudaError_t launch_debug_sssp(int block, const McDev &P, uint32_t r, const int32_t *sources,
                              int32_t nsrc, uint32_t source_warps, uint32_t smem, uint32_t *dist,
                              uint64_t *sigma, cudaStream_t stream) {
  if (source_warps < 1 || source_warps > (uint32_t)block / 32u) return cudaErrorInvalidValue;
#define AFC_X(B)                                                                                 \
  if (block == B)                                                                                \
    return launch_sssp_t<B>(P, r, sources, nsrc, source_warps, smem, dist, sigma, stream);
  AFC_MC_BLOCKS(AFC_X)
#undef AFC_X
  return cudaErrorInvalidValue;
}

}  // namespace afc
