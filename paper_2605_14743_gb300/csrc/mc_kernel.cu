// mc_kernel.cu -- Monte Carlo transition counts on GB300 (sm_103a).
//
// One CTA owns one network realization at a time (persistent over realizations) and keeps
// the whole realization in shared memory:
//   A1  Philox4x32-10 edge draws -> alive-compacted CSR with packed (neighbour, length) arcs
//   A2  components by lock-free union-find (root = smallest id), sizes, candidate flags
//   A3  per source: bucketed (Delta-stepping) integer SSSP over a shared-memory frontier
//   A4  shortest-path counts sigma (exact 64-bit) resolved bucket by bucket
//   A5  dependencies delta in reverse bucket order, betweenness accumulated in FP64
//   A6  tie-ruled argmax per valid component (Sec. 3.2 eq. local-center, Sec. 7.1 Sel_W)
//       and the transition-count update of every anchor (Alg. 1 / Alg. 2)
//   A7  FP32 mode: a realization whose top-two gap is under the margin is redone in FP64
// Several thread groups of G threads each process different sources of the realization
// concurrently; each group owns its per-source state (dist, sigma, delta, bucket lists).
#include <cstdint>
#include <cuda_runtime.h>

#include "afc_device.cuh"
#include "afc_internal.h"

namespace afc {

__device__ __forceinline__ unsigned long long *u64p(uint64_t *p) {
  return reinterpret_cast<unsigned long long *>(p);
}

constexpr uint32_t kInf = 0x7FFFFFFFu;    // unreached distance
constexpr uint32_t kFlag = 0x80000000u;   // "sigma final" (forward) / "delta pending" (backward)
constexpr uint32_t kMask = 0x7FFFFFFFu;
constexpr uint16_t kMark = 0x8000u;       // finalise-this-member mark in the bucket lists
constexpr uint64_t kNoRelax = ~0ull;

// Shared-memory (or global-slab) layout of one CTA for a graph of n nodes and 2m arcs.
struct Layout {
  uint32_t off_rp, off_arc, off_comp, off_cinfo, off_bc, off_src, off_groups, group_bytes, total;
  __host__ __device__ static uint32_t al(uint32_t x) { return (x + 15u) & ~15u; }
  __host__ __device__ void make(uint32_t n, uint32_t arcs, uint32_t ngroups) {
    uint32_t o = al(sizeof(CtaCtl));
    off_rp = o;     o = al(o + 4u * (n + 1));
    off_arc = o;    o = al(o + 4u * (arcs > 0 ? arcs : 1));
    off_comp = o;   o = al(o + 4u * n);
    off_cinfo = o;  o = al(o + 4u * n);
    off_bc = o;     o = al(o + 8u * n);
    off_src = o;    o = al(o + 2u * n);
    off_groups = o;
    group_bytes = al(4u * n) + al(8u * n) + al(8u * n) + al(2u * n) + al(2u * n);
    total = o + ngroups * group_bytes;
  }
};

struct GroupArrays {
  uint32_t *dist;   // [n] distance | flag
  uint64_t *sig;    // [n] last relaxed distance during SSSP, then sigma
  double *dlt;      // [n] rho = (1 + delta) / sigma (FP64) or float pairs (FP32)
  uint16_t *ord;    // [n] settled vertices in bucket order (+ current bucket)
  uint16_t *pend;   // [n] discovered vertices beyond the current bucket
};

__device__ __forceinline__ GroupArrays group_arrays(unsigned char *base, const Layout &L,
                                                    uint32_t n, uint32_t g) {
  unsigned char *p = base + L.off_groups + g * L.group_bytes;
  GroupArrays a;
  a.dist = reinterpret_cast<uint32_t *>(p);  p += Layout::al(4u * n);
  a.sig = reinterpret_cast<uint64_t *>(p);   p += Layout::al(8u * n);
  a.dlt = reinterpret_cast<double *>(p);     p += Layout::al(8u * n);
  a.ord = reinterpret_cast<uint16_t *>(p);   p += Layout::al(2u * n);
  a.pend = reinterpret_cast<uint16_t *>(p);
  return a;
}

struct Realized {
  uint32_t n;
  const uint32_t *rp;    // [n+1] alive-compacted row offsets
  const uint32_t *arc;   // packed: neighbour (low 16 bits) | length << 16
};

// ---------------------------------------------------------------------------------------
// One source: distances, path counts, dependencies; adds delta_s(v) to bc[v] (v != s).
// Returns false on a detected consistency failure (error bits are OR-ed into *err).
// ---------------------------------------------------------------------------------------
template <int G, typename DT>
__device__ bool brandes_one_source(Group<G> &grp, const Realized &H, GroupArrays a,
                                   GroupCtl *gc, uint32_t s, uint32_t delta, double *bc,
                                   bool want_delta, uint32_t *err, uint32_t *ovf) {
  const uint32_t n = H.n;
  const uint32_t t = grp.rank;
  for (uint32_t v = t; v < n; v += G) a.dist[v] = kInf;
  grp.sync();
  if (t == 0) {
    a.dist[s] = 0;
    a.pend[0] = (uint16_t)s;
    gc->npend = 1;
    gc->nm = 0;
  }
  grp.sync();

  uint32_t nset = 0;
  uint32_t my_err = 0, my_ovf = 0;
  bool ok = true;
  for (uint32_t guard = 0;; ++guard) {
    if (guard > n + 1) { my_err |= kErrPassLimit; ok = false; break; }
    // (1) smallest live tentative distance among the pending vertices
    const uint32_t np = gc->npend;
    uint32_t local = kInf;
    for (uint32_t i = t; i < np; i += G) {
      const uint32_t d = a.dist[a.pend[i]];
      if (!(d & kFlag) && d < local) local = d;   // flagged entries are settled (stale)
    }
    const uint32_t dmin = grp.reduce_min(local);
    if (dmin >= kInf) break;
    const uint32_t dstart = (dmin / delta) * delta;
    const uint32_t dend = dstart + delta;
    // (2) move pending vertices of [dstart, dend) into the bucket, drop stale entries,
    //     compact the rest in place (chunk reads complete before any chunk write)
    if (t == 0) gc->npend_next = 0;
    grp.sync();
    for (uint32_t base = 0; base < np; base += G) {
      const uint32_t i = base + t;
      uint32_t v = 0, d = kInf;
      if (i < np) { v = a.pend[i]; d = a.dist[v]; }
      grp.sync();
      if (i < np && !(d & kFlag)) {
        if (d < dend) {
          const uint32_t pos = warp_append(&gc->nm);
          if (pos < n) { a.ord[pos] = (uint16_t)v; a.sig[v] = kNoRelax; }
          else my_err |= kErrCapacity;
        } else {
          const uint32_t pos = warp_append(&gc->npend_next);
          a.pend[pos] = (uint16_t)v;
        }
      }
    }
    grp.sync();
    if (t == 0) gc->npend = gc->npend_next;
    // (3) relaxation passes inside the bucket until no member improves
    const uint32_t mstart = nset;
    for (uint32_t pass = 0;; ++pass) {
      if (pass > n + 1) { my_err |= kErrPassLimit; ok = false; break; }
      const uint32_t nm = gc->nm;
      grp.sync();  // everyone holds the same member count before anyone appends
      bool relaxed = false;
      for (uint32_t idx = mstart + t; idx < nm; idx += G) {
        const uint32_t v = a.ord[idx];
        const uint32_t d = a.dist[v];
        if ((uint64_t)d == a.sig[v]) continue;
        a.sig[v] = d;
        relaxed = true;
        const uint32_t e1 = H.rp[v + 1];
        for (uint32_t e = H.rp[v]; e < e1; ++e) {
          const uint32_t pk = H.arc[e];
          const uint32_t u = pk & 0xFFFFu;
          const uint32_t nd = d + (pk >> 16);
          const uint32_t cur = a.dist[u];
          if ((cur & kFlag) || nd >= cur) continue;
          const uint32_t old = atomicMin(&a.dist[u], nd);
          if (nd >= old) continue;
          if (nd < dend) {
            if (old >= dend) {
              const uint32_t pos = warp_append(&gc->nm);
              if (pos < n) { a.ord[pos] = (uint16_t)u; a.sig[u] = kNoRelax; }
              else my_err |= kErrCapacity;
            }
          } else if (old == kInf) {
            const uint32_t pos = warp_append(&gc->npend);
            if (pos < n) a.pend[pos] = (uint16_t)u;
            else my_err |= kErrCapacity;
          }
        }
      }
      if (!grp.any(relaxed)) break;
    }
    if (!ok) break;
    // (4) path counts of the bucket: a member is final once all its same-bucket
    //     predecessors are final (earlier buckets are final already)
    const uint32_t mend = min(gc->nm, n);
    for (uint32_t idx = mstart + t; idx < mend; idx += G) {
      const uint32_t v = a.ord[idx];
      a.sig[v] = (v == s) ? 1ull : 0ull;
    }
    grp.sync();
    for (uint32_t pass = 0;; ++pass) {
      if (pass > mend - mstart + 1) { my_err |= kErrPassLimit; ok = false; break; }
      bool open = false;
      for (uint32_t idx = mstart + t; idx < mend; idx += G) {
        const uint32_t v = a.ord[idx];
        const uint32_t dv = a.dist[v];
        if (dv & kFlag) continue;
        uint64_t acc = (v == s) ? 1ull : 0ull;
        bool all_final = true;
        if (v != s) {
          const uint32_t e1 = H.rp[v + 1];
          for (uint32_t e = H.rp[v]; e < e1; ++e) {
            const uint32_t pk = H.arc[e];
            const uint32_t u = pk & 0xFFFFu;
            const uint32_t du = a.dist[u];
            if ((du & kMask) + (pk >> 16) != dv) continue;
            const uint64_t su = a.sig[u];
            const uint64_t nx = acc + su;
            if (nx < acc) my_ovf = 1;
            acc = nx;
            if (!(du & kFlag)) all_final = false;
          }
        }
        a.sig[v] = acc;
        if (all_final) a.ord[idx] = (uint16_t)(v | kMark);
        else open = true;
      }
      grp.sync();
      for (uint32_t idx = mstart + t; idx < mend; idx += G) {
        const uint32_t e = a.ord[idx];
        if (e & kMark) {
          a.ord[idx] = (uint16_t)(e & ~kMark);
          a.dist[e & ~kMark] |= kFlag;
        }
      }
      if (!grp.any(open)) break;
    }
    if (!ok) break;
    nset = mend;
  }
  if (!ok) {
    atomicOr(err, my_err);
    return false;
  }

  // (5) dependencies, buckets in reverse order; kFlag now means "delta still pending"
  if (want_delta) {
    uint32_t hi = nset;
    while (hi > 0) {
      const uint32_t bid = (a.dist[a.ord[hi - 1]] & kMask) / delta;
      uint32_t lo = 0;
      for (uint32_t top = hi; top > 0;) {
        const uint32_t base = top > G ? top - G : 0;
        const uint32_t i = base + t;
        uint32_t cand = 0;
        if (i < top && (a.dist[a.ord[i]] & kMask) / delta != bid) cand = i + 1;
        const uint32_t found = grp.reduce_max(cand);
        if (found > 0) { lo = found; break; }
        top = base;
      }
      for (uint32_t pass = 0;; ++pass) {
        if (pass > hi - lo + 1) { my_err |= kErrPassLimit; ok = false; break; }
        bool open = false;
        for (uint32_t idx = lo + t; idx < hi; idx += G) {
          const uint32_t v = a.ord[idx];
          const uint32_t dv = a.dist[v];
          if (!(dv & kFlag)) continue;
          const uint32_t dvm = dv & kMask;
          DT acc = 0;
          bool all_final = true;
          const uint32_t e1 = H.rp[v + 1];
          for (uint32_t e = H.rp[v]; e < e1; ++e) {
            const uint32_t pk = H.arc[e];
            const uint32_t w = pk & 0xFFFFu;
            const uint32_t dw = a.dist[w];
            if ((dw & kMask) != dvm + (pk >> 16)) continue;
            acc += reinterpret_cast<const DT *>(a.dlt)[w];
            if (dw & kFlag) all_final = false;
          }
          if (all_final) {
            const DT sv = (DT)a.sig[v];
            const DT dep = sv * acc;
            reinterpret_cast<DT *>(a.dlt)[v] = ((DT)1 + dep) / sv;
            if (v != s) atomicAdd(&bc[v], (double)dep);
            a.ord[idx] = (uint16_t)(v | kMark);
          } else {
            open = true;
          }
        }
        grp.sync();
        for (uint32_t idx = lo + t; idx < hi; idx += G) {
          const uint32_t e = a.ord[idx];
          if (e & kMark) {
            a.ord[idx] = (uint16_t)(e & ~kMark);
            a.dist[e & ~kMark] &= kMask;
          }
        }
        if (!grp.any(open)) break;
      }
      if (!ok) break;
      hi = lo;
    }
  }
  if (my_err) atomicOr(err, my_err);
  if (my_ovf) atomicOr(ovf, 1u);
  grp.sync();
  return ok;
}

// ---------------------------------------------------------------------------------------
// CTA-wide pieces: realization (A1), components (A2)
// ---------------------------------------------------------------------------------------
__device__ __forceinline__ uint32_t block_exclusive_scan(uint32_t x, uint32_t *tmp,
                                                         uint32_t *total) {
  const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
  const uint32_t nw = (blockDim.x + 31u) >> 5;
  uint32_t inc = x;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(kFull, inc, o);
    if (lane >= (uint32_t)o) inc += y;
  }
  if (lane == 31) tmp[warp] = inc;
  __syncthreads();
  if (warp == 0) {
    uint32_t wv = lane < nw ? tmp[lane] : 0u;
    uint32_t wi = wv;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(kFull, wi, o);
      if (lane >= (uint32_t)o) wi += y;
    }
    if (lane < nw) tmp[lane] = wi - wv;
    if (lane == nw - 1) *total = wi;
  }
  __syncthreads();
  const uint32_t r = tmp[warp] + inc - x;
  __syncthreads();
  return r;
}

__device__ __forceinline__ void edge_draw(const McDev &P, uint32_t r, uint32_t e, bool &alive,
                                          uint32_t &w) {
  const uint4 u = philox4x32_10(make_uint4(e, r, P.graph_tag, 0u), P.key_lo, P.key_hi);
  const uint64_t T = P.thresh ? P.thresh[e] : P.thresh_all;
  const uint32_t lo = P.w_lo ? P.w_lo[e] : P.w_lo_all;
  const uint32_t hi = P.w_hi ? P.w_hi[e] : P.w_hi_all;
  alive = (uint64_t)u.x < T;
  w = lo + (uint32_t)(((uint64_t)u.y * ((uint64_t)hi - lo + 1u)) >> 32);
}

// Builds the alive-compacted CSR of realization r into rp/arc.  Thread-per-vertex over
// contiguous vertex ranges so that the offsets come from one block scan.
__device__ void realize_csr(const McDev &P, uint32_t r, uint32_t *rp, uint32_t *arc,
                            CtaCtl *ctl, uint32_t *err) {
  const uint32_t n = P.n;
  const uint32_t cap = (uint32_t)(2 * P.m);   // arc slots reserved in the layout
  const uint32_t T = blockDim.x;
  const uint32_t per = (n + T - 1) / T;
  const uint32_t v0 = min(n, threadIdx.x * per), v1 = min(n, v0 + per);
  uint32_t cnt = 0;
  for (uint32_t v = v0; v < v1; ++v) {
    const int32_t a0 = P.row_ptr[v], a1 = P.row_ptr[v + 1];
    for (int32_t a = a0; a < a1; ++a) {
      const uint32_t e = (uint32_t)P.eid[a];
      if (e >= (uint64_t)P.m) continue;
      bool alive; uint32_t w;
      edge_draw(P, r, e, alive, w);
      cnt += alive ? 1u : 0u;
    }
  }
  uint32_t off = block_exclusive_scan(cnt, ctl->scan, &ctl->scan_total);
  for (uint32_t v = v0; v < v1; ++v) {
    rp[v] = off;
    const int32_t a0 = P.row_ptr[v], a1 = P.row_ptr[v + 1];
    for (int32_t a = a0; a < a1; ++a) {
      const uint32_t e = (uint32_t)P.eid[a];
      const uint32_t u = (uint32_t)P.col[a];
      if (e >= (uint64_t)P.m || u >= n) { atomicOr(err, kErrInput); continue; }
      bool alive; uint32_t w;
      edge_draw(P, r, e, alive, w);
      if (!alive) continue;
      if (w == 0 || w > 0xFFFFu || off >= cap) { atomicOr(err, kErrInput); continue; }
      arc[off++] = u | (w << 16);
    }
  }
  const uint32_t total = ctl->scan_total;
  if (threadIdx.x == 0) rp[n] = total < cap ? total : cap;
  __syncthreads();
}

__device__ __forceinline__ uint32_t uf_find(const uint32_t *parent, uint32_t x) {
  uint32_t p = parent[x];
  while (p != x) {
    x = p;
    p = parent[x];
  }
  return x;
}

// comp[v] <- smallest id of v's component; cinfo[root] <- size | has-candidate bit.
__device__ void components(const McDev &P, const Realized &H, uint32_t *comp, uint32_t *cinfo) {
  const uint32_t n = H.n;
  for (uint32_t v = threadIdx.x; v < n; v += blockDim.x) { comp[v] = v; cinfo[v] = 0; }
  __syncthreads();
  for (uint32_t v = threadIdx.x; v < n; v += blockDim.x) {
    for (uint32_t e = H.rp[v]; e < H.rp[v + 1]; ++e) {
      const uint32_t u = H.arc[e] & 0xFFFFu;
      if (u <= v) continue;
      uint32_t a = v, b = u;
      for (;;) {
        a = uf_find(comp, a);
        b = uf_find(comp, b);
        if (a == b) break;
        if (a > b) { const uint32_t t = a; a = b; b = t; }
        if (atomicCAS(&comp[b], b, a) == b) break;  // hook the larger root under the smaller
      }
    }
  }
  __syncthreads();
  for (uint32_t v = threadIdx.x; v < n; v += blockDim.x) comp[v] = uf_find(comp, v);
  __syncthreads();
  for (uint32_t v = threadIdx.x; v < n; v += blockDim.x) {
    const uint32_t root = comp[v];
    const bool cand = (P.in_w == nullptr) || P.in_w[v];
    atomicAdd(&cinfo[root], 1u);
    if (cand) atomicOr(&cinfo[root], kHasCand);
  }
  __syncthreads();
}

__device__ __forceinline__ bool comp_valid(uint32_t info, uint32_t k_min) {
  return (info & kHasCand) && (info & kSizeMask) >= k_min;
}

// ---------------------------------------------------------------------------------------
// Select (A6) and count.  Per-root scratch borrows group 0's arrays.
// Returns true when the FP32 gap test asks for an FP64 recheck.
// ---------------------------------------------------------------------------------------
__device__ bool select_and_count(const McDev &P, uint32_t r_local, const uint32_t *comp,
                                 const uint32_t *cinfo, const double *bc, GroupArrays s0,
                                 bool gap_test, bool commit, CtaCtl *ctl) {
  const uint32_t n = P.n;
  unsigned long long *best = reinterpret_cast<unsigned long long *>(s0.sig);   // max over X
  unsigned long long *bestK = reinterpret_cast<unsigned long long *>(s0.dlt);  // max over K
  uint32_t *centre = s0.dist;
  uint32_t *rank = reinterpret_cast<uint32_t *>(s0.ord);  // 2n bytes + 2n bytes of pend: 4n
  uint32_t &need_recheck = ctl->need_recheck;
  if (threadIdx.x == 0) need_recheck = 0;
  for (uint32_t v = threadIdx.x; v < n; v += blockDim.x) {
    best[v] = 0ull; bestK[v] = 0ull; centre[v] = 0xFFFFFFFFu; rank[v] = 1u;
  }
  __syncthreads();
  for (uint32_t v = threadIdx.x; v < n; v += blockDim.x) {
    const uint32_t root = comp[v];
    if (!comp_valid(cinfo[root], P.k_min)) continue;
    const unsigned long long bits = (unsigned long long)__double_as_longlong(bc[v]);
    if (P.top_k) atomicMax(&bestK[root], bits);
    if (P.in_w == nullptr || P.in_w[v]) atomicMax(&best[root], bits);
  }
  __syncthreads();
  for (uint32_t v = threadIdx.x; v < n; v += blockDim.x) {
    const uint32_t root = comp[v];
    if (!comp_valid(cinfo[root], P.k_min)) continue;
    if (!(P.in_w == nullptr || P.in_w[v])) continue;
    const double bstar = __longlong_as_double((long long)best[root]);
    if (bc[v] >= bstar - P.tie_rel * bstar) atomicMin(&centre[root], v);
  }
  __syncthreads();
  if (P.top_k || gap_test) {
    for (uint32_t v = threadIdx.x; v < n; v += blockDim.x) {
      const uint32_t root = comp[v];
      if (!comp_valid(cinfo[root], P.k_min)) continue;
      const uint32_t c = centre[root];
      if (c == v || c >= n) continue;
      if (P.top_k) {
        const double tauK = P.tie_rel * __longlong_as_double((long long)bestK[root]);
        const double diff = bc[v] - bc[c];
        if (diff > tauK || (fabs(diff) <= tauK && v < c)) atomicAdd(&rank[root], 1u);
      }
      if (gap_test && (P.top_k || P.in_w == nullptr || P.in_w[v])) {
        // top-two gap of the candidate set (of the whole component when a rank cutoff is
        // active): another node within the margin of B1 sends the realization to FP64
        const double b1 = bc[c];
        if (b1 > 0.0 && fabs(b1 - bc[v]) < P.recheck_margin * b1) need_recheck = 1;
      }
    }
    __syncthreads();
  }
  const bool recheck = gap_test && need_recheck;
  if (recheck || !commit) return recheck;
  uint32_t *counts = P.counts;
  const size_t stride = (size_t)n + 1;
  for (uint32_t i = threadIdx.x; i < n; i += blockDim.x) {
    const uint32_t root = comp[i];
    uint32_t col = n;
    if (comp_valid(cinfo[root], P.k_min)) {
      const uint32_t c = centre[root];
      if (c < n && (P.top_k == 0 || rank[root] <= P.top_k)) col = c;
    }
    atomicAdd(&counts[(size_t)i * stride + col], 1u);
    if (P.dump_next) P.dump_next[(size_t)r_local * n + i] = (int32_t)col;
  }
  if (P.dump_bc)
    for (uint32_t v = threadIdx.x; v < n; v += blockDim.x)
      P.dump_bc[(size_t)r_local * n + v] = bc[v];
  return false;
}

// ---------------------------------------------------------------------------------------
// The persistent kernel.  Work item w enumerates (problem, realization) pairs of all
// problems; items are visited in strided order by the CTAs.
// ---------------------------------------------------------------------------------------
template <int G>
__global__ void __launch_bounds__(1024, 1)
mc_counts_kernel(const McDev *__restrict__ probs, int nprob, const uint64_t *item_prefix,
                 uint64_t total_items, unsigned char *gslab, uint32_t slab_bytes,
                 uint32_t ngroups) {
  extern __shared__ __align__(16) unsigned char smem[];
  unsigned char *base = gslab ? gslab + (size_t)blockIdx.x * slab_bytes : smem;
  CtaCtl *ctl = reinterpret_cast<CtaCtl *>(smem);  // control block always in shared memory
  const uint32_t gidx = threadIdx.x / G;
  const bool in_group = gidx < ngroups;
  Group<G> grp;
  grp.idx = gidx;
  grp.rank = threadIdx.x % G;
  grp.red = ctl->gred[gidx < kMaxGroups ? gidx : 0];
  grp.turn = 0;

  for (uint64_t item = blockIdx.x; item < total_items; item += gridDim.x) {
    int g = 0;
    while (g + 1 < nprob && item_prefix[g + 1] <= item) ++g;
    const McDev &P = probs[g];
    const uint32_t r_local = (uint32_t)(item - item_prefix[g]);
    const uint32_t r = P.r_begin + r_local;
    const uint32_t n = P.n;
    Layout L;
    L.make(n, (uint32_t)(2 * P.m), ngroups);
    uint32_t *rp = reinterpret_cast<uint32_t *>(base + L.off_rp);
    uint32_t *arc = reinterpret_cast<uint32_t *>(base + L.off_arc);
    uint32_t *comp = reinterpret_cast<uint32_t *>(base + L.off_comp);
    uint32_t *cinfo = reinterpret_cast<uint32_t *>(base + L.off_cinfo);
    double *bc = reinterpret_cast<double *>(base + L.off_bc);
    uint16_t *src = reinterpret_cast<uint16_t *>(base + L.off_src);
    if (threadIdx.x < kMaxGroups * 3) (&ctl->gred[0][0])[threadIdx.x] = 0xFFFFFFFFu;
    if (threadIdx.x == 0) { ctl->err = 0; ctl->ovf = 0; ctl->nsrc = 0; ctl->cursor = 0; ctl->edges = 0; ctl->verts = 0; }
    __syncthreads();

    realize_csr(P, r, rp, arc, ctl, &ctl->err);
    Realized H{n, rp, arc};
    components(P, H, comp, cinfo);

    // sources: every node of a valid component; alive edges per root for the TEPS count
    GroupArrays g0 = group_arrays(base, L, n, 0);
    uint32_t *cedges = g0.dist;
    for (uint32_t v = threadIdx.x; v < n; v += blockDim.x) { cedges[v] = 0; bc[v] = 0.0; }
    __syncthreads();
    for (uint32_t v = threadIdx.x; v < n; v += blockDim.x) {
      const uint32_t root = comp[v];
      if (!comp_valid(cinfo[root], P.k_min)) continue;
      src[atomicAdd(&ctl->nsrc, 1u)] = (uint16_t)v;
      uint32_t up = 0;
      for (uint32_t e = rp[v]; e < rp[v + 1]; ++e) up += ((arc[e] & 0xFFFFu) > v) ? 1u : 0u;
      if (up) atomicAdd(&cedges[root], up);
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
    for (int attempt = 0; attempt < 2; ++attempt) {
      const bool use32 = fp32 && attempt == 0;
      if (attempt == 1) {
        for (uint32_t v = threadIdx.x; v < n; v += blockDim.x) bc[v] = 0.0;
        if (threadIdx.x == 0) ctl->cursor = 0;
        __syncthreads();
      }
      if (in_group) {
        GroupArrays ga = group_arrays(base, L, n, gidx);
        GroupCtl *gc = &ctl->gctl[gidx];
        for (;;) {
          if (grp.rank == 0) gc->claim = atomicAdd(&ctl->cursor, 1u);
          grp.sync();
          const uint32_t k = gc->claim;
          grp.sync();
          if (k >= nsrc) break;
          const uint32_t s = src[k];
          if (use32)
            brandes_one_source<G, float>(grp, H, ga, gc, s, P.delta, bc, true, &ctl->err, &ctl->ovf);
          else
            brandes_one_source<G, double>(grp, H, ga, gc, s, P.delta, bc, true, &ctl->err, &ctl->ovf);
        }
      }
      __syncthreads();
      const bool recheck = select_and_count(P, r_local, comp, cinfo, bc, g0, use32, true, ctl);
      __syncthreads();
      if (!recheck) break;
      if (threadIdx.x == 0 && P.stats) atomicAdd(u64p(&P.stats->rechecked), 1ull);
    }
    if (threadIdx.x == 0) {
      if (ctl->err && P.stats) atomicOr(u64p(&P.stats->device_error), (unsigned long long)ctl->err);
      if (P.stats) {
        atomicAdd(u64p(&P.stats->realizations), 1ull);
        atomicAdd(u64p(&P.stats->sources), (unsigned long long)nsrc);
        atomicAdd(u64p(&P.stats->edge_visits), (unsigned long long)ctl->edges);
        atomicAdd(u64p(&P.stats->vertex_visits), (unsigned long long)ctl->verts);
        if (ctl->ovf) atomicAdd(u64p(&P.stats->overflow), 1ull);
      }
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

__global__ void debug_components_kernel(McDev P, uint32_t ngroups, int32_t *comp_out,
                                        int32_t *csize_out) {
  extern __shared__ __align__(16) unsigned char smem[];
  CtaCtl *ctl = reinterpret_cast<CtaCtl *>(smem);
  Layout L;
  L.make(P.n, (uint32_t)(2 * P.m), 0);
  uint32_t *rp = reinterpret_cast<uint32_t *>(smem + L.off_rp);
  uint32_t *arc = reinterpret_cast<uint32_t *>(smem + L.off_arc);
  uint32_t *comp = reinterpret_cast<uint32_t *>(smem + L.off_comp);
  uint32_t *cinfo = reinterpret_cast<uint32_t *>(smem + L.off_cinfo);
  const uint32_t k = blockIdx.x;
  if (threadIdx.x == 0) ctl->err = 0;
  __syncthreads();
  realize_csr(P, P.r_begin + k, rp, arc, ctl, &ctl->err);
  Realized H{(uint32_t)P.n, rp, arc};
  components(P, H, comp, cinfo);
  for (uint32_t v = threadIdx.x; v < (uint32_t)P.n; v += blockDim.x) {
    comp_out[(size_t)k * P.n + v] = (int32_t)comp[v];
    csize_out[(size_t)k * P.n + v] = (int32_t)(cinfo[comp[v]] & kSizeMask);
  }
  (void)ngroups;
}

template <int G>
__global__ void __launch_bounds__(1024, 1)
debug_sssp_kernel(McDev P, uint32_t r, const int32_t *sources, int32_t nsrc, uint32_t ngroups,
                  uint32_t *dist_out, uint64_t *sigma_out) {
  extern __shared__ __align__(16) unsigned char smem[];
  CtaCtl *ctl = reinterpret_cast<CtaCtl *>(smem);
  const uint32_t n = P.n;
  Layout L;
  L.make(n, (uint32_t)(2 * P.m), ngroups);
  uint32_t *rp = reinterpret_cast<uint32_t *>(smem + L.off_rp);
  uint32_t *arc = reinterpret_cast<uint32_t *>(smem + L.off_arc);
  double *bc = reinterpret_cast<double *>(smem + L.off_bc);
  if (threadIdx.x < kMaxGroups * 3) (&ctl->gred[0][0])[threadIdx.x] = 0xFFFFFFFFu;
  if (threadIdx.x == 0) { ctl->err = 0; ctl->ovf = 0; }
  __syncthreads();
  realize_csr(P, r, rp, arc, ctl, &ctl->err);
  Realized H{n, rp, arc};
  const uint32_t gidx = threadIdx.x / G;
  if (gidx < ngroups) {
    Group<G> grp;
    grp.idx = gidx;
    grp.rank = threadIdx.x % G;
    grp.red = ctl->gred[gidx];
    grp.turn = 0;
    GroupArrays ga = group_arrays(smem, L, n, gidx);
    GroupCtl *gc = &ctl->gctl[gidx];
    for (int32_t k = blockIdx.x * ngroups + gidx; k < nsrc; k += gridDim.x * ngroups) {
      const uint32_t s = (uint32_t)sources[k];
      if (s >= n) continue;
      brandes_one_source<G, double>(grp, H, ga, gc, s, P.delta, bc, false, &ctl->err, &ctl->ovf);
      for (uint32_t v = grp.rank; v < n; v += G) {
        const uint32_t d = ga.dist[v] & kMask;
        const bool reached = d < kInf;
        dist_out[(size_t)k * n + v] = reached ? d : 0xFFFFFFFFu;
        sigma_out[(size_t)k * n + v] = reached ? ga.sig[v] : 0ull;
      }
      grp.sync();
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
uint32_t mc_layout_bytes(uint32_t n, uint64_t arcs, uint32_t ngroups) {
  Layout L;
  L.make(n, (uint32_t)arcs, ngroups);
  return L.total;
}

cudaError_t launch_mc_counts(int G, const McDev *probs_dev, int nprob, const uint64_t *prefix_dev,
                             uint64_t total_items, unsigned char *gslab, uint32_t slab_bytes,
                             uint32_t ngroups, uint32_t smem_bytes, uint32_t grid,
                             cudaStream_t stream) {
  const uint32_t threads = ngroups * (uint32_t)G;
  switch (G) {
    case 32:
      cudaFuncSetAttribute(mc_counts_kernel<32>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_bytes);
      mc_counts_kernel<32><<<grid, threads, smem_bytes, stream>>>(probs_dev, nprob, prefix_dev, total_items, gslab, slab_bytes, ngroups);
      break;
    case 64:
      cudaFuncSetAttribute(mc_counts_kernel<64>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_bytes);
      mc_counts_kernel<64><<<grid, threads, smem_bytes, stream>>>(probs_dev, nprob, prefix_dev, total_items, gslab, slab_bytes, ngroups);
      break;
    case 128:
      cudaFuncSetAttribute(mc_counts_kernel<128>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_bytes);
      mc_counts_kernel<128><<<grid, threads, smem_bytes, stream>>>(probs_dev, nprob, prefix_dev, total_items, gslab, slab_bytes, ngroups);
      break;
    default:
      return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t launch_debug_realize(const McDev &P, uint32_t r_count, uint8_t *alive, uint32_t *w,
                                 cudaStream_t stream) {
  const uint64_t total = (uint64_t)r_count * P.m;
  const uint32_t grid = (uint32_t)((total + 255) / 256 < 4096 ? (total + 255) / 256 : 4096);
  if (total == 0) return cudaSuccess;
  debug_realize_kernel<<<grid, 256, 0, stream>>>(P, r_count, alive, w);
  return cudaGetLastError();
}

cudaError_t launch_debug_components(const McDev &P, uint32_t r_count, int32_t *comp, int32_t *csize,
                                    cudaStream_t stream) {
  const uint32_t smem = mc_layout_bytes(P.n, 2 * P.m, 0);
  cudaFuncSetAttribute(debug_components_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  debug_components_kernel<<<r_count, 256, smem, stream>>>(P, 0, comp, csize);
  return cudaGetLastError();
}

cudaError_t launch_debug_sssp(int G, const McDev &P, uint32_t r, const int32_t *sources, int32_t nsrc,
                              uint32_t ngroups, uint32_t smem, uint32_t grid, uint32_t *dist,
                              uint64_t *sigma, cudaStream_t stream) {
  const uint32_t threads = ngroups * (uint32_t)G;
  switch (G) {
    case 32:
      cudaFuncSetAttribute(debug_sssp_kernel<32>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
      debug_sssp_kernel<32><<<grid, threads, smem, stream>>>(P, r, sources, nsrc, ngroups, dist, sigma);
      break;
    case 64:
      cudaFuncSetAttribute(debug_sssp_kernel<64>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
      debug_sssp_kernel<64><<<grid, threads, smem, stream>>>(P, r, sources, nsrc, ngroups, dist, sigma);
      break;
    case 128:
      cudaFuncSetAttribute(debug_sssp_kernel<128>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
      debug_sssp_kernel<128><<<grid, threads, smem, stream>>>(P, r, sources, nsrc, ngroups, dist, sigma);
      break;
    default:
      return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

}  // namespace afc
