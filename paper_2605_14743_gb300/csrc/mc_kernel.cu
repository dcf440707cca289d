// mc_kernel.cu -- Monte Carlo transition counts on GB300 (sm_103a), shared-memory path.
//
// One CTA owns one network realization at a time (persistent over realizations) and keeps
// it in shared memory:
//   A1  Philox4x32-10 edge draws -> alive-compacted CSR with packed (neighbour, length) arcs,
//       and the smallest alive length at every node
//   A2  components by lock-free union-find (root = smallest id), sizes, candidate flags
//   A3  one warp per source: Dijkstra by settle steps (mc_steps.cuh), source slots on chip
//   A4  path counts sigma (exact 64-bit) pulled from the settled predecessors in the same arc
//       scan that relaxes the step's outgoing arcs: one scan per arc in the forward direction
//   A5  dependencies delta step by step in reverse, one scan per arc; betweenness accumulated
//       exactly in 128-bit fixed point
//   A6  tie-ruled argmax per valid component (Sec. 3.2 eq. local-center, Sec. 7.1 Sel_W)
//       and the transition-count update of every anchor (Alg. 1 / Alg. 2)
//   A7  FP32 mode: a realization whose top-two gap is under the margin is redone in FP64
// Per-source results do not depend on which warp or CTA runs the source, and the exact
// betweenness sum does not depend on the order in which sources finish, so B and every count
// are the same bit for bit for any launch shape.
#include "afc_internal.h"
#include "mc_steps.cuh"

namespace afc {

// Shared-memory layout of a counting CTA: control head, the realization (rp, arcs, smallest
// incident length) and the source slots.  What the source warps do not touch while they run
// (components, the source list, selection scratch, betweenness accumulators) lives in the
// CTA's region of device memory (CtaScratch), so that more source slots fit on chip.  The slot
// region holds nsw compact slots (12 bytes per node, see StepSlot) and, reusing the same bytes,
// wide_slots() 16-byte slots for a realization with a length above kCompactMaxLen or a path
// count above 2^32 - 1; it is never smaller than one wide slot.
struct StepLayout {
  uint32_t off_rp, off_arc, off_mw, off_slots;
  uint32_t slot_bytes, wide_bytes, total;
  __host__ __device__ static uint32_t al(uint32_t x) { return al16(x); }
  __host__ __device__ void make(uint32_t n, uint32_t arcs, uint32_t nsw) {
    uint32_t o = al(sizeof(CtaHead));
    off_rp = o;     o = al(o + 4u * (n + 1));
    off_arc = o;    o = al(o + 4u * (arcs > 0 ? arcs : 1));
    off_mw = o;     o = al(o + 2u * n);
    off_slots = o;
    slot_bytes = al(4u * n) + al(8u * n);
    wide_bytes = slot_bytes + 2u * al(2u * n);
    const uint32_t region = nsw * slot_bytes;
    total = o + (nsw == 0 ? 0u : (region > wide_bytes ? region : wide_bytes));
  }
  // wide slots in the region of nsw compact ones (at least one)
  __host__ __device__ uint32_t wide_slots(uint32_t nsw) const {
    const uint32_t k = nsw * slot_bytes / wide_bytes;
    return k > 0 ? k : 1u;
  }
  __device__ StepSlot slot(unsigned char *smem, uint32_t i, uint32_t n, bool wide) const {
    unsigned char *p = smem + off_slots + i * (wide ? wide_bytes : slot_bytes);
    StepSlot s;
    s.dist = reinterpret_cast<uint32_t *>(p);  p += al(4u * n);
    s.sig = reinterpret_cast<uint64_t *>(p);   p += al(8u * n);
    s.ord = wide ? reinterpret_cast<uint16_t *>(p) : nullptr;   p += al(2u * n);
    s.plist = wide ? reinterpret_cast<uint16_t *>(p) : nullptr;
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
      ctl->err = 0; ctl->ovf = 0; ctl->nsrc = 0; ctl->cursor = 0; ctl->wide_redo = 0;
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

    // Attempts: compact slots first (wide ones from the start for a length above
    // kCompactMaxLen); a path count above 2^32 - 1 redoes the realization with wide slots
    // (fewer sources at a time), and in FP32 mode a top-two gap under the margin redoes it with
    // FP64 dependencies.  Each can happen once: at most three attempts.
    bool use32 = (P.precision == 1), wide = ctl->wmax > kCompactMaxLen;
    const StepSlot s0 = L.slot(smem, 0, n, false);
    for (int attempt = 0; attempt < 3; ++attempt) {
      if (attempt > 0) {
        for (uint32_t v = threadIdx.x; v < n; v += blockDim.x) {
          cs.a0[v] = 0ull; cs.a1[v] = 0ull; cs.a2[v] = 0ull;
        }
        if (threadIdx.x == 0) { ctl->cursor = 0; ctl->wide_redo = 0; }
        __syncthreads();
      }
      if (warp < (wide ? L.wide_slots(nsw) : nsw)) {
        const StepSlot sl = L.slot(smem, warp, n, wide);
        uint32_t err = 0, ovf = 0;
        for (;;) {
          uint32_t k = 0;
          if (lane == 0)
            k = *reinterpret_cast<volatile uint32_t *>(&ctl->wide_redo) ? nsrc
                                                                         : atomicAdd(&ctl->cursor, 1u);
          k = __shfl_sync(kFull, k, 0);
          if (k >= nsrc) break;
          const uint32_t s = src[k];
          const BcAcc acc{cs.a0, cs.a1, cs.a2};
          bool ok;
          if (wide)
            ok = use32 ? source_steps<float, false, true>(H, mw, sl, s, true, acc, err, ovf)
                       : source_steps<double, false, true>(H, mw, sl, s, true, acc, err, ovf);
          else
            ok = use32 ? source_steps<float, true, true>(H, mw, sl, s, true, acc, err, ovf)
                       : source_steps<double, true, true>(H, mw, sl, s, true, acc, err, ovf);
          if (!ok) break;
          if (__any_sync(kFull, ovf & kOvfWide)) {
            if (lane == 0) atomicOr(&ctl->wide_redo, 1u);
            break;
          }
        }
        err = __reduce_or_sync(kFull, err);
        ovf = __reduce_or_sync(kFull, ovf);
        if (lane == 0) {
          if (err) atomicOr(&ctl->err, err);
          if (ovf & 1u) atomicOr(&ctl->ovf, 1u);
        }
      }
      __syncthreads();
      if (ctl->wide_redo) {
        wide = true;
        if (threadIdx.x == 0 && P.stats) atomicAdd(u64p(&P.stats->wide_redone), 1ull);
        continue;
      }
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
      use32 = false;
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

// Distances and path counts of given sources from the production forward routine, on the
// wide slots (64-bit path counts) of a layout of nsw compact slots: warp w of CTA b handles
// source b * W + w of the list on realization r, W = the layout's wide slots.
template <int BLOCK>
__global__ void __launch_bounds__(BLOCK, 1)
debug_sssp_kernel(McDev P, uint32_t r, const int32_t *sources, int32_t nsrc, uint32_t nsw_layout,
                  uint32_t *dist_out, uint64_t *sigma_out) {
  extern __shared__ __align__(16) unsigned char smem[];
  CtaHead *ctl = reinterpret_cast<CtaHead *>(smem);
  const uint32_t n = P.n, warp = threadIdx.x >> 5, lane = threadIdx.x & 31u;
  StepLayout L;
  L.make(n, (uint32_t)(2 * P.m), nsw_layout);
  const uint32_t nsw = L.wide_slots(nsw_layout);
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
    const StepSlot sl = L.slot(smem, warp, n, true);   // wide slots: 64-bit path counts
    uint32_t err = 0, ovf = 0;
    source_steps<double, false, true>(H, mw, sl, s, false, BcAcc{}, err, ovf);
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

uint32_t mc_slots_within(uint32_t n, uint64_t arcs, uint32_t bytes) {
  StepLayout L;
  L.make(n, (uint32_t)arcs, 0);
  if (L.off_slots > bytes) return 0u;
  const uint32_t room = bytes - L.off_slots;
  return room >= L.wide_bytes ? room / L.slot_bytes : 0u;
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
  StepLayout L;
  L.make((uint32_t)P.n, (uint32_t)(2 * P.m), nsw);
  const int32_t nw = (int32_t)L.wide_slots(nsw);
  const uint32_t grid = (uint32_t)((nsrc + nw - 1) / nw);
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
