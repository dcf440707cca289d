// mc_kernel.cu -- Monte Carlo transition counts on GB300 (sm_103a).
//
// One CTA owns one network realization at a time (persistent over realizations) and keeps
// it in shared memory:
//   A1  Philox4x32-10 edge draws -> alive-compacted CSR with packed (neighbour, length) arcs
//   A2  components by lock-free union-find (root = smallest id), sizes, candidate flags
//   A3  bucketed (Delta-stepping) integer SSSP for a batch of S sources advanced in lockstep:
//       all S sources work on the same bucket [b*Delta, (b+1)*Delta) at once, so one set of
//       CTA barriers serves S sources and the bucket members of all sources fill the threads
//   A4  shortest-path counts sigma (exact 64-bit), resolved bucket by bucket
//   A5  dependencies delta in reverse bucket order; betweenness accumulated in FP64
//   A6  tie-ruled argmax per valid component (Sec. 3.2 eq. local-center, Sec. 7.1 Sel_W)
//       and the transition-count update of every anchor (Alg. 1 / Alg. 2)
//   A7  FP32 mode: a realization whose top-two gap is under the margin is redone in FP64
//
#include "mc_common.cuh"

namespace afc {

// ---------------------------------------------------------------------------------------
// The persistent kernel.  Work item w enumerates (problem, realization) pairs of all
// problems; items are visited in strided order by the CTAs.  Inside a realization the CTA's
// teams claim batches of sources dynamically.
// ---------------------------------------------------------------------------------------
template <int BLOCK, int TS>
__global__ void __launch_bounds__(BLOCK, 1)
mc_counts_kernel(const McDev *__restrict__ probs, int nprob, const uint64_t *item_prefix,
                 uint64_t total_items, uint32_t spt) {
  extern __shared__ __align__(16) unsigned char smem[];
  constexpr uint32_t NT = BLOCK / TS;
  CtaCtl *ctl = reinterpret_cast<CtaCtl *>(smem);
  Team<TS, BLOCK> team;
  team.id = threadIdx.x / TS;
  team.rank = threadIdx.x % TS;
  team.tc = &ctl->team[team.id];
  for (uint64_t item = blockIdx.x; item < total_items; item += gridDim.x) {
    int g = 0;
    while (g + 1 < nprob && item_prefix[g + 1] <= item) ++g;
    const McDev &P = probs[g];
    // sources per team: per problem in a batched launch (small graphs take more slots of the
    // launch's shared memory), else the launch's value
    const uint32_t spt_g = P.spt ? P.spt : spt;
    const uint32_t nslots = NT * spt_g;
    const uint32_t r_local = (uint32_t)(item - item_prefix[g]);
    uint32_t anchor;
    const uint32_t r = item_rho(P, r_local, anchor);
    const uint32_t n = P.n;
    Layout L;
    L.make(n, (uint32_t)(2 * P.m), nslots);
    uint32_t *rp = reinterpret_cast<uint32_t *>(smem + L.off_rp);
    uint32_t *arc = reinterpret_cast<uint32_t *>(smem + L.off_arc);
    uint32_t *comp = reinterpret_cast<uint32_t *>(smem + L.off_comp);
    uint32_t *cinfo = reinterpret_cast<uint32_t *>(smem + L.off_cinfo);
    double *bc = reinterpret_cast<double *>(smem + L.off_bc);
    uint32_t *bci = reinterpret_cast<uint32_t *>(smem + L.off_bci);
    uint16_t *src = reinterpret_cast<uint16_t *>(smem + L.off_src);
    uint32_t *sel = reinterpret_cast<uint32_t *>(smem + L.off_sel);
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
    bucket_setup(ctl, P.delta);
    const uint32_t dsh = ctl->dsh;
    const SlotSpace sp = smem_slots(smem, L, n);

    // sources: every node of a valid component (ascending), alive edges per root for TEPS
    uint32_t *cedges = sel;
    for (uint32_t v = threadIdx.x; v < n; v += blockDim.x) { cedges[v] = 0; bc[v] = 0.0; bci[v] = 0; }
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
    for (int attempt = 0; attempt < 2; ++attempt) {
      const bool use32 = fp32 && attempt == 0;
      if (attempt == 1) {
        for (uint32_t v = threadIdx.x; v < n; v += blockDim.x) { bc[v] = 0.0; bci[v] = 0; }
        if (threadIdx.x == 0) ctl->cursor = 0;
        __syncthreads();
      }
      for (;;) {
        if (team.rank == 0) team.tc->claim = atomicAdd(&ctl->cursor, spt_g);
        team.sync();
        const uint32_t k0 = team.tc->claim;
        team.sync();
        if (k0 >= nsrc) break;
        const uint32_t S = min(spt_g, nsrc - k0);
        if (use32)
          brandes_batch<TS, BLOCK, float>(team, H, sp, team.id * spt_g, S, src + k0, dsh, bc, bci,
                                          true, ctl, &ctl->err, &ctl->ovf);
        else
          brandes_batch<TS, BLOCK, double>(team, H, sp, team.id * spt_g, S, src + k0, dsh, bc,
                                           bci, true, ctl, &ctl->err, &ctl->ovf);
      }
      __syncthreads();
      // betweenness = integral part (unique-path subtrees, exact) + floating part
      for (uint32_t v = threadIdx.x; v < n; v += blockDim.x) bc[v] += (double)bci[v];
      __syncthreads();
      const bool recheck = select_and_count(P, r_local, comp, cinfo, bc, slot_arrays(sp, 0),
                                            sel, src, use32, ctl);
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

__global__ void debug_components_kernel(McDev P, int32_t *comp_out, int32_t *csize_out) {
  extern __shared__ __align__(16) unsigned char smem[];
  CtaCtl *ctl = reinterpret_cast<CtaCtl *>(smem);
  Layout L;
  L.make(P.n, (uint32_t)(2 * P.m), 0);
  uint32_t *rp = reinterpret_cast<uint32_t *>(smem + L.off_rp);
  uint32_t *arc = reinterpret_cast<uint32_t *>(smem + L.off_arc);
  uint32_t *comp = reinterpret_cast<uint32_t *>(smem + L.off_comp);
  uint32_t *cinfo = reinterpret_cast<uint32_t *>(smem + L.off_cinfo);
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

// Distances and path counts of given sources from the production batch routine: team t of
// CTA b handles the sources [(b * NT + t) * spt, ... + spt) of the list on realization r.
template <int BLOCK, int TS>
__global__ void __launch_bounds__(BLOCK, 1)
debug_sssp_kernel(McDev P, uint32_t r, const int32_t *sources, int32_t nsrc, uint32_t spt,
                  uint32_t *dist_out, uint64_t *sigma_out) {
  extern __shared__ __align__(16) unsigned char smem[];
  constexpr uint32_t NT = BLOCK / TS;
  CtaCtl *ctl = reinterpret_cast<CtaCtl *>(smem);
  const uint32_t n = P.n;
  Layout L;
  L.make(n, (uint32_t)(2 * P.m), NT * spt);
  uint32_t *rp = reinterpret_cast<uint32_t *>(smem + L.off_rp);
  uint32_t *arc = reinterpret_cast<uint32_t *>(smem + L.off_arc);
  double *bc = reinterpret_cast<double *>(smem + L.off_bc);
  uint32_t *bci = reinterpret_cast<uint32_t *>(smem + L.off_bci);
  uint16_t *src = reinterpret_cast<uint16_t *>(smem + L.off_src);
  if (threadIdx.x == 0) { ctl->err = 0; ctl->ovf = 0; ctl->wmax = 1; }
  __syncthreads();
  realize_csr(P, r, rp, arc, ctl);
  Realized H{n, rp, arc};
  bucket_setup(ctl, P.delta);
  Team<TS, BLOCK> team;
  team.id = threadIdx.x / TS;
  team.rank = threadIdx.x % TS;
  team.tc = &ctl->team[team.id];
  const uint32_t k0 = (blockIdx.x * NT + team.id) * spt;
  uint16_t *tsrc = src + team.id * spt;
  if (k0 < (uint32_t)nsrc) {
    const uint32_t S = min(spt, (uint32_t)nsrc - k0);
    for (uint32_t i = team.rank; i < S; i += TS) {
      const int32_t s = sources[k0 + i];
      tsrc[i] = (uint16_t)((s >= 0 && (uint32_t)s < n) ? s : 0);
    }
    team.sync();
    const SlotSpace sp = smem_slots(smem, L, n);
    brandes_batch<TS, BLOCK, double>(team, H, sp, team.id * spt, S, tsrc, ctl->dsh, bc, bci,
                                     false, ctl, &ctl->err, &ctl->ovf);
    for (uint32_t t = team.rank; t < S * n; t += TS) {
      const uint32_t i = t / n, v = t - i * n;
      SlotArrays a = slot_arrays(sp, team.id * spt + i);
      const uint32_t d = a.dist[v] & kMask;
      const bool reached = d < kInf;
      dist_out[(size_t)(k0 + i) * n + v] = reached ? d : 0xFFFFFFFFu;
      sigma_out[(size_t)(k0 + i) * n + v] = reached ? a.sig[v] : 0ull;
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
uint32_t mc_layout_bytes(uint32_t n, uint64_t arcs, uint32_t nslots) {
  Layout L;
  L.make(n, (uint32_t)arcs, nslots);
  return L.total;
}

// (block, team) pairs with an instantiation; named-barrier teams need ids <= 15.
#define AFC_MC_CONFIGS(X) \
  X(256, 32) X(256, 64) X(256, 128) X(256, 256) \
  X(512, 32) X(512, 64) X(512, 128) X(512, 256) X(512, 512) \
  X(1024, 32) X(1024, 128) X(1024, 256) X(1024, 1024)

bool mc_config_supported(int block, int team) {
#define AFC_X(B, T) if (block == B && team == T) return true;
  AFC_MC_CONFIGS(AFC_X)
#undef AFC_X
  return false;
}

template <int BLOCK, int TS>
static cudaError_t launch_counts_t(const McDev *probs_dev, int nprob, const uint64_t *prefix_dev,
                                   uint64_t total_items, uint32_t spt, uint32_t smem,
                                   uint32_t grid, cudaStream_t stream) {
  cudaFuncSetAttribute(mc_counts_kernel<BLOCK, TS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       smem);
  mc_counts_kernel<BLOCK, TS><<<grid, BLOCK, smem, stream>>>(probs_dev, nprob, prefix_dev,
                                                             total_items, spt);
  return cudaGetLastError();
}

cudaError_t launch_mc_counts(int block, int team, const McDev *probs_dev, int nprob,
                             const uint64_t *prefix_dev, uint64_t total_items,
                             uint32_t slots_per_team, uint32_t smem_bytes, uint32_t grid,
                             cudaStream_t stream) {
#define AFC_X(B, T)                                                                        \
  if (block == B && team == T)                                                             \
    return launch_counts_t<B, T>(probs_dev, nprob, prefix_dev, total_items, slots_per_team, \
                                 smem_bytes, grid, stream);
  AFC_MC_CONFIGS(AFC_X)
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
  const uint32_t smem = mc_layout_bytes(P.n, 2 * P.m, 0);
  cudaFuncSetAttribute(debug_components_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  debug_components_kernel<<<r_count, 256, smem, stream>>>(P, comp, csize);
  return cudaGetLastError();
}

template <int BLOCK, int TS>
static cudaError_t launch_sssp_t(const McDev &P, uint32_t r, const int32_t *sources, int32_t nsrc,
                                 uint32_t spt, uint32_t smem, uint32_t *dist, uint64_t *sigma,
                                 cudaStream_t stream) {
  const uint32_t per_cta = (BLOCK / TS) * spt;
  const uint32_t grid = (uint32_t)((nsrc + (int32_t)per_cta - 1) / (int32_t)per_cta);
  cudaFuncSetAttribute(debug_sssp_kernel<BLOCK, TS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       smem);
  debug_sssp_kernel<BLOCK, TS><<<grid, BLOCK, smem, stream>>>(P, r, sources, nsrc, spt, dist,
                                                              sigma);
  return cudaGetLastError();
}

cudaError_t launch_debug_sssp(int block, int team, const McDev &P, uint32_t r,
                              const int32_t *sources, int32_t nsrc, uint32_t slots_per_team,
                              uint32_t smem, uint32_t *dist, uint64_t *sigma,
                              cudaStream_t stream) {
#define AFC_X(B, T)                                                                    \
  if (block == B && team == T)                                                         \
    return launch_sssp_t<B, T>(P, r, sources, nsrc, slots_per_team, smem, dist, sigma, \
                               stream);
  AFC_MC_CONFIGS(AFC_X)
#undef AFC_X
  return cudaErrorInvalidValue;
}

}  // namespace afc
