// mc_global.cu -- Monte Carlo transition counts for graphs whose per-CTA state does not fit in
// shared memory (sm_103a).
//
// The realizations of a problem are processed in batches of G ("groups").  Per batch:
//   prep     one CTA per group: Philox edge draws -> alive-compacted CSR in device memory
//            (A1), components and candidate flags (A2), the list of sources (nodes of valid
//            components), zeroed betweenness accumulators
//   brandes  a persistent grid; the teams of every CTA claim batches of sources of the G
//            realizations from per-group cursors (group by group, so the realized graph being
//            worked on stays hot in L2) and run the bucketed Brandes routine (A3-A5), with
//            their source slots in a per-CTA region of a device arena (or on chip where they
//            fit) and betweenness accumulated exactly (128-bit fixed point, device atomics)
//   select   one CTA per group: tie-ruled argmax and transition counts (A6); in FP32 mode a
//            realization whose top-two gap is under the margin is flagged, its accumulators
//            cleared, and a second brandes + select pair redoes exactly the flagged groups in
//            FP64 (A7)
// All launches are stream ordered; nothing waits on the host.
#include "afc_internal.h"
#include "mc_steps.cuh"

namespace afc {

__host__ __device__ inline size_t al256(size_t x) { return (x + 255u) & ~size_t(255); }

namespace {

constexpr int kPrepThreads = 1024;

__global__ void __launch_bounds__(kPrepThreads, 1)
big_prep_kernel(const McDev *__restrict__ Pd, BigGroup *groups, uint32_t r0, uint32_t r_count) {
  extern __shared__ __align__(16) unsigned char smem[];
  CtaCtl *ctl = reinterpret_cast<CtaCtl *>(smem);
  const McDev &P = *Pd;
  BigGroup &G = groups[blockIdx.x];
  const uint32_t r_local = r0 + blockIdx.x;
  if (r_local >= r_count) {
    if (threadIdx.x == 0) G.active = 0;
    return;
  }
  const uint32_t n = (uint32_t)P.n;
  if (threadIdx.x == 0) {
    ctl->err = 0; ctl->wmax = 1; ctl->edges = 0; ctl->verts = 0; ctl->nsrc = 0;
  }
  __syncthreads();
  uint32_t anchor;
  const uint32_t rho = item_rho(P, r_local, anchor);
  const bool ball = P.per_row && P.hop_radius;
  if (ball) hop_ball(P, anchor, G.cinfo);   // cinfo is free until the components
  realize_csr(P, rho, G.rp, G.arc, ctl, ball ? G.cinfo : nullptr);
  Realized H{n, G.rp, G.arc};
  components(P, H, G.comp, G.cinfo);
  if (P.per_row) keep_anchor_component(n, anchor, G.comp, G.cinfo);
  bucket_setup(ctl, P.delta);
  min_lengths(H, G.mw);
  uint32_t *cedges = G.centre;   // scratch until selection
  for (uint32_t v = threadIdx.x; v < n; v += blockDim.x) {
    cedges[v] = 0; reinterpret_cast<unsigned long long *>(G.bc)[v] = 0ull;
    G.a1[v] = 0ull; G.a2[v] = 0ull;
  }
  __syncthreads();
  for (uint32_t v = threadIdx.x; v < n; v += blockDim.x) {
    const uint32_t root = G.comp[v];
    if (!comp_valid(G.cinfo[root], P.k_min)) continue;
    uint32_t up = 0;
    for (uint32_t e = G.rp[v]; e < G.rp[v + 1]; ++e) up += ((G.arc[e] & 0xFFFFu) > v) ? 1u : 0u;
    if (up) atomicAdd(&cedges[root], up);
  }
  {
    const uint32_t per = (n + blockDim.x - 1) / blockDim.x;
    const uint32_t v0 = min(n, threadIdx.x * per), v1 = min(n, v0 + per);
    uint32_t cnt = 0;
    for (uint32_t v = v0; v < v1; ++v) cnt += comp_valid(G.cinfo[G.comp[v]], P.k_min) ? 1u : 0u;
    uint32_t off = block_exclusive_scan(cnt, ctl->scan, &ctl->scan_total);
    for (uint32_t v = v0; v < v1; ++v)
      if (comp_valid(G.cinfo[G.comp[v]], P.k_min)) G.src[off++] = (uint16_t)v;
    if (threadIdx.x == 0) ctl->nsrc = ctl->scan_total;
  }
  __syncthreads();
  {
    unsigned long long local = 0, lv = 0;
    for (uint32_t v = threadIdx.x; v < n; v += blockDim.x)
      if (G.comp[v] == v && comp_valid(G.cinfo[v], P.k_min)) {
        const unsigned long long sz = G.cinfo[v] & kSizeMask;
        local += sz * cedges[v];
        lv += sz * sz;
      }
    if (local) atomicAdd(&ctl->edges, local);
    if (lv) atomicAdd(&ctl->verts, lv);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    G.r_local = r_local;
    G.nsrc = ctl->nsrc;
    G.cursor = 0;
    G.dsh = ctl->dsh;
    G.err = ctl->err;
    G.ovf = 0;
    G.redo = 0;
    G.edges = ctl->edges;
    G.verts = ctl->verts;
    G.active = 1;
  }
}

// mode 0: FP64, every active group.  1: FP32, every active group.  2: FP64, groups flagged
// for a recheck only.  slots_on_chip 0: the CTA's source slots live in its region of the
// device arena; 1: their distance arrays live in shared memory after the control block, the
// rest in the arena; 2: the whole slots live in shared memory (the arena is not used).
template <int BLOCK, int TS>
__global__ void __launch_bounds__(BLOCK, 1)
big_brandes_kernel(const McDev *__restrict__ Pd, BigGroup *groups, uint32_t ngroups,
                   unsigned char *arena, size_t slot_stride, uint32_t spt, int mode,
                   int slots_on_chip) {
  extern __shared__ __align__(16) unsigned char smem[];
  constexpr uint32_t NT = BLOCK / TS;
  CtaCtl *ctl = reinterpret_cast<CtaCtl *>(smem);
  const uint32_t n = (uint32_t)Pd->n;
  Team<TS, BLOCK> team;
  team.id = threadIdx.x / TS;
  team.rank = threadIdx.x % TS;
  team.tc = &ctl->team[team.id];
  const uint32_t nslots = NT * spt;
  unsigned char *const chip = smem + al16((uint32_t)sizeof(CtaCtl));
  SlotSpace sp{slots_on_chip == 2 ? chip : arena + (size_t)blockIdx.x * nslots * slot_stride,
               slot_stride, n, (n + 31u) / 32u};
  if (slots_on_chip == 1) {
    sp.dist_base = chip;
    sp.dist_stride = al16(4u * n);
  }
  for (uint32_t g = 0; g < ngroups; ++g) {
    BigGroup &G = groups[g];
    if (!G.active || (mode == 2 && !G.redo)) continue;
    const Realized H{n, G.rp, G.arc};
    const uint32_t nsrc = G.nsrc, dsh = G.dsh;
    for (;;) {
      if (team.rank == 0) team.tc->claim = atomicAdd(&G.cursor, spt);
      team.sync();
      const uint32_t k0 = team.tc->claim;
      team.sync();
      if (k0 >= nsrc) break;
      const uint32_t S = min(spt, nsrc - k0);
      const BcAcc acc{reinterpret_cast<unsigned long long *>(G.bc), G.a1, G.a2};
      if (mode == 1)
        brandes_batch<TS, BLOCK, float>(team, H, sp, team.id * spt, S, G.src + k0, dsh, acc,
                                        ctl, &G.err, &G.ovf);
      else
        brandes_batch<TS, BLOCK, double>(team, H, sp, team.id * spt, S, G.src + k0, dsh, acc,
                                         ctl, &G.err, &G.ovf);
    }
  }
}

// Settle-step Brandes (mc_steps.cuh) for the realizations in flight: a persistent grid whose
// warps each own one source slot -- its distance array in shared memory where it fits (every
// arc reads it and the relaxations update it atomically), its path counts, settle order and
// pending list in the warp's region of the device arena -- and claim the sources of the
// groups one at a time, group by group, so the realized graph being worked on stays hot in L2.
// mode as for big_brandes_kernel.
template <int BLOCK>
__global__ void __launch_bounds__(BLOCK, 1)
big_steps_kernel(const McDev *__restrict__ Pd, BigGroup *groups, uint32_t ngroups,
                 unsigned char *arena, size_t slot_stride, uint32_t nsw, int mode,
                 int dist_on_chip) {
  extern __shared__ __align__(16) unsigned char smem[];
  const uint32_t warp = threadIdx.x >> 5, lane = threadIdx.x & 31u;
  if (warp >= nsw) return;   // the warps are independent: no CTA barrier below
  const uint32_t n = (uint32_t)Pd->n;
  unsigned char *mine = arena + ((size_t)blockIdx.x * nsw + warp) * slot_stride;
  StepSlot sl;
  sl.sig = reinterpret_cast<uint64_t *>(mine);
  mine += al256(8ull * n);
  sl.ord = reinterpret_cast<uint16_t *>(mine);
  mine += al256(2ull * n);
  sl.plist = reinterpret_cast<uint16_t *>(mine);
  mine += al256(2ull * n);
  sl.dist = dist_on_chip ? reinterpret_cast<uint32_t *>(smem + (size_t)warp * al16(4u * n))
                         : reinterpret_cast<uint32_t *>(mine);
  for (uint32_t g = 0; g < ngroups; ++g) {
    BigGroup &G = groups[g];
    if (!G.active || (mode == 2 && !G.redo)) continue;
    const Realized H{n, G.rp, G.arc};
    const BcAcc acc{reinterpret_cast<unsigned long long *>(G.bc), G.a1, G.a2};
    const uint32_t nsrc = G.nsrc;
    uint32_t err = 0, ovf = 0;
    for (;;) {
      uint32_t k = 0;
      if (lane == 0) k = atomicAdd(&G.cursor, 1u);
      k = __shfl_sync(kFull, k, 0);
      if (k >= nsrc) break;
      const uint32_t s = G.src[k];
      const bool ok =
          mode == 1 ? source_steps<float, false, false>(H, G.mw, sl, s, true, acc, err, ovf)
                    : source_steps<double, false, false>(H, G.mw, sl, s, true, acc, err, ovf);
      if (!ok) break;
    }
    err = __reduce_or_sync(kFull, err);
    ovf = __reduce_or_sync(kFull, ovf);
    if (lane == 0) {
      if (err) atomicOr(&G.err, err);
      if (ovf) atomicOr(&G.ovf, 1u);
    }
  }
}

__global__ void __launch_bounds__(kPrepThreads, 1)
big_select_kernel(const McDev *__restrict__ Pd, BigGroup *groups, int gap_test, int redo_only) {
  extern __shared__ __align__(16) unsigned char smem[];
  CtaCtl *ctl = reinterpret_cast<CtaCtl *>(smem);
  const McDev &P = *Pd;
  BigGroup &G = groups[blockIdx.x];
  if (!G.active || (redo_only && !G.redo)) return;
  const uint32_t n = (uint32_t)P.n;
  fx_finalize3(reinterpret_cast<unsigned long long *>(G.bc), G.a1, G.a2, n);   // doubles in place
  __syncthreads();
  SlotArrays s0{};
  s0.sig = reinterpret_cast<uint64_t *>(G.best);
  s0.dist = G.centre;
  const bool recheck =
      select_and_count(P, G.r_local, G.comp, G.cinfo, G.bc, s0, G.rank, G.src, gap_test != 0,
                       ctl);
  __syncthreads();
  if (recheck) {
    for (uint32_t v = threadIdx.x; v < n; v += blockDim.x) {
      reinterpret_cast<unsigned long long *>(G.bc)[v] = 0ull;
      G.a1[v] = 0ull;
      G.a2[v] = 0ull;
    }
    if (threadIdx.x == 0) {
      G.redo = 1;
      G.cursor = 0;
      if (P.stats) atomicAdd(u64p(&P.stats->rechecked), 1ull);
    }
    return;
  }
  if (threadIdx.x == 0) {
    G.redo = 0;
    if (P.stats) {
      if (G.err) atomicOr(u64p(&P.stats->device_error), (unsigned long long)G.err);
      atomicAdd(u64p(&P.stats->realizations), 1ull);
      atomicAdd(u64p(&P.stats->sources), (unsigned long long)G.nsrc);
      atomicAdd(u64p(&P.stats->edge_visits), G.edges);
      atomicAdd(u64p(&P.stats->vertex_visits), G.verts);
      if (G.ovf) atomicAdd(u64p(&P.stats->overflow), 1ull);
    }
  }
}

template <int BLOCK, int TS>
cudaError_t launch_brandes_t(const McDev *Pd, BigGroup *groups, uint32_t ngroups,
                             unsigned char *arena, size_t stride, uint32_t spt, int mode,
                             uint32_t smem_bytes, int slots_on_chip, uint32_t grid,
                             cudaStream_t stream) {
  const uint32_t smem = slots_on_chip ? smem_bytes : (uint32_t)sizeof(CtaCtl);
  if (smem > 48u * 1024u)
    cudaFuncSetAttribute(big_brandes_kernel<BLOCK, TS>,
                         cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  big_brandes_kernel<BLOCK, TS><<<grid, BLOCK, smem, stream>>>(
      Pd, groups, ngroups, arena, stride, spt, mode, slots_on_chip);
  return cudaGetLastError();
}

// (block, team) pairs of the global path
#define AFC_BIG_CONFIGS(X) \
  X(256, 64) X(256, 128) X(256, 256) X(512, 128) X(512, 256) X(512, 512) \
  X(1024, 128) X(1024, 256) X(1024, 512) X(1024, 1024)

template <int BLOCK>
cudaError_t launch_steps_t(const McDev *Pd, BigGroup *groups, uint32_t ngroups,
                           unsigned char *arena, size_t stride, uint32_t nsw, int mode,
                           uint32_t smem_bytes, int dist_on_chip, uint32_t grid,
                           cudaStream_t stream) {
  if (smem_bytes > 48u * 1024u)
    cudaFuncSetAttribute(big_steps_kernel<BLOCK>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         smem_bytes);
  big_steps_kernel<BLOCK><<<grid, BLOCK, smem_bytes, stream>>>(Pd, groups, ngroups, arena, stride,
                                                               nsw, mode, dist_on_chip);
  return cudaGetLastError();
}

// team 0: the settle-step kernel with spt source warps per CTA (slots_on_chip: their distance
// arrays in shared memory) in CTAs of 256 or 512 threads (1024 would cap the registers below
// what the routine needs); otherwise the bucketed kernel with teams of `team` threads
cudaError_t launch_brandes(int block, int team, const McDev *Pd, BigGroup *groups,
                           uint32_t ngroups, unsigned char *arena, size_t stride, uint32_t spt,
                           int mode, uint32_t smem_bytes, int slots_on_chip, uint32_t grid,
                           cudaStream_t stream) {
  if (team == 0) {
    if (spt < 1 || spt > (uint32_t)block / 32u) return cudaErrorInvalidValue;
    if (block == 256)
      return launch_steps_t<256>(Pd, groups, ngroups, arena, stride, spt, mode, smem_bytes,
                                 slots_on_chip, grid, stream);
    if (block == 512)
      return launch_steps_t<512>(Pd, groups, ngroups, arena, stride, spt, mode, smem_bytes,
                                 slots_on_chip, grid, stream);
    return cudaErrorInvalidValue;
  }
#define AFC_X(B, T)                                                                   \
  if (block == B && team == T)                                                        \
    return launch_brandes_t<B, T>(Pd, groups, ngroups, arena, stride, spt, mode,      \
                                  smem_bytes, slots_on_chip, grid, stream);
  AFC_BIG_CONFIGS(AFC_X)
#undef AFC_X
  return cudaErrorInvalidValue;
}

}  // namespace

bool big_config_supported(int block, int team) {
#define AFC_X(B, T) if (block == B && team == T) return true;
  AFC_BIG_CONFIGS(AFC_X)
#undef AFC_X
  return false;
}


size_t big_group_bytes(uint32_t n, uint64_t arcs) {
  return al256(4ull * (n + 1)) + al256(4ull * (arcs > 0 ? arcs : 1)) + 4 * al256(4ull * n) +
         2 * al256(2ull * n) + 4 * al256(8ull * n);
}

uint32_t big_slot_bytes(uint32_t n) { return (slot_bytes_for(n) + 255u) & ~255u; }

size_t big_step_slot_bytes(uint32_t n, bool dist_in_arena) {
  return al256(8ull * n) + 2 * al256(2ull * n) + (dist_in_arena ? al256(4ull * n) : 0);
}

void big_group_carve(BigGroup &G, unsigned char *base, uint32_t n, uint64_t arcs) {
  unsigned char *p = base;
  auto take = [&](size_t bytes) { unsigned char *q = p; p += al256(bytes); return q; };
  G = BigGroup{};
  G.rp = reinterpret_cast<uint32_t *>(take(4ull * (n + 1)));
  G.arc = reinterpret_cast<uint32_t *>(take(4ull * (arcs > 0 ? arcs : 1)));
  G.comp = reinterpret_cast<uint32_t *>(take(4ull * n));
  G.cinfo = reinterpret_cast<uint32_t *>(take(4ull * n));
  G.centre = reinterpret_cast<uint32_t *>(take(4ull * n));
  G.rank = reinterpret_cast<uint32_t *>(take(4ull * n));
  G.src = reinterpret_cast<uint16_t *>(take(2ull * n));
  G.bc = reinterpret_cast<double *>(take(8ull * n));
  G.a1 = reinterpret_cast<unsigned long long *>(take(8ull * n));
  G.a2 = reinterpret_cast<unsigned long long *>(take(8ull * n));
  G.mw = reinterpret_cast<uint16_t *>(take(2ull * n));
  G.best = reinterpret_cast<unsigned long long *>(take(8ull * n));
}

uint32_t big_dist_smem_bytes(uint32_t n, uint32_t nslots) {
  return al16((uint32_t)sizeof(CtaCtl)) + nslots * al16(4u * n);
}

uint32_t big_slots_smem_bytes(uint32_t n, uint32_t nslots) {
  return al16((uint32_t)sizeof(CtaCtl)) + nslots * big_slot_bytes(n);
}

cudaError_t launch_mc_global(int block, int team, const McDev *Pd, int precision,
                             BigGroup *groups_d, uint32_t ngroups, uint32_t r_count,
                             unsigned char *arena, size_t slot_stride, uint32_t spt,
                             uint32_t smem_bytes, int slots_on_chip, uint32_t grid,
                             cudaStream_t stream) {
  if (team != 0 && !big_config_supported(block, team)) return cudaErrorInvalidValue;
  const bool fp32 = (precision == 1);
  for (uint32_t r0 = 0; r0 < r_count; r0 += ngroups) {
    big_prep_kernel<<<ngroups, kPrepThreads, sizeof(CtaCtl), stream>>>(Pd, groups_d, r0, r_count);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    e = launch_brandes(block, team, Pd, groups_d, ngroups, arena, slot_stride, spt, fp32 ? 1 : 0,
                       smem_bytes, slots_on_chip, grid, stream);
    if (e != cudaSuccess) return e;
    big_select_kernel<<<ngroups, kPrepThreads, sizeof(CtaCtl), stream>>>(Pd, groups_d, fp32 ? 1 : 0, 0);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if (fp32) {
      e = launch_brandes(block, team, Pd, groups_d, ngroups, arena, slot_stride, spt, 2,
                         smem_bytes, slots_on_chip, grid, stream);
      if (e != cudaSuccess) return e;
      big_select_kernel<<<ngroups, kPrepThreads, sizeof(CtaCtl), stream>>>(Pd, groups_d, 0, 1);
      if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
  }
  return cudaSuccess;
}

}  // namespace afc
