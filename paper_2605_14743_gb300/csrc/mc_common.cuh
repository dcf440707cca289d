// mc_common.cuh -- device routines of the Monte Carlo counting path shared by the
// shared-memory kernel (graphs that fit on chip) and the global-memory kernels (larger
// graphs): realization, components, the exact betweenness accumulators, the warp-cooperative
// arc loop, the bucketed Brandes routine of the global path and selection.
//
// Per source ("slot") state of the bucketed routine: dist[n] (u32 distance | flag), sig[n]
// (u64: last relaxed distance while tentative, then sigma, then rho = (1 + delta) / sigma in
// the same slot), ord[n] (u16 settled vertices grouped by bucket) and a ring of kRing bucket
// bitmaps that holds the discovered-but-unsettled vertices by bucket.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "afc_device.cuh"
#include "mc_types.h"

namespace afc {

__device__ __forceinline__ unsigned long long *u64p(uint64_t *p) {
  return reinterpret_cast<unsigned long long *>(p);
}

constexpr uint32_t kInf = 0x7FFFFFFFu;    // unreached distance
constexpr uint32_t kFlag = 0x80000000u;   // "sigma final" (forward) / "delta pending" (backward)
constexpr uint32_t kMask = 0x7FFFFFFFu;
constexpr uint64_t kNoRelax = ~0ull;
constexpr uint64_t kIntTag = 0x8000000000000000ull;   // rho stored as an exact integer

__device__ __forceinline__ uint32_t ld_volatile(const uint32_t *p) {
  return *reinterpret_cast<const volatile uint32_t *>(p);
}
__device__ __forceinline__ void st_volatile(uint32_t *p, uint32_t v) {
  *reinterpret_cast<volatile uint32_t *>(p) = v;
}

// Bytes of one source slot: dist[n] u32, sig[n] u64, ord[n] u16, ring[kRing][words] u32.
__host__ __device__ __forceinline__ uint32_t al16(uint32_t x) { return (x + 15u) & ~15u; }
__host__ __device__ __forceinline__ uint32_t slot_bytes_for(uint32_t n) {
  const uint32_t words = (n + 31u) / 32u;
  return al16(4u * n) + al16(8u * n) + al16(2u * n) + al16(4u * kRing * words);
}

struct SlotArrays {
  uint32_t *dist;
  uint64_t *sig;
  uint16_t *ord;
  uint32_t *ring;   // [kRing][words]
};

// Where the source slots of one CTA live: shared memory (graphs that fit) or a per-CTA
// region of a global arena (larger graphs); slot i starts at base + i * stride.
struct SlotSpace {
  unsigned char *base;
  size_t stride;
  uint32_t n, words;
  unsigned char *dist_base = nullptr;   // if set: dist of slot i at dist_base + i * dist_stride
  uint32_t dist_stride = 0;             // (the global path keeps dist in shared memory)
};

__device__ __forceinline__ SlotArrays slot_arrays(const SlotSpace &sp, uint32_t i) {
  unsigned char *p = sp.base + (size_t)i * sp.stride;
  const uint32_t n = sp.n;
  SlotArrays a;
  a.dist = reinterpret_cast<uint32_t *>(sp.dist_base ? sp.dist_base + (size_t)i * sp.dist_stride
                                                     : p);
  p += al16(4u * n);
  a.sig = reinterpret_cast<uint64_t *>(p);   p += al16(8u * n);
  a.ord = reinterpret_cast<uint16_t *>(p);   p += al16(2u * n);
  a.ring = reinterpret_cast<uint32_t *>(p);
  return a;
}

struct Realized {
  uint32_t n;
  const uint32_t *rp;    // [n+1] alive-compacted row offsets
  const uint32_t *arc;   // packed: neighbour (low 16 bits) | length << 16
};

// A team of TS threads (whole warps) of a BLOCK-thread CTA that advances its own subset of
// source slots in lockstep.  TS == 32: warp-synchronous; TS == BLOCK: CTA barriers; otherwise
// named barrier (team + 1) with bar.red for the OR reductions.
template <int TS, int BLOCK>
struct Team {
  uint32_t id, rank;
  TeamCtl *tc;
  __device__ __forceinline__ void sync() const {
    if constexpr (TS == 32) {
      __syncwarp();
    } else if constexpr (TS == BLOCK) {
      __syncthreads();
    } else {
      asm volatile("bar.sync %0, %1;" ::"r"(id + 1), "n"(TS) : "memory");
    }
  }
  __device__ __forceinline__ bool any(bool p) const {
    if constexpr (TS == 32) {
      return __any_sync(kFull, p);
    } else if constexpr (TS == BLOCK) {
      return __syncthreads_or(p) != 0;
    } else {
      uint32_t r;
      asm volatile(
          "{ .reg .pred pa, pb;\n"
          "  setp.ne.u32 pa, %1, 0;\n"
          "  bar.red.or.pred pb, %2, %3, pa;\n"
          "  selp.u32 %0, 1, 0, pb; }"
          : "=r"(r)
          : "r"((uint32_t)p), "r"(id + 1), "n"(TS)
          : "memory");
      return r != 0;
    }
  }
};

// Exclusive prefix of per-slot counts into tc->pref[0..S] (S <= 32); team's first warp only.
template <typename F>
__device__ __forceinline__ void slot_prefix(TeamCtl *tc, uint32_t rank, uint32_t S, F count) {
  if (rank >= 32) return;
  const uint32_t x = rank < S ? count(rank) : 0u;
  uint32_t inc = x;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(kFull, inc, o);
    if (rank >= (uint32_t)o) inc += y;
  }
  if (rank < S) tc->pref[rank] = inc - x;
  if (rank == 31) tc->pref[S] = inc;
}

// Largest slot i with pref[i] <= k (pref ascending, pref[S] = total > k).
__device__ __forceinline__ uint32_t find_slot(const uint32_t *pref, uint32_t S, uint32_t k) {
  uint32_t lo = 0, hi = S;
  while (hi - lo > 1) {
    const uint32_t mid = (lo + hi) >> 1;
    if (pref[mid] <= k) lo = mid; else hi = mid;
  }
  return lo;
}

// Warp-cooperative loop over the arcs of up to 32 items, one per lane: lane j holds an item
// with `deg` arcs starting at arc index `e0` (deg 0: nothing to do).  The warp walks the
// concatenation of the items' arc ranges in windows of 32 positions, lane L taking position
// w0 + L, so a warp's time follows its total arc count instead of its heaviest lane.  For
// each position f(valid, owner_lane, arc[arc_index]) runs on every lane (valid = false past
// the end, arc word 0 then); f fetches the owner's item data with __shfl_sync from owner_lane.
// After f, g(lo, hi) runs on every lane with [lo, hi) the positions of the window (0..32) that
// belong to the lane's own item (lo == hi when none): the owner can then read, in arc order,
// what f left per position.  All 32 lanes must call it (warp-uniform control flow).  Returns
// at once when no lane has arcs.  PREFETCH (arcs in device memory) issues the next window's
// arc loads before f runs on the current window, so their latency overlaps f's work.
struct NoWindowHook {
  __device__ __forceinline__ void operator()(uint32_t, uint32_t) const {}
};

template <bool PREFETCH, typename F, typename G = NoWindowHook>
__device__ __forceinline__ void warp_arcs(uint32_t deg, uint32_t e0, uint8_t *table,
                                          const uint32_t *arc, F &&f, G &&g = G{}) {
  const uint32_t lane = lane_id();
  const uint32_t nz = __ballot_sync(kFull, deg > 0);
  if (nz == 0u) return;
  uint32_t incl = deg;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(kFull, incl, o);
    if (lane >= (uint32_t)o) incl += y;
  }
  const uint32_t tot = __shfl_sync(kFull, incl, 31);
  const uint32_t excl = incl - deg;
  if (deg > 0) table[__popc(nz & lanemask_lt())] = (uint8_t)lane;
  __syncwarp();
  uint32_t prior = 0;   // items whose range starts before the window
  // owner lane and arc index of this lane's position in the window starting at w0
  auto locate = [&](uint32_t w0, bool &valid, uint32_t &ol, uint32_t &e) {
    const uint32_t rel = excl - w0;   // wraps (large) when the range starts before w0
    const uint32_t starts = __reduce_or_sync(kFull, (deg > 0 && rel < 32u) ? (1u << rel) : 0u);
    const uint32_t pos = w0 + lane;
    valid = pos < tot;
    const uint32_t rank = prior + __popc(starts & (0xFFFFFFFFu >> (31u - lane))) - 1u;
    ol = valid ? (uint32_t)table[rank] : 0u;
    const uint32_t oex = __shfl_sync(kFull, excl, ol);
    const uint32_t oe0 = __shfl_sync(kFull, e0, ol);
    e = oe0 + (pos - oex);
    prior += __popc(starts);
  };
  // this lane's own positions inside the window starting at w0
  auto own = [&](uint32_t w0) {
    const uint32_t a = max(excl, w0), b = min(excl + deg, w0 + 32u);
    return a < b ? make_uint2(a - w0, b - w0) : make_uint2(0u, 0u);
  };
  if constexpr (PREFETCH) {
    bool valid;
    uint32_t ol, e;
    locate(0u, valid, ol, e);
    uint32_t pk = valid ? arc[e] : 0u;
    for (uint32_t w0 = 0; w0 < tot; w0 += 32u) {
      bool nvalid = false;
      uint32_t nol = 0, npk = 0;
      if (w0 + 32u < tot) {   // warp-uniform
        uint32_t ne;
        locate(w0 + 32u, nvalid, nol, ne);
        npk = nvalid ? arc[ne] : 0u;
      }
      f(valid, ol, pk);
      const uint2 r = own(w0);
      g(r.x, r.y);
      valid = nvalid;
      ol = nol;
      pk = npk;
    }
  } else {
    for (uint32_t w0 = 0; w0 < tot; w0 += 32u) {
      bool valid;
      uint32_t ol, e;
      locate(w0, valid, ol, e);
      f(valid, ol, valid ? arc[e] : 0u);
      const uint2 r = own(w0);
      g(r.x, r.y);
    }
  }
  __syncwarp();
}

// Betweenness accumulators of a realization: B_v 2^64 = a0 2^64 + a1 2^32 + a2 (see fx_red).
struct BcAcc {
  unsigned long long *a0, *a1, *a2;
};

// Betweenness accumulation without return values (device-memory reductions): the addend x
// (0 <= x < 2^64) is split exactly, from its bits, into x 2^64 = xi 2^64 + xf (xf < 2^64,
// truncated below 2^-64, i.e. exact whenever x >= 2^-12), and xi, the top and the bottom 32 bits of xf go to three
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

// Correctly rounded reciprocal in the dependency precision.
__device__ __forceinline__ double recip(double x) { return __drcp_rn(x); }
__device__ __forceinline__ float recip(float x) { return __frcp_rn(x); }

// The dependency step of v from acc = sum of its successors' rho (Sec. 3.1, Brandes):
// delta(v) = sigma(v) acc and rho(v) = (1 + delta(v)) / sigma(v) = acc + 1 / sigma(v).
template <typename DT>
__device__ __forceinline__ void dependency(uint64_t sg, DT acc, DT &dep, DT &rho) {
  if (sg == 1ull) {
    dep = acc;
    rho = (DT)1 + dep;
  } else {
    const DT sv = (DT)sg;
    dep = sv * acc;
    rho = acc + recip(sv);
  }
}

// ---------------------------------------------------------------------------------------
// Bucketed Brandes for graphs whose per-source state does not fit on chip (the global-memory
// path).  A batch of S sources (srcs[0..S)) in the slots [slot0, slot0 + S) is advanced in
// lockstep by one team, bucket by bucket (integer Delta-stepping), every pass warp-cooperative
// over the members' arcs.  Adds delta_s(v) for v != s to the exact accumulators (fx_red).
// Every thread of the team must call it.
// ---------------------------------------------------------------------------------------
template <int TS, int BLOCK, typename DT>
__device__ __forceinline__ bool brandes_batch(const Team<TS, BLOCK> &team, const Realized &H,
                                              const SlotSpace &sp, uint32_t slot0, uint32_t S,
                                              const uint16_t *srcs, uint32_t dsh, const BcAcc &acc,
                                              CtaCtl *ctl, uint32_t *err_out, uint32_t *ovf_out) {
  const uint32_t n = H.n, W = sp.words;
  constexpr uint32_t kRingMask = kRing - 1u;
  const uint32_t tid = team.rank;
  TeamCtl *tc = team.tc;
  SlotCtl *sl = ctl->slot + slot0;
  uint32_t my_err = 0, my_ovf = 0;
  const uint32_t lane = tid & 31u, warp = tid >> 5;
  constexpr uint32_t NW = TS / 32;
  WarpScratch *ws = &ctl->warp[threadIdx.x >> 5];

  // ---- init
  for (uint32_t i = 0; i < S; ++i) {
    SlotArrays a = slot_arrays(sp, slot0 + i);
    for (uint32_t v = tid; v < n; v += TS) a.dist[v] = kInf;
    for (uint32_t t = tid; t < kRing * W; t += TS) a.ring[t] = 0u;
  }
  team.sync();
  for (uint32_t i = tid; i < S; i += TS) {
    SlotArrays a = slot_arrays(sp, slot0 + i);
    const uint32_t s = srcs[i];
    SlotCtl &sc = sl[i];
    sc.s = s;
    sc.nm = 0; sc.mstart = 0; sc.hi = 0; sc.lo = 0;
    sc.ring_mask = 1u;            // ring_mask: bucket 0 holds the source
    a.dist[s] = 0;
    a.ring[s >> 5] = 1u << (s & 31u);
  }
  team.sync();

  // ---- forward: buckets in increasing order
  bool ok = true;
  uint32_t b = 0;
  for (uint32_t guard = 0;; ++guard) {
    if (guard > 2u * n + 2u) { my_err |= kErrPassLimit; ok = false; break; }
    if (tid < 32) {
      // first ring offset k (bucket b + k) holding discovered vertices in any slot
      uint32_t m = tid < S ? sl[tid].ring_mask : 0u;
      m = __reduce_or_sync(kFull, m);
      const uint32_t sh = b & kRingMask;   // bit k of rot <-> ring slot (b + k) mod kRing
      const uint32_t rot = ((m >> sh) | (m << ((kRing - sh) & 31u))) & ((1u << kRing) - 1u);
      if (tid == 0) tc->bucket = rot ? b + (uint32_t)(__ffs(rot) - 1) : 0xFFFFFFFFu;
    }
    team.sync();
    if (tc->bucket == 0xFFFFFFFFu) break;
    b = tc->bucket;
    const uint32_t rs = b & kRingMask;
    const uint32_t dend = (b + 1u) << dsh;
    // extraction of bucket b into the member lists, appends aggregated per warp and slot
    // words interleaved over the team's warps (item increases with the lane, so the lanes of
    // one slot stay contiguous for the keyed prefix below)
    for (uint32_t base = 0; base < S * W; base += TS) {
      const uint32_t item = base + lane * NW + warp;
      uint32_t i = 0xFFFFu, live = 0;
      uint16_t vb = 0;
      if (item < S * W) {
        i = item / W;
        const uint32_t w = item - i * W;
        SlotArrays a = slot_arrays(sp, slot0 + i);
        uint32_t word = a.ring[rs * W + w];
        if (word) {
          a.ring[rs * W + w] = 0u;
          while (word) {
            const uint32_t j = __ffs(word) - 1;
            word &= word - 1u;
            const uint32_t d = a.dist[w * 32u + j];
            if (!(d & kFlag) && d < dend) live |= 1u << j;   // else settled (stale bit)
          }
        }
        vb = (uint16_t)(w * 32u);
      }
      const uint32_t cnt = __popc(live);
      uint32_t inc = cnt;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(kFull, inc, o);
        if (lane >= (uint32_t)o) inc += y;
      }
      const uint32_t peers = __match_any_sync(kFull, i);
      const uint32_t leader = __ffs(peers) - 1, last = 31 - __clz(peers);
      const uint32_t before = __shfl_sync(kFull, inc, leader == 0 ? 0 : leader - 1);
      const uint32_t gbase = leader == 0 ? 0u : before;
      const uint32_t gtotal = __shfl_sync(kFull, inc, last) - gbase;
      uint32_t pos0 = 0;
      if (lane == leader && i != 0xFFFFu && gtotal) pos0 = atomicAdd(&sl[i].nm, gtotal);
      pos0 = __shfl_sync(kFull, pos0, leader);
      if (live) {
        SlotArrays a = slot_arrays(sp, slot0 + i);
        uint32_t pos = pos0 + inc - cnt - gbase;
        while (live) {
          const uint32_t j = __ffs(live) - 1;
          live &= live - 1u;
          const uint32_t v = (uint32_t)vb + j;
          if (pos < n) { a.ord[pos] = (uint16_t)v; a.sig[v] = kNoRelax; }
          else my_err |= kErrCapacity;
          ++pos;
        }
      }
    }
    for (uint32_t i = tid; i < S; i += TS) sl[i].ring_mask &= ~(1u << rs);
    team.sync();
    // relaxation passes until no member of the bucket improves; a pass takes the members in
    // chunks of 32 per warp and relaxes their arcs warp-cooperatively
    for (uint32_t pass = 0;; ++pass) {
      if (pass > n + 1) { my_err |= kErrPassLimit; ok = false; break; }
      slot_prefix(tc, tid, S, [&](uint32_t i) { return min(sl[i].nm, n) - sl[i].mstart; });
      team.sync();
      const uint32_t total = tc->pref[S];
      bool improved = false;
      for (uint32_t base = 0; base < total; base += TS) {
        const uint32_t k = base + lane * NW + warp;   // members interleaved over the warps
        uint32_t i = 0, d = 0, e0 = 0, deg = 0;
        if (k < total) {
          i = find_slot(tc->pref, S, k);
          SlotArrays a = slot_arrays(sp, slot0 + i);
          const uint32_t v = a.ord[sl[i].mstart + k - tc->pref[i]];
          if (v >= n) {
            my_err |= kErrCapacity;
          } else {
            d = a.dist[v];
            if ((uint64_t)d != a.sig[v]) {   // not yet relaxed at its current distance
              a.sig[v] = d;
              e0 = H.rp[v];
              deg = H.rp[v + 1] - e0;
            }
          }
        }
        warp_arcs<true>(deg, e0, ws->table, H.arc, [&](bool valid, uint32_t ol, uint32_t pk) {
          const uint32_t oi = __shfl_sync(kFull, i, ol);
          const uint32_t od = __shfl_sync(kFull, d, ol);
          if (!valid) return;
          SlotArrays a = slot_arrays(sp, slot0 + oi);
          const uint32_t u = pk & 0xFFFFu;
          const uint32_t nd = od + (pk >> 16);
          const uint32_t cur = a.dist[u];
          if ((cur & kFlag) || nd >= cur) return;
          const uint32_t old = atomicMin(&a.dist[u], nd);
          if (nd >= old) return;
          if (nd < dend) {
            improved = true;
            if (old >= dend) {
              const uint32_t pos = warp_append_keyed(&sl[oi].nm, oi);
              if (pos < n) { a.ord[pos] = (uint16_t)u; a.sig[u] = kNoRelax; }
              else my_err |= kErrCapacity;
            }
          } else {
            const uint32_t r2 = (nd >> dsh) & kRingMask;
            const uint32_t bit = 1u << (u & 31u);
            // the old word is not needed: a reduction, off the dependency chain (on the
            // global path the ring lives in device memory)
            atomicOr(&a.ring[r2 * W + (u >> 5)], bit);
            if (!(sl[oi].ring_mask & (1u << r2))) atomicOr(&sl[oi].ring_mask, 1u << r2);
          }
        });
      }
      if (!team.any(improved)) break;
    }
    if (!ok) break;
    // path counts of the bucket.  A member is final once all its predecessors are (earlier
    // buckets are); it then publishes sigma before its flag (fence), and a reader that sees
    // the flag of a same-bucket predecessor fences before reading that sigma.  All arcs of the
    // open members are walked warp-cooperatively, sums through per-warp accumulators (exact
    // 64-bit integers)
    slot_prefix(tc, tid, S, [&](uint32_t i) { return min(sl[i].nm, n) - sl[i].mstart; });
    team.sync();
    const uint32_t total = tc->pref[S];
    const uint32_t dstart = b << dsh;
    for (uint32_t pass = 0;; ++pass) {
      if (pass > n + 1) { my_err |= kErrPassLimit; ok = false; break; }
      bool open = false;
      for (uint32_t base = 0; base < total; base += TS) {
        const uint32_t k = base + lane * NW + warp;   // members interleaved over the warps
        uint32_t i = 0, v = 0, dv = 0, e0 = 0, deg = 0;
        ws->acc[lane] = 0ull;
        ws->flags[lane] = 0u;
        if (k < total) {
          i = find_slot(tc->pref, S, k);
          SlotArrays a = slot_arrays(sp, slot0 + i);
          v = a.ord[sl[i].mstart + k - tc->pref[i]];
          if (v >= n) {
            my_err |= kErrCapacity;
          } else {
            dv = a.dist[v];
            if (!(dv & kFlag)) {
              if (v == sl[i].s) {
                a.sig[v] = 1ull;
                __threadfence_block();
                st_volatile(&a.dist[v], dv | kFlag);
              } else {
                e0 = H.rp[v];
                deg = H.rp[v + 1] - e0;
              }
            }
          }
        }
        // sum sigma over the predecessors; one that is not final yet leaves the member open
        warp_arcs<true>(deg, e0, ws->table, H.arc, [&](bool valid, uint32_t ol, uint32_t pk) {
          const uint32_t oi = __shfl_sync(kFull, i, ol);
          const uint32_t odv = __shfl_sync(kFull, dv, ol);
          if (!valid) return;
          SlotArrays a = slot_arrays(sp, slot0 + oi);
          const uint32_t u = pk & 0xFFFFu;
          const uint32_t du = a.dist[u];
          if ((du & kMask) + (pk >> 16) != odv) return;
          if (!(du & kFlag)) { atomicOr(&ws->flags[ol], 1u); return; }
          if ((du & kMask) >= dstart) __threadfence_block();   // same-bucket predecessor
          const unsigned long long x = a.sig[u];
          const unsigned long long prev = atomicAdd(&ws->acc[ol], x);
          if (prev + x < prev) my_ovf = 1;
        });
        if (deg > 0) {
          SlotArrays a = slot_arrays(sp, slot0 + i);
          if (!(ws->flags[lane] & 1u)) {
            a.sig[v] = ws->acc[lane];
            __threadfence_block();
            st_volatile(&a.dist[v], dv | kFlag);
          } else {
            open = true;
          }
        }
        __syncwarp();
      }
      if (!team.any(open)) break;
    }
    if (!ok) break;
    for (uint32_t i = tid; i < S; i += TS) sl[i].mstart = min(sl[i].nm, n);
    team.sync();
    b += 1;
  }
  if (!ok) {
    if (my_err) atomicOr(err_out, my_err);
    team.sync();
    return false;
  }

  // ---- backward: dependencies, buckets in decreasing order; kFlag = "delta pending"
  // where each bucket's run of the settled list starts: bit p of a bitmap over list
  // positions, set when ord[p] opens a new bucket (kept in the ring words, unused from here on)
  for (uint32_t i = 0; i < S; ++i) {
    SlotArrays a = slot_arrays(sp, slot0 + i);
    const uint32_t cnt = sl[i].mstart;
    for (uint32_t base = 0; base < cnt; base += TS) {   // TS is a multiple of 32
      const uint32_t p = base + tid;
      bool start = false;
      if (p < cnt) {
        const uint32_t v = a.ord[p];
        const uint32_t bv = v < n ? (a.dist[v] & kMask) >> dsh : 0xFFFFFFFFu;
        uint32_t bu = 0xFFFFFFFEu;
        if (p > 0) {
          const uint32_t u = a.ord[p - 1];
          bu = u < n ? (a.dist[u] & kMask) >> dsh : 0xFFFFFFFFu;
        }
        start = bu != bv;
      }
      const uint32_t word = __ballot_sync(kFull, start);
      const uint32_t p0 = base + (tid & ~31u);
      if (lane == 0 && p0 < cnt) a.ring[p0 >> 5] = word;
    }
  }
  for (uint32_t i = tid; i < S; i += TS) sl[i].hi = sl[i].mstart;
  team.sync();
  for (uint32_t guard = 0;; ++guard) {
    if (guard > 2u * n + 2u) { my_err |= kErrPassLimit; ok = false; break; }
    if (tid < 32) {
      uint32_t best = 0;  // 1 + bucket id of the last unprocessed member, 0 if none
      if (lane < S) {
        const uint32_t hi = sl[lane].hi;
        if (hi > 0) {
          SlotArrays a = slot_arrays(sp, slot0 + lane);
          const uint32_t v = a.ord[hi - 1];
          best = v < n ? ((a.dist[v] & kMask) >> dsh) + 1u : 1u;
        }
      }
      best = __reduce_max_sync(kFull, best);
      if (lane == 0) tc->bucket = best;
    }
    team.sync();
    const uint32_t bb = tc->bucket;
    if (bb == 0) break;
    const uint32_t bcur = bb - 1u;
    // per slot: start of the run of bucket bcur at the end of its settled list
    for (uint32_t i = warp; i < S; i += NW) {
      SlotArrays a = slot_arrays(sp, slot0 + i);
      const uint32_t hi = sl[i].hi;
      uint32_t lo = hi;
      const uint32_t vh = hi > 0 ? a.ord[hi - 1] : 0u;
      if (hi > 0 && vh < n && ((a.dist[vh] & kMask) >> dsh) == bcur) {
        // the run's start: the highest start bit at or below position hi - 1 (bit 0 is set),
        // 32 bitmap words per step, lane l taking the l-th word down
        lo = 0;
        const int32_t wtop = (int32_t)((hi - 1u) >> 5);
        for (int32_t w0 = wtop; w0 >= 0; w0 -= 32) {
          const int32_t w = w0 - (int32_t)lane;
          uint32_t word = 0;
          if (w >= 0) {
            word = a.ring[w];
            if (w == wtop) word &= (2u << ((hi - 1u) & 31u)) - 1u;
          }
          const uint32_t nz = __ballot_sync(kFull, word != 0u);
          if (nz) {
            const uint32_t l = __ffs(nz) - 1;
            const uint32_t wl = __shfl_sync(kFull, word, l);
            lo = (uint32_t)(w0 - (int32_t)l) * 32u + 31u - __clz(wl);
            break;
          }
        }
      }
      if (lane == 0) sl[i].lo = lo;
    }
    team.sync();
    slot_prefix(tc, tid, S, [&](uint32_t i) { return sl[i].hi - sl[i].lo; });
    team.sync();
    const uint32_t total = tc->pref[S];
    const uint32_t dhi = (bcur << dsh) + (1u << dsh);
    for (uint32_t pass = 0;; ++pass) {
      if (pass > n + 1) { my_err |= kErrPassLimit; ok = false; break; }
      bool open = false;
      for (uint32_t base = 0; base < total; base += TS) {
        const uint32_t k = base + lane * NW + warp;   // members interleaved over the warps
        uint32_t i = 0, v = 0, dvm = 0, e0 = 0, deg = 0;
        ws->acci[lane] = 0u;      // integral part of the successors' rho
        ws->flags[lane] = 0u;     // bit 0: a successor is still pending
        if (k < total) {
          i = find_slot(tc->pref, S, k);
          SlotArrays a = slot_arrays(sp, slot0 + i);
          v = a.ord[sl[i].lo + k - tc->pref[i]];
          if (v >= n) {
            my_err |= kErrCapacity;
          } else {
            const uint32_t dv = a.dist[v];
            if (dv & kFlag) {
              dvm = dv & kMask;
              e0 = H.rp[v];
              deg = H.rp[v + 1] - e0;
              if (deg == 0) deg = 0x80000000u;   // marker: pending, no arcs
            }
          }
        }
        const bool pending = deg != 0;
        if (deg == 0x80000000u) deg = 0;
        // the successors' rho: integral ones summed exactly, the others by the owner in arc
        // order (so the sum is the same whatever the window split)
        DT acc_f = 0;
        bool any_f = false;
        uint32_t fpm = 0;
        warp_arcs<true>(
            deg, e0, ws->table, H.arc,
            [&](bool valid, uint32_t ol, uint32_t pk) {
              const uint32_t oi = __shfl_sync(kFull, i, ol);
              const uint32_t odv = __shfl_sync(kFull, dvm, ol);
              bool fp = false;
              double x = 0.0;
              if (valid) {
                SlotArrays a = slot_arrays(sp, slot0 + oi);
                const uint32_t w = pk & 0xFFFFu;
                const uint32_t dw = a.dist[w];
                if ((dw & kMask) == odv + (pk >> 16)) {
                  if (dw & kFlag) {
                    atomicOr(&ws->flags[ol], 1u);
                  } else {
                    if ((dw & kMask) < dhi) __threadfence_block();   // same-bucket successor
                    const uint64_t rw = a.sig[w];
                    if (rw & kIntTag) {
                      atomicAdd(&ws->acci[ol], (uint32_t)rw);
                    } else {
                      x = (double)*reinterpret_cast<const DT *>(&rw);
                      fp = true;
                    }
                  }
                }
              }
              fpm = __ballot_sync(kFull, fp);
              if (fpm) ws->buf[lane] = x;
            },
            [&](uint32_t lo, uint32_t hi) {
              if (fpm) {   // warp-uniform
                __syncwarp();
                for (uint32_t t = lo; t < hi; ++t)
                  if ((fpm >> t) & 1u) { acc_f += (DT)ws->buf[t]; any_f = true; }
                __syncwarp();
              }
            });
        if (pending) {
          SlotArrays a = slot_arrays(sp, slot0 + i);
          if (ws->flags[lane] & 1u) {
            open = true;
          } else {
            const uint32_t acc_i = ws->acci[lane];
            const uint64_t sg = a.sig[v];
            const bool is_src = (v == sl[i].s);
            if (sg == 1ull && !any_f) {
              // delta(v) = sum of the successors' subtree sizes: exact in integers
              a.sig[v] = kIntTag | (uint64_t)(1u + acc_i);
              if (!is_src && acc_i) atomicAdd(&acc.a0[v], (unsigned long long)acc_i);
            } else {
              DT dep, rho;
              dependency<DT>(sg, (DT)acc_i + acc_f, dep, rho);
              uint64_t bits = 0;
              *reinterpret_cast<DT *>(&bits) = rho;
              a.sig[v] = bits;
              if (!is_src) fx_red(acc.a0, acc.a1, acc.a2, v, (double)dep);
            }
            __threadfence_block();
            st_volatile(&a.dist[v], dvm);
          }
        }
        __syncwarp();
      }
      if (!team.any(open)) break;
    }
    if (!ok) break;
    for (uint32_t i = tid; i < S; i += TS) sl[i].hi = sl[i].lo;
    team.sync();
  }
  if (my_err) atomicOr(err_out, my_err);
  if (my_ovf) atomicOr(ovf_out, 1u);
  team.sync();
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
  if (P.wtab_ptr) {
    // discrete law: lo + #{thresholds <= u}, capped at hi; the thresholds are non-decreasing,
    // so the count is the upper-bound position (a binary search: its short loop also keeps
    // the counting kernel's register allocation lower than a linear count does)
    uint32_t a = P.wtab_ptr[e], b = P.wtab_ptr[e + 1];
    const uint32_t a0 = a;
    while (a < b) {
      const uint32_t mid = (a + b) >> 1;
      if (P.wtab[mid] <= u.y) a = mid + 1; else b = mid;
    }
    w = min(lo + (a - a0), hi);
  } else {
    w = lo + (uint32_t)(((uint64_t)u.y * ((uint64_t)hi - lo + 1u)) >> 32);
  }
}

// Item r_local of a problem: its realization index and, in the row-wise mode (independent
// draws per row, Alg. 2), its anchor (draw m of row i uses realization m n + i); otherwise
// anchor = 0xFFFFFFFF and the realization serves every row.
__device__ __forceinline__ uint32_t item_rho(const McDev &P, uint32_t r_local, uint32_t &anchor) {
  if (!P.per_row) {
    anchor = 0xFFFFFFFFu;
    return P.r_begin + r_local;
  }
  const uint32_t n = (uint32_t)P.n;
  anchor = r_local % n;
  return (P.r_begin + r_local / n) * n + anchor;
}

// Hop distances from the anchor in the base graph, up to P.hop_radius (0xFFFFFFFF beyond):
// the neighbourhood S_r(i) of the r-hop mode.  Level-synchronous; a node reached twice in one
// level gets the same value from every writer.
__device__ inline void hop_ball(const McDev &P, uint32_t anchor, uint32_t *hop) {
  const uint32_t n = (uint32_t)P.n;
  for (uint32_t v = threadIdx.x; v < n; v += blockDim.x) hop[v] = v == anchor ? 0u : 0xFFFFFFFFu;
  __syncthreads();
  for (uint32_t lev = 0; lev < P.hop_radius; ++lev) {
    for (uint32_t v = threadIdx.x; v < n; v += blockDim.x) {
      if (hop[v] != lev) continue;
      for (int32_t a = P.row_ptr[v]; a < P.row_ptr[v + 1]; ++a) {
        const uint32_t u = (uint32_t)P.col[a];
        if (u < n && hop[u] == 0xFFFFFFFFu) hop[u] = lev + 1;
      }
    }
    __syncthreads();
  }
}

// Row-wise mode: only the anchor's component stays valid (the other components neither
// contribute sources nor report).
__device__ inline void keep_anchor_component(uint32_t n, uint32_t anchor, const uint32_t *comp,
                                             uint32_t *cinfo) {
  const uint32_t ra = comp[anchor];
  for (uint32_t v = threadIdx.x; v < n; v += blockDim.x)
    if (comp[v] == v && v != ra) cinfo[v] &= ~kHasCand;
  __syncthreads();
}

// Builds the alive-compacted CSR of realization r into rp/arc (thread per contiguous vertex
// range, offsets from one block scan) and the largest alive length into ctl->wmax.  With hop
// distances given, only arcs between nodes within P.hop_radius of the anchor are kept.
__device__ inline void realize_csr(const McDev &P, uint32_t r, uint32_t *rp, uint32_t *arc,
                            CtaHead *ctl, const uint32_t *hop = nullptr) {
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
      if (hop && (hop[v] > P.hop_radius || (uint32_t)P.col[a] >= n ||
                  hop[P.col[a]] > P.hop_radius)) continue;
      bool alive; uint32_t w;
      edge_draw(P, r, e, alive, w);
      cnt += alive ? 1u : 0u;
    }
  }
  uint32_t off = block_exclusive_scan(cnt, ctl->scan, &ctl->scan_total);
  uint32_t wmax = 1, err = 0;
  for (uint32_t v = v0; v < v1; ++v) {
    rp[v] = off;
    const int32_t a0 = P.row_ptr[v], a1 = P.row_ptr[v + 1];
    for (int32_t a = a0; a < a1; ++a) {
      const uint32_t e = (uint32_t)P.eid[a];
      const uint32_t u = (uint32_t)P.col[a];
      if (e >= (uint64_t)P.m || u >= n) { err = kErrInput; continue; }
      if (hop && (hop[v] > P.hop_radius || hop[u] > P.hop_radius)) continue;
      bool alive; uint32_t w;
      edge_draw(P, r, e, alive, w);
      if (!alive) continue;
      if (w == 0 || w > 0xFFFFu || off >= cap) { err = kErrInput; continue; }
      arc[off++] = u | (w << 16);
      wmax = max(wmax, w);
    }
  }
  if (err) atomicOr(&ctl->err, err);
  wmax = __reduce_max_sync(kFull, wmax);
  if ((threadIdx.x & 31u) == 0) atomicMax(&ctl->wmax, wmax);
  const uint32_t total = ctl->scan_total;
  if (threadIdx.x == 0) rp[n] = total < cap ? total : cap;
  __syncthreads();
}

// Root of x.  Volatile loads: parents change under concurrent hooks (also in global memory,
// where a cached line could otherwise hide a hook and make the CAS loop retry forever).
__device__ __forceinline__ uint32_t uf_find(const uint32_t *parent, uint32_t x) {
  const volatile uint32_t *vp = parent;
  uint32_t p = vp[x];
  while (p != x) {
    x = p;
    p = vp[x];
  }
  return x;
}

// comp[v] <- smallest id of v's component; cinfo[root] <- size | has-candidate bit.
__device__ inline void components(const McDev &P, const Realized &H, uint32_t *comp, uint32_t *cinfo) {
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

// Bucket width Delta: the smallest power of two that is at least the requested width and at
// least ceil(wmax / (kRing - 2)).  A relaxation out of bucket b reaches at most
// (b + 1) * Delta - 1 + wmax < (b + kRing) * Delta, so every discovered distance beyond the
// current bucket has its own entry in the ring of kRing bucket bitmaps; powers of two turn the
// bucket and ring arithmetic into shifts and masks.
__device__ __forceinline__ void bucket_setup(CtaHead *ctl, uint32_t delta_req) {
  if (threadIdx.x == 0) {
    const uint32_t wmax = ctl->wmax;
    const uint32_t dmin = (wmax + (kRing - 2) - 1) / (kRing - 2);
    const uint32_t want = max(max(delta_req, 1u), dmin);
    uint32_t sh = 0;
    while ((1u << sh) < want && sh < 30u) ++sh;
    ctl->dsh = sh;
    ctl->delta = 1u << sh;
  }
  __syncthreads();
}

// ---------------------------------------------------------------------------------------
// Select (A6) and count.  Scratch: slot 0's sig (u64 per root), slot 0's dist (centre per
// root), the layout's sel array (rank per root).  Returns true when the FP32 gap test asks
// for an FP64 recheck (then nothing is committed).
// ---------------------------------------------------------------------------------------
__device__ inline bool select_and_count(const McDev &P, uint32_t r_local, const uint32_t *comp,
                                        const uint32_t *cinfo, const double *bc, SlotArrays s0,
                                        uint32_t *rank, uint16_t *mark, bool gap_test,
                                        CtaHead *ctl) {
  const uint32_t n = P.n;
  unsigned long long *best = reinterpret_cast<unsigned long long *>(s0.sig);
  uint32_t *centre = s0.dist;
  if (threadIdx.x == 0) ctl->need_recheck = 0;
  if (P.reward_k || P.report_rank > 1) {
    // Ordered local Top-k (Sec. 2.3 eq. topk-comp): round t picks the tie-broken centre of the
    // nodes of K not picked before (B* over the remaining nodes, relative band, smallest id).
    // Round report_rank - 1 gives the reported node (rank-r centre), rounds below reward_k the
    // valued Top-k step reward of every anchor of K (Sec. 6.2, pool-restricted: Sec. 6.3).
    // The host admits this mode only in FP64, without a candidate pool or rank cutoff, where
    // round 0 is exactly the centre rule below.
    const uint32_t rr = P.report_rank > 1 ? P.report_rank : 1u;
    const uint32_t rounds = P.reward_k > rr ? P.reward_k : rr;
    uint32_t *pick = rank;   // per root: node picked in the current round
    for (uint32_t v = threadIdx.x; v < n; v += blockDim.x) { mark[v] = 0; centre[v] = 0xFFFFFFFFu; }
    for (uint32_t t = 0; t < rounds; ++t) {
      for (uint32_t v = threadIdx.x; v < n; v += blockDim.x) { best[v] = 0ull; pick[v] = 0xFFFFFFFFu; }
      __syncthreads();
      for (uint32_t v = threadIdx.x; v < n; v += blockDim.x) {
        const uint32_t root = comp[v];
        if (comp_valid(cinfo[root], P.k_min) && !mark[v])
          atomicMax(&best[root], (unsigned long long)__double_as_longlong(bc[v]));
      }
      __syncthreads();
      for (uint32_t v = threadIdx.x; v < n; v += blockDim.x) {
        const uint32_t root = comp[v];
        if (!comp_valid(cinfo[root], P.k_min) || mark[v]) continue;
        const double bstar = __longlong_as_double((long long)best[root]);
        if (bc[v] >= bstar - P.tie_rel * bstar) atomicMin(&pick[root], v);
      }
      __syncthreads();
      for (uint32_t v = threadIdx.x; v < n; v += blockDim.x) {
        if (comp[v] == v && pick[v] < n) {
          mark[pick[v]] = 1;
          if (t == rr - 1) centre[v] = pick[v];
        }
        if (t < P.reward_k && P.psi) {
          const uint32_t p = pick[comp[v]];
          if (p < n && (P.reward_pool == nullptr || P.reward_pool[p]))
            atomicAdd(&P.psi[v], P.reward_gamma ? P.reward_gamma[p] : 1.0);
        }
      }
      __syncthreads();
    }
    for (uint32_t v = threadIdx.x; v < n; v += blockDim.x) rank[v] = 1u;
    __syncthreads();
  } else {
  for (uint32_t v = threadIdx.x; v < n; v += blockDim.x) {
    best[v] = 0ull; centre[v] = 0xFFFFFFFFu; rank[v] = 1u;
  }
  __syncthreads();
  for (uint32_t v = threadIdx.x; v < n; v += blockDim.x) {
    const uint32_t root = comp[v];
    if (!comp_valid(cinfo[root], P.k_min)) continue;
    if (P.in_w == nullptr || P.in_w[v])
      atomicMax(&best[root], (unsigned long long)__double_as_longlong(bc[v]));
  }
  __syncthreads();
  for (uint32_t v = threadIdx.x; v < n; v += blockDim.x) {
    const uint32_t root = comp[v];
    if (!comp_valid(cinfo[root], P.k_min)) continue;
    if (!(P.in_w == nullptr || P.in_w[v])) continue;
    const double bstar = __longlong_as_double((long long)best[root]);
    if (bc[v] >= bstar - P.tie_rel * bstar) {
      atomicMin(&centre[root], v);
      if (P.tie_random) atomicAdd(&rank[root], 1u);   // 1 + number of ties
    }
  }
  __syncthreads();
  if (P.tie_random) {
    // uniformly randomised tie-break (Remark on randomized tie-breaking, Sec. 4.1): the
    // floor(u |ties| / 2^32)-th tied candidate in ascending id, u from Philox counter
    // (root, realization, graph tag, 3); the root is the smallest id of its component
    for (uint32_t v = threadIdx.x; v < n; v += blockDim.x) {
      if (comp[v] != v || !comp_valid(cinfo[v], P.k_min)) continue;
      const uint32_t ties = rank[v] - 1u;
      if (ties < 2u) continue;
      uint32_t anchor_unused;
      const uint4 u = philox4x32_10(make_uint4(v, item_rho(P, r_local, anchor_unused),
                                               P.graph_tag, 3u), P.key_lo, P.key_hi);
      uint32_t k = (uint32_t)(((uint64_t)u.x * (uint64_t)ties) >> 32);
      const double bstar = __longlong_as_double((long long)best[v]);
      for (uint32_t w = v; w < n && k > 0u; ++w) {
        if (comp[w] != v || !(P.in_w == nullptr || P.in_w[w])) continue;
        if (bc[w] < bstar - P.tie_rel * bstar) continue;
        if (--k == 0u) {
          // the next tied candidate after w
          for (uint32_t x = w + 1; x < n; ++x)
            if (comp[x] == v && (P.in_w == nullptr || P.in_w[x]) &&
                bc[x] >= bstar - P.tie_rel * bstar) { centre[v] = x; break; }
        }
      }
    }
    __syncthreads();
    for (uint32_t v = threadIdx.x; v < n; v += blockDim.x) rank[v] = 1u;
    __syncthreads();
  }
  if (P.top_k || gap_test) {
    if (P.top_k) {   // best now becomes the maximum over the whole component
      for (uint32_t v = threadIdx.x; v < n; v += blockDim.x) best[v] = 0ull;
      __syncthreads();
      for (uint32_t v = threadIdx.x; v < n; v += blockDim.x) {
        const uint32_t root = comp[v];
        if (comp_valid(cinfo[root], P.k_min))
          atomicMax(&best[root], (unsigned long long)__double_as_longlong(bc[v]));
      }
      __syncthreads();
    }
    for (uint32_t v = threadIdx.x; v < n; v += blockDim.x) {
      const uint32_t root = comp[v];
      if (!comp_valid(cinfo[root], P.k_min)) continue;
      const uint32_t c = centre[root];
      if (c == v || c >= n) continue;
      if (P.top_k) {
        const double tauK = P.tie_rel * __longlong_as_double((long long)best[root]);
        const double diff = bc[v] - bc[c];
        if (diff > tauK || (fabs(diff) <= tauK && v < c)) atomicAdd(&rank[root], 1u);
      }
      if (gap_test && (P.top_k || P.in_w == nullptr || P.in_w[v])) {
        // top-two gap of the candidate set (of the whole component when a rank cutoff is
        // active): another node within the margin of B1 sends the realization to FP64
        const double b1 = bc[c];
        if (b1 > 0.0 && fabs(b1 - bc[v]) < P.recheck_margin * b1) ctl->need_recheck = 1;
      }
    }
    __syncthreads();
  }
  }
  if (gap_test && ctl->need_recheck) return true;
  uint32_t *counts = P.counts;
  const size_t stride = (size_t)n + 1;
  uint32_t anchor;
  item_rho(P, r_local, anchor);
  for (uint32_t i = threadIdx.x; i < n; i += blockDim.x) {
    if (anchor != 0xFFFFFFFFu && i != anchor) continue;   // row-wise mode: the anchor's row only
    const uint32_t root = comp[i];
    uint32_t col = n;
    const uint32_t info = cinfo[root];
    if ((info & kSizeMask) >= P.k_min) {
      // a component without a candidate of W has no centre (and no betweenness was computed)
      const uint32_t c = (info & kHasCand) ? centre[root] : 0xFFFFFFFFu;
      if (c < n && (P.top_k == 0 || rank[root] <= P.top_k)) {
        col = c;
      } else if (P.fb_node < n) {   // Sel_{W,fb} (Sec. 7.3): valid but infeasible -> v_fb
        col = P.fb_node;
        if (P.fb_count) atomicAdd(&P.fb_count[i], 1u);
      }
    }
    atomicAdd(&counts[(size_t)i * stride + col], 1u);
    if (P.dump_next) P.dump_next[(size_t)r_local * n + i] = (int32_t)col;
  }
  if (P.dump_bc)
    for (uint32_t v = threadIdx.x; v < n; v += blockDim.x)
      P.dump_bc[(size_t)r_local * n + v] = bc[v];
  return false;
}

}  // namespace afc
