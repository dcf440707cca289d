// w1.cu -- Wasserstein-1 distances under a graph's hop metric on the device, the second
// discrepancy of the sampled robust search (Sec. 9 robust experiment).
//
// With the shortest-path metric of an unweighted graph, W1(x, y) is the cost of the cheapest
// flow over the graph's edges (one unit of cost per unit of mass per edge, no capacities) that
// turns x into y.  Each warp solves one row x_k exactly by the primal-dual method for
// min-cost flow, in phases:
//   1. Dijkstra from every node with excess mass over the residual graph, with the reduced
//      costs c(u,v) + pi_u - pi_v >= 0 (c = +1 for a new unit on u -> v, -1 for cancelling
//      flow that runs v -> u), level by level, stopping at the first level that holds a node
//      with a deficit (distance D);
//   2. potentials pi_v += min(d_v, D): every shortest path to a deficit now has reduced cost 0
//      on all its arcs, and no residual arc has a negative one;
//   3. the zero-reduced-cost arcs layered by hop count from the excess nodes up to the first
//      layer with a deficit, pruned backwards to the nodes that reach a deficit in the next
//      layers, and a blocking flow on them (Dinic): a warp-cooperative depth-first search with
//      current-arc pointers, each augmentation moving min(source excess, sink deficit,
//      cancelled flow on the path) and retreating to the first arc it used up.
// Costs are integers, so distances and potentials are exact; masses are doubles, settled to a
// relative 1e-14 of the largest |x_v - y_v|.  The result is sum_e |flow_e| (an exact
// minimiser's cost), summed in a fixed order.  The levels and layers advance through
// appended frontier lists, so a phase costs a few passes over the arcs it reaches.
#include <cfloat>
#include <cstdint>
#include <cuda_runtime.h>

#include "afc_internal.h"

namespace afc {
namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int32_t kInf = 0x3fffffff;
constexpr int32_t kDead = -2;           // layer mark of a node that reaches no deficit
constexpr uint32_t kW1Leftover = 1u;    // excess left that reaches no deficit
constexpr uint32_t kW1Limit = 2u;       // a phase or search-step bound was hit
constexpr uint32_t kW1Invariant = 4u;   // a negative reduced cost or a missing zero-cost path

__host__ __device__ inline size_t al16w(size_t x) { return (x + 15u) & ~size_t(15); }

// One warp's state for one row (shared memory when it fits, else the warp's device slab),
// and the graph it reads (a shared-memory copy when that fits too).
struct W1Slot {
  double *ex;       // [n] excess x - y, driven to zero
  double *g;        // [m] signed flow of edge e: positive from its lower-id end to its higher
  int32_t *pot;     // [n] potentials
  int32_t *dist;    // [n] Dijkstra distance, then the hop layer (-1 none, kDead)
  int32_t *cur;     // [n] current arc of the depth-first search
  int32_t *stk;     // [n+1] layer offsets into ord, then the search path
  int32_t *ord;     // [n] settled nodes in order; the layers in order
  uint8_t *done;    // [n] settled by the Dijkstra
  uint32_t *ctr;    // append counter of ord
  const int32_t *rp, *col, *eid;
};

__host__ __device__ inline size_t slot_bytes(int32_t n, int64_t m) {
  const size_t nn = (size_t)(n > 0 ? n : 1), mm = (size_t)(m > 0 ? m : 1);
  return al16w(8 * nn) + al16w(8 * mm) + 3 * al16w(4 * nn) + al16w(4 * (nn + 1)) +
         al16w(4 * nn) + al16w(nn) + 16;
}

__host__ __device__ inline size_t graph_bytes(int32_t n, int64_t m) {
  const size_t nn = (size_t)(n > 0 ? n : 1), mm = (size_t)(m > 0 ? m : 1);
  return al16w(4 * (nn + 1)) + 2 * al16w(8 * mm);
}

__device__ inline W1Slot carve(unsigned char *p, int32_t n, int64_t m) {
  const size_t nn = (size_t)(n > 0 ? n : 1), mm = (size_t)(m > 0 ? m : 1);
  W1Slot s;
  s.ex = reinterpret_cast<double *>(p);    p += al16w(8 * nn);
  s.g = reinterpret_cast<double *>(p);     p += al16w(8 * mm);
  s.pot = reinterpret_cast<int32_t *>(p);  p += al16w(4 * nn);
  s.dist = reinterpret_cast<int32_t *>(p); p += al16w(4 * nn);
  s.cur = reinterpret_cast<int32_t *>(p);  p += al16w(4 * nn);
  s.stk = reinterpret_cast<int32_t *>(p);  p += al16w(4 * (nn + 1));
  s.ord = reinterpret_cast<int32_t *>(p);  p += al16w(4 * nn);
  s.done = p;                              p += al16w(nn);
  s.ctr = reinterpret_cast<uint32_t *>(p);
  return s;
}

// The residual arc u -> v of edge e: cancelling flow that runs v -> u (cost -1, capacity that
// flow) when more than tol of it runs, else a new unit on u -> v (cost +1, no capacity).
__device__ __forceinline__ int32_t arc_cost(const W1Slot &S, int32_t u, int32_t v, int32_t e,
                                            double tol, double &cap) {
  const double gf = u < v ? S.g[e] : -S.g[e];   // flow in the direction u -> v
  if (gf < -tol) {
    cap = -gf;
    return -1;
  }
  cap = DBL_MAX;
  return 1;
}

__device__ __forceinline__ double warp_sum_d(double x) {
  for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(kFull, x, o);
  return x;
}

__device__ __forceinline__ double warp_max_d(double x) {
  for (int o = 16; o > 0; o >>= 1) x = fmax(x, __shfl_xor_sync(kFull, x, o));
  return x;
}

__device__ __forceinline__ double warp_min_d(double x) {
  for (int o = 16; o > 0; o >>= 1) x = fmin(x, __shfl_xor_sync(kFull, x, o));
  return x;
}

// Appends the nodes v < n with pred(v), in increasing order, to S.ord at position `at`;
// returns the new end (all lanes).
template <typename Pred>
__device__ __forceinline__ uint32_t collect(const W1Slot &S, int32_t n, uint32_t at, Pred pred) {
  const uint32_t lane = threadIdx.x & 31u;
  for (int32_t v0 = 0; v0 < n; v0 += 32) {
    const int32_t v = v0 + (int32_t)lane;
    const bool f = v < n && pred(v);
    const uint32_t bal = __ballot_sync(kFull, f);
    if (f) S.ord[at + __popc(bal & ((1u << lane) - 1u))] = v;
    at += __popc(bal);
  }
  __syncwarp();
  return at;
}

// Solves one row: returns W1 (all lanes) and ORs failure bits into err.
__device__ double w1_row(const W1Slot &S, int32_t n, int64_t m, const double *xk,
                         const double *y, uint32_t &err) {
  const int32_t lane = (int32_t)(threadIdx.x & 31u);
  const int32_t *rp = S.rp, *col = S.col, *eid = S.eid;
  double scale = 0.0, pos = 0.0;
  for (int32_t v = lane; v < n; v += 32) {
    const double e = xk[v] - y[v];
    S.ex[v] = e;
    S.pot[v] = 0;
    scale = fmax(scale, fabs(e));
    pos += e > 0.0 ? e : 0.0;
  }
  for (int64_t e = lane; e < m; e += 32) S.g[e] = 0.0;
  scale = warp_max_d(scale);
  pos = warp_sum_d(pos);
  const double tol = 1e-14 * fmax(scale, 1e-300);
  __syncwarp();
  uint32_t bad = 0;
  const int64_t phase_limit = 4 * ((int64_t)n + m) + 64;
  for (int64_t phase = 0;; ++phase) {
    if (phase >= phase_limit) {
      bad |= kW1Limit;
      break;
    }
    // 1. Dijkstra by levels from every node with excess; ord receives the nodes in the order
    //    they settle, a level's frontier being the window [head, tail)
    for (int32_t v = lane; v < n; v += 32) {
      S.dist[v] = S.ex[v] > tol ? 0 : kInf;
      S.done[v] = 0;
    }
    __syncwarp();
    uint32_t tail = collect(S, n, 0, [&](int32_t v) { return S.dist[v] == 0; });
    if (tail == 0) break;   // no excess left
    if (lane == 0) *S.ctr = tail;
    uint32_t head = 0;
    int32_t L = 0, D = kInf;
    for (;;) {
      bool sink = false;
      while (head < tail) {
        for (uint32_t i = head + lane; i < tail; i += 32) {
          const int32_t u = S.ord[i];
          S.done[u] = 1;
          sink |= S.ex[u] < -tol;
        }
        __syncwarp();
        if (__any_sync(kFull, sink)) break;
        for (uint32_t i = head + lane; i < tail; i += 32) {
          const int32_t u = S.ord[i], pu = S.pot[u];
          for (int32_t a = rp[u]; a < rp[u + 1]; ++a) {
            const int32_t v = col[a];
            if (S.done[v]) continue;
            double cap;
            int32_t rc = arc_cost(S, u, v, eid[a], tol, cap) + pu - S.pot[v];
            if (rc < 0) {
              bad |= kW1Invariant;
              rc = 0;
            }
            const int32_t old = atomicMin(&S.dist[v], L + rc);
            if (rc == 0 && old > L) S.ord[atomicAdd(S.ctr, 1u)] = v;   // joins level L
          }
        }
        __syncwarp();
        head = tail;
        tail = *S.ctr;
        __syncwarp();
      }
      if (__any_sync(kFull, sink)) {
        D = L;
        break;
      }
      int32_t nl = kInf;
      for (int32_t v = lane; v < n; v += 32)
        if (!S.done[v]) nl = min(nl, S.dist[v]);
      nl = __reduce_min_sync(kFull, nl);
      if (nl >= kInf) break;
      L = nl;
      tail = collect(S, n, tail, [&](int32_t v) { return !S.done[v] && S.dist[v] == nl; });
      if (lane == 0) *S.ctr = tail;
      __syncwarp();
    }
    if (D >= kInf) break;   // what excess is left reaches no deficit
    // 2. potentials
    for (int32_t v = lane; v < n; v += 32) S.pot[v] += S.done[v] ? S.dist[v] : D;
    __syncwarp();
    // 3a. hop layers of the zero-reduced-cost arcs, up to the first layer with a deficit;
    //     layer h is ord[stk[h] .. stk[h+1])
    for (int32_t v = lane; v < n; v += 32) S.dist[v] = S.ex[v] > tol ? 0 : -1;
    __syncwarp();
    tail = collect(S, n, 0, [&](int32_t v) { return S.dist[v] == 0; });
    if (lane == 0) {
      *S.ctr = tail;
      S.stk[0] = 0;
    }
    head = 0;
    int32_t h = 0;
    bool reached = false;
    while (head < tail && !reached) {
      bool r = false;
      for (uint32_t i = head + lane; i < tail; i += 32) {
        const int32_t u = S.ord[i], pu = S.pot[u];
        for (int32_t a = rp[u]; a < rp[u + 1]; ++a) {
          const int32_t v = col[a];
          if (S.dist[v] != -1) continue;
          double cap;
          if (arc_cost(S, u, v, eid[a], tol, cap) + pu - S.pot[v] != 0) continue;
          if (atomicCAS(&S.dist[v], -1, h + 1) == -1) {
            S.ord[atomicAdd(S.ctr, 1u)] = v;
            r |= S.ex[v] < -tol;
          }
        }
      }
      __syncwarp();
      reached = __any_sync(kFull, r);
      head = tail;
      tail = *S.ctr;
      ++h;
      if (lane == 0) S.stk[h] = (int32_t)head;
      __syncwarp();
    }
    if (!reached) {   // a shortest path of reduced cost 0 exists after step 2
      bad |= kW1Invariant;
      break;
    }
    const int32_t hmax = h;
    if (lane == 0) S.stk[hmax + 1] = (int32_t)tail;
    __syncwarp();
    // 3b. prune: the last layer keeps its deficits, every earlier node an arc into a kept node
    //     of the next layer
    for (int32_t i = S.stk[hmax] + lane; i < S.stk[hmax + 1]; i += 32) {
      const int32_t u = S.ord[i];
      if (!(S.ex[u] < -tol)) S.dist[u] = kDead;
    }
    __syncwarp();
    for (int32_t l = hmax - 1; l >= 0; --l) {
      for (int32_t i = S.stk[l] + lane; i < S.stk[l + 1]; i += 32) {
        const int32_t u = S.ord[i], pu = S.pot[u];
        bool keep = false;
        for (int32_t a = rp[u]; a < rp[u + 1] && !keep; ++a) {
          const int32_t v = col[a];
          if (S.dist[v] != l + 1) continue;
          double cap;
          keep = arc_cost(S, u, v, eid[a], tol, cap) + pu - S.pot[v] == 0;
        }
        if (!keep) S.dist[u] = kDead;
      }
      __syncwarp();
    }
    // 3c. blocking flow from the kept excess nodes
    for (int32_t v = lane; v < n; v += 32) S.cur[v] = rp[v];
    __syncwarp();
    int64_t steps = 0;
    const int64_t step_limit = 2 * (3 * (int64_t)n + m + 64) * (hmax + 2);
    for (int32_t s0 = 0; s0 < n && !bad; s0 += 32) {
      const int32_t vv = s0 + lane;
      uint32_t srcs = __ballot_sync(kFull, vv < n && S.dist[vv] == 0 && S.ex[vv] > tol);
      while (srcs && !bad) {
        const int32_t s = s0 + __ffs(srcs) - 1;
        srcs &= srcs - 1u;
        int32_t top = 0, u = s;
        if (lane == 0) S.stk[0] = s;
        __syncwarp();
        while (S.ex[s] > tol) {
          if (++steps > step_limit) {
            bad |= kW1Limit;
            break;
          }
          if (top > 0 && S.ex[u] < -tol) {
            // augment along stk[0..top]; then retreat to the tail of the first arc used up
            double delta = fmin(S.ex[s], -S.ex[u]);
            for (int32_t i = lane; i < top; i += 32) {
              const int32_t w = S.stk[i], a = S.cur[w];
              double cap;
              arc_cost(S, w, col[a], eid[a], tol, cap);
              delta = fmin(delta, cap);
            }
            delta = warp_min_d(delta);
            int32_t first = top;
            for (int32_t i0 = 0; i0 < top; i0 += 32) {
              const int32_t i = i0 + lane;
              bool used = false;
              if (i < top) {
                const int32_t w = S.stk[i], a = S.cur[w];
                double cap;
                used = arc_cost(S, w, col[a], eid[a], tol, cap) < 0 && cap == delta;
              }
              const uint32_t b = __ballot_sync(kFull, used);
              if (b) {
                first = i0 + __ffs(b) - 1;
                break;
              }
            }
            __syncwarp();
            for (int32_t i = lane; i < top; i += 32) {
              const int32_t w = S.stk[i], a = S.cur[w];
              S.g[eid[a]] += w < col[a] ? delta : -delta;
            }
            if (lane == 0) {
              S.ex[s] -= delta;
              S.ex[u] += delta;
            }
            __syncwarp();
            if (first < top) {
              top = first;
              u = S.stk[top];
            }
            continue;   // else the sink is met (it is dropped next) or the source is empty
          }
          // advance along the first admissible arc at or after cur[u] into the next layer
          const int32_t lu = S.dist[u], a1 = rp[u + 1];
          int32_t next = -1;
          if (lu >= 0 && lu < hmax) {
            const int32_t pu = S.pot[u];
            for (int32_t a0 = S.cur[u]; a0 < a1; a0 += 32) {
              const int32_t a = a0 + lane;
              bool ok = false;
              if (a < a1) {
                const int32_t z = col[a];
                if (S.dist[z] == lu + 1) {
                  double cap;
                  ok = arc_cost(S, u, z, eid[a], tol, cap) + pu - S.pot[z] == 0;
                }
              }
              const uint32_t b = __ballot_sync(kFull, ok);
              if (b) {
                next = a0 + __ffs(b) - 1;
                break;
              }
            }
          }
          if (next >= 0) {
            const int32_t z = col[next];
            if (lane == 0) {
              S.cur[u] = next;
              S.stk[top + 1] = z;
            }
            __syncwarp();
            ++top;
            u = z;
          } else {
            if (lane == 0) {
              S.cur[u] = a1;
              S.dist[u] = kDead;
            }
            __syncwarp();
            if (top == 0) break;   // no path left from s in this phase
            --top;
            u = S.stk[top];
          }
        }
      }
    }
    bad = __reduce_or_sync(kFull, bad);
    if (bad) break;
  }
  bad = __reduce_or_sync(kFull, bad);
  double left = 0.0;
  for (int32_t v = lane; v < n; v += 32) left += S.ex[v] > tol ? S.ex[v] : 0.0;
  left = warp_sum_d(left);
  if (left > 1e-9 * fmax(pos, 1e-300)) bad |= kW1Leftover;
  double w = 0.0;
  for (int64_t e = lane; e < m; e += 32) w += fabs(S.g[e]);
  err |= bad;
  return warp_sum_d(w);
}

// mode 2: row state and graph in shared memory; 1: row state only; 0: both in device memory
__global__ void __launch_bounds__(32, 16)
w1_kernel(int32_t n, int64_t m, const int32_t *rp, const int32_t *col, const int32_t *eid,
          const double *x, const double *y, int32_t count, double *out, unsigned char *slab,
          size_t stride, int mode, uint32_t *status) {
  extern __shared__ __align__(16) unsigned char smem[];
  unsigned char *base = mode ? smem : slab + (size_t)blockIdx.x * stride;
  W1Slot S = carve(base, n, m);
  S.rp = rp;
  S.col = col;
  S.eid = eid;
  if (mode == 2) {
    const size_t nn = (size_t)(n > 0 ? n : 1), mm = (size_t)(m > 0 ? m : 1);
    unsigned char *g = smem + slot_bytes(n, m);
    int32_t *srp = reinterpret_cast<int32_t *>(g);
    int32_t *scol = reinterpret_cast<int32_t *>(g + al16w(4 * (nn + 1)));
    int32_t *seid = reinterpret_cast<int32_t *>(g + al16w(4 * (nn + 1)) + al16w(8 * mm));
    for (int32_t i = threadIdx.x; i <= n; i += 32) srp[i] = rp[i];
    for (int64_t a = threadIdx.x; a < 2 * m; a += 32) {
      scol[a] = col[a];
      seid[a] = eid[a];
    }
    __syncwarp();
    S.rp = srp;
    S.col = scol;
    S.eid = seid;
  }
  uint32_t err = 0;
  for (int32_t k = blockIdx.x; k < count; k += gridDim.x) {
    const double w = w1_row(S, n, m, x + (size_t)k * (size_t)n, y, err);
    if (threadIdx.x == 0) out[k] = w;
    __syncwarp();
  }
  if (threadIdx.x == 0 && err) atomicOr(status, err);
}

}  // namespace

size_t w1_slot_bytes(int32_t n, int64_t m) { return slot_bytes(n, m); }
size_t w1_graph_bytes(int32_t n, int64_t m) { return graph_bytes(n, m); }

cudaError_t launch_w1(int32_t n, int64_t m, const int32_t *rp, const int32_t *col,
                      const int32_t *eid, const double *x, const double *y, int32_t count,
                      double *out, unsigned char *slab, int mode, int grid, uint32_t *status,
                      cudaStream_t stream) {
  if (count <= 0) return cudaSuccess;
  const size_t slot = slot_bytes(n, m);
  const int dyn = mode == 2 ? (int)(slot + graph_bytes(n, m)) : mode == 1 ? (int)slot : 0;
  cudaFuncSetAttribute(w1_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, dyn);
  w1_kernel<<<grid, 32, dyn, stream>>>(n, m, rp, col, eid, x, y, count, out, slab, slot, mode,
                                       status);
  return cudaGetLastError();
}

}  // namespace afc
