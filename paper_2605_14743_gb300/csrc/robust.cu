// robust.cu -- robust analysis on the estimated AMC.
//
// Device (Sec. 8 post-processing; uncertainty set of Sec. 5.1):
//   robust_inner_kernel  T_i(v) = inf over q_i in U_i of sum_j q_ij v_j + (1 - sum_j q_ij) v_bot,
//                        U_i the box [(Q0_ij - eps)_+, min(Q0_ij + eps, 1)] (on the row's
//                        support, or on every j) with sum_j q_ij <= 1 - r_min.  A warp per row
//                        solves the LP exactly: every entry starts at its lower bound, then the
//                        budget goes to the entries in ascending order of v_j - v_bot (ties by
//                        j) while that coefficient is negative, each up to its upper bound.
//   eval_kernel          one CTA: A = I - Q*, V = A^-1 f (blocked FP64 LU with partial pivoting) and
//                        the change of V; the robust value comes from policy iteration on the
//                        host (inner problem at V, evaluate, until V stops changing)
//   star_kernel          the AFC of the scenario kernel: A^T mu = s with the last factors
// Host (Sec. 9 robust experiment): the Wasserstein-1 distance between two node distributions
// under the base graph's hop metric.
//
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <functional>
#include <limits>
#include <queue>
#include <utility>
#include <vector>

#include <cuda_runtime.h>

#include "afc_internal.h"
#include "linalg.cuh"

namespace afc {

namespace {

// The transient row of the estimated kernel: Q0_ij = scale_i counts_ij with the assembly's
// row-scale rule.  Returns scale_i; the warp's lanes all get it.
__device__ double row_scale_warp(const uint32_t *row, int32_t n, uint32_t R, double alpha,
                                 double eta) {
  unsigned long long all = 0;
  for (int32_t j = threadIdx.x & 31; j < n; j += 32) all += row[j];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) all += __shfl_xor_sync(0xFFFFFFFFu, all, o);
  const double q_sum = (1.0 - alpha) * (double)all / (double)R;
  const double r_i = alpha + (1.0 - alpha) * (double)row[n] / (double)R;
  double scale = (1.0 - alpha) / (double)R;
  if (r_i == 0.0 && q_sum > 0.0) scale *= (1.0 - eta) / q_sum;
  return scale;
}

__device__ __forceinline__ double warp_sum_d(double x) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xFFFFFFFFu, x, o);
  return x;
}

// Row-wise inner problem (warp per row, rows warp, warp + nwarps, ...) at the continuation
// value vsign * (v, v_bot).
__device__ void inner_rows(int32_t n, uint32_t R, double alpha, double eta,
                           const uint32_t *counts, double eps, double r_min, int support_only,
                           const double *v, double v_bot, double vsign, double *T, double *Qstar,
                           uint32_t *status, uint32_t warp, uint32_t nwarps) {
  const uint32_t lane = threadIdx.x & 31u;
  const size_t stride = (size_t)n + 1;
  const double vb = vsign * v_bot;
  for (uint32_t i = warp; i < (uint32_t)n; i += nwarps) {
    const uint32_t *row = counts + (size_t)i * stride;
    const double scale = row_scale_warp(row, n, R, alpha, eta);
    double *qs = Qstar ? Qstar + (size_t)i * n : nullptr;
    // every entry at its lower bound
    double base = 0.0, low = 0.0;
    for (int32_t j = lane; j < n; j += 32) {
      const double q = scale * (double)row[j];
      const double l = q > eps ? q - eps : 0.0;
      base += l * (vsign * v[j] - vb);
      low += l;
      if (qs) qs[j] = l;
    }
    base = warp_sum_d(base);
    low = warp_sum_d(low);
    __syncwarp();   // the lower bounds written by every lane, before lane 0 adds to them
    double budget = (1.0 - r_min) - low;
    if (budget < -1e-12) {
      if (lane == 0) atomicOr(status, kErrInput);   // U_i is empty
      budget = 0.0;
    }
    // the budget to the most negative coefficients first, each entry up to its upper bound
    double acc = 0.0, last_c = -INFINITY;
    int32_t last_j = -1;
    while (budget > 0.0) {
      double bc = 0.0;
      int32_t bj = 0x7FFFFFFF;
      double bcap = 0.0;
      for (int32_t j = lane; j < n; j += 32) {
        const double cf = vsign * v[j] - vb;
        if (!(cf < 0.0)) continue;
        if (cf < last_c || (cf == last_c && j <= last_j)) continue;   // already filled
        const double q = scale * (double)row[j];
        double cap;
        if (q > 0.0) cap = fmin(q + eps, 1.0) - (q > eps ? q - eps : 0.0);
        else cap = support_only ? 0.0 : fmin(eps, 1.0);
        if (!(cap > 0.0)) continue;
        if (bj == 0x7FFFFFFF || cf < bc || (cf == bc && j < bj)) { bc = cf; bj = j; bcap = cap; }
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const double oc = __shfl_xor_sync(0xFFFFFFFFu, bc, o);
        const int32_t oj = __shfl_xor_sync(0xFFFFFFFFu, bj, o);
        const double ocap = __shfl_xor_sync(0xFFFFFFFFu, bcap, o);
        if (oj != 0x7FFFFFFF && (bj == 0x7FFFFFFF || oc < bc || (oc == bc && oj < bj))) {
          bc = oc; bj = oj; bcap = ocap;
        }
      }
      if (bj == 0x7FFFFFFF) break;
      const double d = fmin(bcap, budget);
      acc += d * bc;
      budget -= d;
      if (qs && lane == 0) qs[bj] += d;
      last_c = bc;
      last_j = bj;
    }
    if (lane == 0) T[i] = vsign * (vb + base + acc);
  }
}

__global__ void robust_inner_kernel(int32_t n, uint32_t R, double alpha, double eta,
                                    const uint32_t *counts, double eps, double r_min,
                                    int support_only, const double *v, double v_bot, double vsign,
                                    double *T, double *Qstar, uint32_t *status) {
  inner_rows(n, R, alpha, eta, counts, eps, r_min, support_only, v, v_bot, vsign, T, Qstar,
             status, (blockIdx.x * blockDim.x + threadIdx.x) >> 5,
             (gridDim.x * blockDim.x) >> 5);
}

__global__ void build_a_kernel(int32_t n, const double *Qstar, double *A) {
  const size_t nn = (size_t)n * n;
  for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < nn;
       k += (size_t)gridDim.x * blockDim.x)
    A[k] = ((k / n) == (k % n) ? 1.0 : 0.0) - Qstar[k];
}

// One CTA of 256 threads: factor A (the blocked LU: the matrix is in device memory), V_new =
// A^-1 f (f = 1 when null), diff = max |V_new - V|, V <- V_new.
__device__ void eval_body(int32_t n, double *A, int32_t *piv, const double *f, double *V,
                          double *x, double *diff, uint32_t *status, LinScratch ls, double *red,
                          double *tiles) {
  if (!lu_factor_blocked(A, n, n, piv, ls, tiles)) {
    if (threadIdx.x == 0) { atomicOr(status, kErrSolve); *diff = 0.0; }
    return;
  }
  for (int32_t i = threadIdx.x; i < n; i += blockDim.x) x[i] = f ? f[i] : 1.0;
  __syncthreads();
  lu_solve(A, n, n, piv, x, ls);
  double m = 0.0, scale = 1.0;
  for (int32_t i = threadIdx.x; i < n; i += blockDim.x) {
    m = fmax(m, fabs(x[i] - V[i]));
    scale = fmax(scale, fabs(x[i]));
  }
  m = block_max(m, red);
  scale = block_max(scale, red);
  for (int32_t i = threadIdx.x; i < n; i += blockDim.x) V[i] = x[i];
  if (threadIdx.x == 0) *diff = m / scale;
}

__global__ void __launch_bounds__(256, 1)
eval_kernel(int32_t n, double *A, int32_t *piv, const double *f, double *V, double *x,
            double *diff, uint32_t *status) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ double sval[33];
  __shared__ int32_t sidx[32];
  __shared__ double sb[2];
  __shared__ int32_t sflag[1];
  __shared__ double red[33];
  LinScratch ls{sval, sidx, sb, sflag};
  eval_body(n, A, piv, f, V, x, diff, status, ls, red, reinterpret_cast<double *>(smem));
}

// The AFC of the scenario kernel from the factors of the last evaluation: A^T mu = s,
// out[0] = E_s[T] = sum mu, out[1] = b . f (f = 1 when null gives 1).
__global__ void __launch_bounds__(1024, 1)
star_kernel(int32_t n, const double *A, const int32_t *piv, const double *s, const double *f,
            double *mu, double *b, double *out) {
  __shared__ double sval[33];
  __shared__ int32_t sidx[32];
  __shared__ double sb[2];
  __shared__ int32_t sflag[1];
  __shared__ double red[33];
  LinScratch ls{sval, sidx, sb, sflag};
  for (int32_t i = threadIdx.x; i < n; i += blockDim.x) mu[i] = s ? s[i] : 1.0 / (double)n;
  __syncthreads();
  lu_solve_transposed(A, n, n, piv, mu, ls);
  double t = 0.0, tf = 0.0;
  for (int32_t i = threadIdx.x; i < n; i += blockDim.x) {
    t += mu[i];
    tf += mu[i] * (f ? f[i] : 1.0);
  }
  const double T = block_sum(t, red);
  const double TF = block_sum(tf, red);
  for (int32_t i = threadIdx.x; i < n; i += blockDim.x) b[i] = mu[i] / T;
  if (threadIdx.x == 0) { out[0] = T; out[1] = TF / T; }
}

// ---- batched robust problems (the envelopes): problem p's arrays at p times the stride ----

// inner problem of every active problem (blockIdx.y = problem)
__global__ void inner_batched_kernel(int32_t n, uint32_t R, double alpha, double eta,
                                     const uint32_t *counts, double eps, double r_min,
                                     int support_only, const EnvBatch B, uint32_t *status) {
  const uint32_t p = blockIdx.y;
  if (!B.active[p]) return;
  const size_t nn = (size_t)n * n;
  inner_rows(n, R, alpha, eta, counts, eps, r_min, support_only, B.V + p * B.vstride, 0.0,
             B.vsign[p], B.T + p * B.vstride, B.Qs + p * nn, status,
             (blockIdx.x * blockDim.x + threadIdx.x) >> 5, (gridDim.x * blockDim.x) >> 5);
}

// one CTA per active problem: A = I - Q*, its LU, V <- A^-1 f, diff
__global__ void __launch_bounds__(256, 1)
eval_batched_kernel(int32_t n, const EnvBatch B, uint32_t *status) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ double sval[33];
  __shared__ int32_t sidx[32];
  __shared__ double sb[2];
  __shared__ int32_t sflag[1];
  __shared__ double red[33];
  const uint32_t p = blockIdx.x;
  if (!B.active[p]) return;
  LinScratch ls{sval, sidx, sb, sflag};
  const size_t nn = (size_t)n * n;
  const double *Qs = B.Qs + p * nn;
  double *A = B.A + p * nn;
  for (size_t k = threadIdx.x; k < nn; k += blockDim.x)
    A[k] = ((k / n) == (k % n) ? 1.0 : 0.0) - Qs[k];
  __syncthreads();
  eval_body(n, A, B.piv + p * B.vstride, B.f + p * B.vstride, B.V + p * B.vstride,
            B.x + p * B.vstride, B.diff + p, status, ls, red, reinterpret_cast<double *>(smem));
}

// one CTA per active problem: the visits mu of its kernel (A^T mu = s from the last factors),
// ratio[p] = mu_v / sum mu = b_v for the problem's node v
__global__ void __launch_bounds__(1024, 1)
star_batched_kernel(int32_t n, const double *s, const EnvBatch B) {
  __shared__ double sval[33];
  __shared__ int32_t sidx[32];
  __shared__ double sb[2];
  __shared__ int32_t sflag[1];
  __shared__ double red[33];
  const uint32_t p = blockIdx.x;
  if (!B.active[p]) return;
  LinScratch ls{sval, sidx, sb, sflag};
  double *mu = B.x + p * B.vstride;
  for (int32_t i = threadIdx.x; i < n; i += blockDim.x) mu[i] = s ? s[i] : 1.0 / (double)n;
  __syncthreads();
  lu_solve_transposed(B.A + p * (size_t)n * n, n, n, B.piv + p * B.vstride, mu, ls);
  double t = 0.0;
  for (int32_t i = threadIdx.x; i < n; i += blockDim.x) t += mu[i];
  const double T = block_sum(t, red);
  if (threadIdx.x == 0) B.ratio[p] = mu[B.node[p]] / T;
}

// f_p = e_v - lambda_p for every active problem
__global__ void env_reward_kernel(int32_t n, uint32_t P, const EnvBatch B) {
  const size_t total = (size_t)P * n;
  for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < total;
       k += (size_t)gridDim.x * blockDim.x) {
    const uint32_t p = (uint32_t)(k / n);
    const int32_t j = (int32_t)(k % n);
    if (!B.active[p]) continue;
    B.f[p * B.vstride + j] = (j == B.node[p] ? 1.0 : 0.0) - B.lambda[p];
    B.V[p * B.vstride + j] = 0.0;
  }
}

}  // namespace

cudaError_t launch_env_reward(int32_t n, uint32_t P, const EnvBatch &B, cudaStream_t stream) {
  const size_t total = (size_t)P * n;
  const int grid = (int)std::max<size_t>(1, std::min<size_t>((total + 255) / 256, 4096));
  env_reward_kernel<<<grid, 256, 0, stream>>>(n, P, B);
  return cudaGetLastError();
}

cudaError_t launch_env_round(int32_t n, uint32_t R, double alpha, double eta,
                             const uint32_t *counts, double eps, double r_min, int support_only,
                             uint32_t P, const EnvBatch &B, uint32_t *status,
                             cudaStream_t stream) {
  const dim3 grid((unsigned)std::min<int64_t>(((int64_t)n + 7) / 8, 1024), P);
  inner_batched_kernel<<<grid, 256, 0, stream>>>(n, R, alpha, eta, counts, eps, r_min,
                                                 support_only, B, status);
  eval_batched_kernel<<<P, 256, sizeof(double) * lu_blocked_smem_doubles(), stream>>>(n, B,
                                                                                     status);
  return cudaGetLastError();
}

cudaError_t launch_env_ratio(int32_t n, const double *s, uint32_t P, const EnvBatch &B,
                             cudaStream_t stream) {
  star_batched_kernel<<<P, 1024, 0, stream>>>(n, s, B);
  return cudaGetLastError();
}

cudaError_t launch_robust_inner(int32_t n, uint32_t R, double alpha, double eta,
                                const uint32_t *counts, double eps, double r_min,
                                int support_only, const double *v, double v_bot, double vsign,
                                double *T, double *Qstar, uint32_t *status, cudaStream_t stream) {
  const int grid = (int)std::min<int64_t>(((int64_t)n + 7) / 8, 1024);
  robust_inner_kernel<<<grid, 256, 0, stream>>>(n, R, alpha, eta, counts, eps, r_min,
                                                support_only, v, v_bot, vsign, T, Qstar, status);
  return cudaGetLastError();
}

cudaError_t launch_robust_eval(int32_t n, const double *Qstar, double *A, int32_t *piv,
                               const double *f, double *V, double *x, double *diff,
                               uint32_t *status, cudaStream_t stream) {
  const int grid = (int)std::min<int64_t>(((int64_t)n * n + 255) / 256, 4096);
  build_a_kernel<<<grid, 256, 0, stream>>>(n, Qstar, A);
  eval_kernel<<<1, 256, sizeof(double) * lu_blocked_smem_doubles(), stream>>>(n, A, piv, f, V, x,
                                                                              diff, status);
  return cudaGetLastError();
}

cudaError_t launch_robust_star(int32_t n, const double *A, const int32_t *piv, const double *s,
                               const double *f, double *mu, double *b, double *out,
                               cudaStream_t stream) {
  star_kernel<<<1, 1024, 0, stream>>>(n, A, piv, s, f, mu, b, out);
  return cudaGetLastError();
}

namespace {

// Order of numpy's argmax: a larger value first (NaN above every number), then a smaller index.
__device__ __forceinline__ bool beats(double a, int32_t ia, double b, int32_t ib) {
  const bool na = isnan(a), nb = isnan(b);
  if (na != nb) return na;
  if (!na && a != b) return a > b;
  return ia < ib;
}

// arg[0] = argmax of d1, arg[1] = argmax of d2 (-1 for a NULL array or count 0).
__global__ void __launch_bounds__(256) argmax2_kernel(int32_t count, const double *d1,
                                                      const double *d2, int32_t *arg) {
  __shared__ double sv[256];
  __shared__ int32_t si[256];
  const int t = threadIdx.x;
  for (int w = 0; w < 2; ++w) {
    const double *d = w ? d2 : d1;
    if (!d) {
      if (t == 0) arg[w] = -1;
      continue;
    }
    double bv = 0.0;
    int32_t bi = -1;
    for (int32_t k = t; k < count; k += blockDim.x) {
      const double x = d[k];
      if (bi < 0 || beats(x, k, bv, bi)) {
        bv = x;
        bi = k;
      }
    }
    sv[t] = bv;
    si[t] = bi;
    __syncthreads();
    for (int s = 128; s > 0; s >>= 1) {
      if (t < s && si[t + s] >= 0 && (si[t] < 0 || beats(sv[t + s], si[t + s], sv[t], si[t]))) {
        sv[t] = sv[t + s];
        si[t] = si[t + s];
      }
      __syncthreads();
    }
    if (t == 0) arg[w] = si[0];
    __syncthreads();
  }
}

// Sampled envelopes: lo[v] / hi[v] = the smallest / largest of b0[v] and rows[k][v].
__global__ void envelope_kernel(int32_t n, int32_t count, const double *rows, const double *b0,
                                double *lo, double *hi) {
  for (int32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
    double a = b0[v], z = a;
    for (int32_t k = 0; k < count; ++k) {
      const double x = rows[(size_t)k * (size_t)n + v];
      a = fmin(a, x);
      z = fmax(z, x);
    }
    if (lo) lo[v] = a;
    if (hi) hi[v] = z;
  }
}

}  // namespace

cudaError_t launch_robust_summary(int32_t n, int32_t count, const double *rows, const double *b0,
                                  const double *d1, const double *d2, int32_t *arg, double *lo,
                                  double *hi, cudaStream_t stream) {
  if (arg) argmax2_kernel<<<1, 256, 0, stream>>>(count, d1, d2, arg);
  if (lo || hi) {
    const int grid = std::max(1, std::min((n + 255) / 256, 1024));
    envelope_kernel<<<grid, 256, 0, stream>>>(n, count, rows, b0, lo, hi);
  }
  return cudaGetLastError();
}

// W1 on a graph metric is an uncapacitated transshipment problem on the graph itself (each
// unit of mass moved across an edge costs 1).  It is solved exactly by successive shortest
// paths: node potentials keep the reduced arc costs non-negative, each round runs a
// multi-source Dijkstra from every node with excess mass and stops at the first node with a
// deficit, then pushes as much as the path allows (the source's excess, the sink's deficit,
// the flow on any arc the path cancels).  Costs are integers, so distances and potentials are
// exact; the masses are doubles and are settled to within a relative 1e-14.
double w1_graph_host(int32_t n, const int32_t *rp, const int32_t *col, const int32_t *eid,
                     const double *x, const double *y) {
  const int32_t arcs = rp[n];
  // partner arc of every arc (the other direction of the same edge)
  std::vector<int32_t> rev(std::max<int32_t>(arcs, 1), -1);
  int32_t maxe = 0;
  for (int32_t a = 0; a < arcs; ++a) maxe = std::max(maxe, eid[a] + 1);
  std::vector<int32_t> seen((size_t)maxe, -1);
  for (int32_t a = 0; a < arcs; ++a) {
    const int32_t e = eid[a];
    if (seen[e] < 0) { seen[e] = a; } else { rev[a] = seen[e]; rev[seen[e]] = a; }
  }
  std::vector<double> ex(n), flow(std::max<int32_t>(arcs, 1), 0.0);
  double scale = 0.0;
  for (int32_t v = 0; v < n; ++v) {
    ex[v] = x[v] - y[v];
    scale = std::max(scale, std::fabs(ex[v]));
  }
  const double tol = 1e-14 * std::max(scale, 1e-300);
  std::vector<int64_t> pot(n, 0), dist(n);
  std::vector<int32_t> par(n);        // arc into the node on the shortest path (-1: a source)
  std::vector<int32_t> pnode(n);      // the node that arc leaves
  std::vector<uint8_t> cancel(n), done(n);
  using Item = std::pair<int64_t, int32_t>;
  const int64_t kInf = std::numeric_limits<int64_t>::max() / 4;
  double cost = 0.0;
  for (int32_t guard = 0; guard < 8 * n + 8 * arcs + 64; ++guard) {
    std::priority_queue<Item, std::vector<Item>, std::greater<Item>> pq;
    std::fill(dist.begin(), dist.end(), kInf);
    std::fill(done.begin(), done.end(), 0);
    for (int32_t v = 0; v < n; ++v)
      if (ex[v] > tol) { dist[v] = 0; par[v] = -1; pq.push({0, v}); }
    if (pq.empty()) break;
    int32_t t = -1;
    while (!pq.empty()) {
      const auto [d, u] = pq.top();
      pq.pop();
      if (done[u] || d != dist[u]) continue;
      done[u] = 1;
      if (ex[u] < -tol) { t = u; break; }
      for (int32_t a = rp[u]; a < rp[u + 1]; ++a) {
        const int32_t v = col[a];
        // cancelling flow on v -> u costs -1, a new unit on u -> v costs +1
        const bool can = rev[a] >= 0 && flow[rev[a]] > tol;
        const int64_t nd = d + (can ? -1 : 1) + pot[u] - pot[v];
        if (nd < dist[v]) {
          dist[v] = nd; par[v] = a; pnode[v] = u; cancel[v] = can ? 1 : 0;
          pq.push({nd, v});
        }
      }
    }
    if (t < 0) break;   // mass left without a reachable deficit (disconnected support)
    const int64_t dt = dist[t];
    for (int32_t v = 0; v < n; ++v) pot[v] += done[v] ? dist[v] : dt;
    // bottleneck along the path t <- ... <- s
    double delta = -ex[t];
    int32_t v = t;
    while (par[v] >= 0) {
      if (cancel[v]) delta = std::min(delta, flow[rev[par[v]]]);
      v = pnode[v];
    }
    delta = std::min(delta, ex[v]);
    const int32_t s = v;
    for (v = t; par[v] >= 0; v = pnode[v]) {
      const int32_t a = par[v];
      if (cancel[v]) { flow[rev[a]] -= delta; cost -= delta; }
      else { flow[a] += delta; cost += delta; }
    }
    ex[s] -= delta;
    ex[t] += delta;
  }
  return cost;
}

}  // namespace afc
