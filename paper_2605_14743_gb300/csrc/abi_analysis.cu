// abi_analysis.cu -- C-ABI entry points of the analyses built on an estimated chain:
// set-constrained summaries and 3-clique pools (Sec. 7, Sec. 9), the realization-level
// bootstrap (Sec. 8), the robust inner problem, robust value and graph Wasserstein-1 distance
// (Sec. 5, 8, 9), and the discrete length-law tables (Sec. 9).
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdint>
#include <thread>
#include <vector>

#include <cuda_runtime.h>

#include "abi_util.h"
#include "afc_internal.h"

using namespace afc;

namespace {

// Bootstrap workspace: [status | b_rep [B][n] | per-CTA slabs], at most 4 GB of slabs.
size_t boot_ws_head(int32_t n, uint32_t B) {
  return 256 + ((8ull * (size_t)B * (size_t)n + 255) & ~size_t(255));
}

int robust_checks(const afc_chain *chain, const uint32_t *counts, double eps, double r_min) {
  if (!chain || !counts) return fail(AFC_EINVAL, "null argument");
  if (const int st = chain_params_check(chain)) return st;
  if (!(eps >= 0.0) || !(r_min > 0.0 && r_min < 1.0)) return fail(AFC_EINVAL, "need eps >= 0 and 0 < r_min < 1");
  return AFC_OK;
}

size_t al256h(size_t x) { return (x + 255u) & ~size_t(255); }

// Rows of afc_w1_batch in flight: one 32-thread CTA each.  Its state and a copy of the graph
// in shared memory when both fit, else its state alone, else both in device memory (a slab
// per CTA); as many CTAs per SM as shared memory holds (at most 16), 8 per SM on the slab.
struct W1Plan {
  int mode = 0, grid = 1;
  size_t slot = 0, slab = 0;
};

W1Plan w1_plan(int32_t n, int64_t m, int32_t count) {
  const DevInfo d = dev_info();
  W1Plan p;
  p.slot = w1_slot_bytes(n, m);
  const size_t cap = (size_t)std::max(0, d.smem_optin - 1024);
  const size_t both = p.slot + w1_graph_bytes(n, m);
  p.mode = both <= cap ? 2 : p.slot <= cap ? 1 : 0;
  const size_t dyn = p.mode == 2 ? both : p.slot;
  const size_t per_sm = p.mode ? std::min<size_t>(16, (228u * 1024u) / (dyn + 1024u)) : 8;
  p.grid = (int)std::max<int64_t>(
      1, std::min<int64_t>(count, (int64_t)std::max(1, d.sms) * (int64_t)std::max<size_t>(1, per_sm)));
  p.slab = p.mode ? 0 : p.slot * (size_t)p.grid;
  return p;
}

}  // namespace

extern "C" {

int afc_weight_table_normal(int64_t m, const uint32_t *w0, uint32_t wmax, double rho_mu,
                            double rho_sigma, uint32_t *ptr, uint32_t *tab, size_t capacity,
                            size_t *used) {
  if (m < 0 || !ptr || (m > 0 && !w0) || wmax < 1 || wmax > 65535 || !(rho_sigma >= 0.0) ||
      !std::isfinite(rho_mu))
    return fail(AFC_EINVAL, "bad arguments");
  size_t need = 0;
  for (int64_t e = 0; e < m; ++e) {
    if (w0[e] < 1 || w0[e] > wmax) return fail(AFC_EINVAL, "w0[%lld] = %u outside [1, wmax]", (long long)e, w0[e]);
    need += wmax - w0[e];
  }
  if (need > 0xFFFFFFFFull)
    return fail(AFC_EUNSUPPORTED, "%zu thresholds do not fit 32-bit table offsets", need);
  if (need > capacity || (need > 0 && !tab))
    return fail(AFC_ENOMEM, "%zu thresholds needed, capacity %zu", need, capacity);
  size_t o = 0;
  for (int64_t e = 0; e < m; ++e) {
    ptr[e] = (uint32_t)o;
    const double span = (double)wmax - (double)w0[e];
    const double mu = (double)w0[e] + rho_mu * span, sigma = rho_sigma * span;
    for (uint32_t x = w0[e]; x < wmax; ++x) {
      // P(the rounded, clipped draw is at most x) = Phi((x + 1/2 - mu) / sigma)
      double F;
      if (sigma > 0.0) F = 0.5 * std::erfc(-(((double)x + 0.5 - mu) / sigma) / std::sqrt(2.0));
      else F = ((double)x + 0.5 >= mu) ? 1.0 : 0.0;
      const double t = std::floor(std::ldexp(F, 32));
      tab[o++] = t >= 4294967295.0 ? 0xFFFFFFFFu : (uint32_t)t;
    }
  }
  ptr[m] = (uint32_t)o;
  if (used) *used = o;
  return AFC_OK;
}

int afc_feasibility(const afc_chain *chain, const uint32_t *counts, const uint32_t *fallback_count,
                    double *xi, void *stream) {
  NvtxRange nvtx_range("afc.feasibility");
  if (!chain || !counts || !xi) return fail(AFC_EINVAL, "null argument");
  if (const int st = chain_params_check(chain)) return st;
  cudaError_t e = launch_feasibility(chain->n, chain->realizations, chain->alpha,
                                     chain->absorb_floor, counts, fallback_count, xi,
                                     (cudaStream_t)stream);
  return e == cudaSuccess ? AFC_OK : cuda_fail(e, "feasibility");
}

int afc_pool_summaries(int32_t n, const double *b, const uint8_t *in_w, const uint8_t *fallback_set,
                       double *b_pool, double *b_censored, double *mass, void *stream) {
  if (n < 1 || !b || !in_w || !mass) return fail(AFC_EINVAL, "bad arguments");
  cudaError_t e = launch_pool_summaries(n, b, in_w, fallback_set, b_pool, b_censored, mass,
                                        (cudaStream_t)stream);
  return e == cudaSuccess ? AFC_OK : cuda_fail(e, "pool_summaries");
}

int afc_clique_pool(int32_t n, int64_t m, const int32_t *eu, const int32_t *ev, int32_t S,
                    uint8_t *in_w, int32_t *fallback_node, int32_t *triangles, int32_t *kept) {
  return guarded("afc_clique_pool", [&]() -> int {
    if (n < 1 || m < 0 || S < 0 || !in_w || !fallback_node || (m > 0 && (!eu || !ev)))
      return fail(AFC_EINVAL, "bad arguments");
    std::vector<int32_t> rp((size_t)n + 1), col((size_t)std::max<int64_t>(2 * m, 1)),
        eid((size_t)std::max<int64_t>(2 * m, 1));
    int st = afc_csr_from_edges(n, m, eu, ev, rp.data(), col.data(), eid.data());
    if (st) return st;
    std::vector<int32_t> tri;
    clique_pool_host(n, rp.data(), col.data(), S, tri);
    const int32_t k = (int32_t)(tri.size() / 3);
    std::fill(in_w, in_w + n, (uint8_t)0);
    for (int32_t t = 0; t < 3 * k; ++t) in_w[tri[t]] = 1;
    *fallback_node = k > 0 ? tri[0] : -1;
    if (triangles) std::copy(tri.begin(), tri.begin() + 3 * k, triangles);
    if (kept) *kept = k;
    return AFC_OK;
  });
}

size_t afc_bootstrap_workspace(int32_t n, int32_t c, uint32_t R, uint32_t B) {
  if (n < 1 || c < 0 || c > n || R == 0 || B == 0) return 0;
  const DevInfo d = dev_info();
  const size_t slab = bootstrap_slab_bytes(n, c, R);
  size_t grid = std::min<size_t>((size_t)B, (size_t)std::max(1, d.sms) * 2);
  grid = std::max<size_t>(1, std::min<size_t>(grid, (4ull << 30) / std::max<size_t>(slab, 1)));
  return boot_ws_head(n, B) + grid * slab;
}

int afc_bootstrap(const afc_chain *chain, const int32_t *next_states, const int32_t *c_index,
                  const int32_t *c_list, int32_t c, uint32_t B, uint64_t seed, double level,
                  double *b_rep, double *T_rep, double *b_lo, double *b_hi, void *workspace,
                  size_t workspace_bytes, void *stream) {
  NvtxRange nvtx_range("afc.bootstrap");
  if (!chain || !next_states || !c_index || !c_list) return fail(AFC_EINVAL, "null argument");
  if (const int st = chain_params_check(chain)) return st;
  if (c < 0 || c > chain->n) return fail(AFC_EINVAL, "bad n or c");
  if (B == 0) return fail(AFC_EINVAL, "B must be > 0");
  if (!(level > 0.0 && level < 1.0)) return fail(AFC_EINVAL, "level outside (0, 1)");
  const int32_t n = chain->n;
  const uint32_t R = chain->realizations;
  const size_t head = boot_ws_head(n, B);
  const size_t slab = bootstrap_slab_bytes(n, c, R);
  if (!workspace || workspace_bytes < head + slab)
    return fail(AFC_ENOMEM, "workspace of %zu bytes given, at least %zu needed", workspace_bytes,
                head + slab);
  cudaStream_t s = (cudaStream_t)stream;
  unsigned char *ws = static_cast<unsigned char *>(workspace);
  uint32_t *status = reinterpret_cast<uint32_t *>(ws);
  double *rep = b_rep ? b_rep : reinterpret_cast<double *>(ws + 256);
  AFC_CUDA(cudaMemsetAsync(status, 0, sizeof(uint32_t), s));
  ChainDev C{};
  C.n = n;
  C.R = R;
  C.alpha = chain->alpha;
  C.eta = chain->absorb_floor;
  C.s = chain->s_init;
  C.f = chain->reward;
  C.c_index = c_index;
  C.c_list = c_list;
  C.c = c;
  const DevInfo d = dev_info();
  cudaError_t e = launch_bootstrap(C, next_states, R, B, seed, level, rep, T_rep, b_lo, b_hi,
                                   ws + head, workspace_bytes - head, status, d.sms, s);
  if (e != cudaSuccess) return cuda_fail(e, "bootstrap launch");
  uint32_t st_host = 0;
  AFC_CUDA(cudaMemcpyAsync(&st_host, status, sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
  AFC_CUDA(cudaStreamSynchronize(s));
  if (st_host & kErrInput)
    return fail(AFC_EINVAL, "a next state is neither absorption nor an observed state of c_index");
  if (st_host & kErrSolve) return fail(AFC_ESINGULAR, "zero pivot in a bootstrap replicate");
  return AFC_OK;
}

int afc_robust_inner(const afc_chain *chain, const uint32_t *counts, double eps, double r_min,
                     int32_t support_only, const double *v, double v_bot, double *T, double *Qstar,
                     void *workspace, size_t workspace_bytes, void *stream) {
  NvtxRange nvtx_range("afc.robust_inner");
  int st = robust_checks(chain, counts, eps, r_min);
  if (st) return st;
  if (!v || !T) return fail(AFC_EINVAL, "null argument");
  if (!workspace || workspace_bytes < 256) return fail(AFC_ENOMEM, "need 256 bytes of workspace");
  cudaStream_t s = (cudaStream_t)stream;
  uint32_t *status = static_cast<uint32_t *>(workspace);
  AFC_CUDA(cudaMemsetAsync(status, 0, sizeof(uint32_t), s));
  cudaError_t e = launch_robust_inner(chain->n, chain->realizations, chain->alpha,
                                      chain->absorb_floor, counts, eps, r_min, support_only ? 1 : 0,
                                      v, v_bot, 1.0, T, Qstar, status, s);
  if (e != cudaSuccess) return cuda_fail(e, "robust inner launch");
  uint32_t h = 0;
  AFC_CUDA(cudaMemcpyAsync(&h, status, sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
  AFC_CUDA(cudaStreamSynchronize(s));
  if (h) return fail(AFC_EINVAL, "empty uncertainty set: a row's lower bounds exceed 1 - r_min");
  return AFC_OK;
}

size_t afc_robust_value_workspace(int32_t n) {
  if (n < 1 || n > 4096) return 0;
  const size_t nn = (size_t)n * (size_t)n;
  return 256 + 2 * al256h(8 * nn) + al256h(4 * (size_t)n) + 3 * al256h(8 * (size_t)n);
}

int afc_robust_value(const afc_chain *chain, const uint32_t *counts, double eps, double r_min,
                     int32_t support_only, int32_t sense, double *V, double *Qstar, double *b_star,
                     double *scalars, int32_t *iterations, void *workspace, size_t workspace_bytes,
                     void *stream) {
  NvtxRange nvtx_range("afc.robust_value");
  int st = robust_checks(chain, counts, eps, r_min);
  if (st) return st;
  if (!V || !b_star || !scalars) return fail(AFC_EINVAL, "null argument");
  if (sense != -1 && sense != 1) return fail(AFC_EINVAL, "sense must be -1 (min) or +1 (max)");
  const int32_t n = chain->n;
  if (n > 4096) return fail(AFC_EUNSUPPORTED, "the robust value takes n <= 4096 (dense LU)");
  const size_t need = afc_robust_value_workspace(n);
  if (!workspace || workspace_bytes < need)
    return fail(AFC_ENOMEM, "workspace of %zu bytes given, %zu needed", workspace_bytes, need);
  cudaStream_t s = (cudaStream_t)stream;
  const size_t nn = (size_t)n * (size_t)n;
  unsigned char *ws = static_cast<unsigned char *>(workspace);
  uint32_t *status = reinterpret_cast<uint32_t *>(ws);
  double *diff = reinterpret_cast<double *>(ws + 8);
  size_t o = 256;
  double *Qs = reinterpret_cast<double *>(ws + o); o += al256h(8 * nn);
  double *A = reinterpret_cast<double *>(ws + o);  o += al256h(8 * nn);
  int32_t *piv = reinterpret_cast<int32_t *>(ws + o); o += al256h(4 * (size_t)n);
  double *x = reinterpret_cast<double *>(ws + o);  o += al256h(8 * (size_t)n);
  double *T = reinterpret_cast<double *>(ws + o);  o += al256h(8 * (size_t)n);
  double *mu = reinterpret_cast<double *>(ws + o);
  AFC_CUDA(cudaMemsetAsync(status, 0, sizeof(uint32_t), s));
  AFC_CUDA(cudaMemsetAsync(V, 0, sizeof(double) * (size_t)n, s));
  // policy iteration: the inner problem's minimiser (or maximiser) at V, then V of that kernel
  int it = 0;
  for (; it < 100; ++it) {
    cudaError_t e = launch_robust_inner(n, chain->realizations, chain->alpha, chain->absorb_floor,
                                        counts, eps, r_min, support_only ? 1 : 0, V, 0.0,
                                        sense < 0 ? 1.0 : -1.0, T, Qs, status, s);
    if (e == cudaSuccess) e = launch_robust_eval(n, Qs, A, piv, chain->reward, V, x, diff, status, s);
    if (e != cudaSuccess) return cuda_fail(e, "robust value launch");
    double h_diff = 0.0;
    uint32_t h_st = 0;
    AFC_CUDA(cudaMemcpyAsync(&h_diff, diff, sizeof(double), cudaMemcpyDeviceToHost, s));
    AFC_CUDA(cudaMemcpyAsync(&h_st, status, sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
    AFC_CUDA(cudaStreamSynchronize(s));
    if (h_st & kErrInput) return fail(AFC_EINVAL, "empty uncertainty set: a row's lower bounds exceed 1 - r_min");
    if (h_st & kErrSolve) return fail(AFC_ESINGULAR, "zero pivot in I - Q*");
    if (it > 0 && h_diff <= 1e-13) { ++it; break; }
  }
  if (Qstar) AFC_CUDA(cudaMemcpyAsync(Qstar, Qs, sizeof(double) * nn, cudaMemcpyDeviceToDevice, s));
  cudaError_t e = launch_robust_star(n, A, piv, chain->s_init, chain->reward, mu, b_star, scalars, s);
  if (e != cudaSuccess) return cuda_fail(e, "robust star launch");
  AFC_CUDA(cudaStreamSynchronize(s));
  if (iterations) *iterations = it;
  return AFC_OK;
}

// Envelope workspace: [status | per-problem scalars | per-problem slabs (Q*, A, V, x, T, f, piv)].
static size_t env_head_bytes(size_t P) { return 256 + al256h(P * 48); }
static size_t env_problem_bytes(size_t n) {
  return 2 * al256h(8 * n * n) + 4 * al256h(8 * n) + al256h(4 * n);
}

size_t afc_robust_envelope_workspace(int32_t n, int32_t k) {
  if (n < 1 || n > 4096 || k < 1) return 0;
  const size_t P = 2 * (size_t)k;
  return env_head_bytes(P) + P * env_problem_bytes((size_t)n);
}

int afc_robust_envelope(const afc_chain *chain, const uint32_t *counts, double eps, double r_min,
                        int32_t support_only, int32_t k, const int32_t *nodes, double *b_lo,
                        double *b_hi, int32_t *iterations, void *workspace,
                        size_t workspace_bytes, void *stream) {
  NvtxRange nvtx_range("afc.robust_envelope");
  int st = robust_checks(chain, counts, eps, r_min);
  if (st) return st;
  const int32_t n = chain->n;
  if (k < 1 || !nodes || !b_lo || !b_hi) return fail(AFC_EINVAL, "bad arguments");
  for (int32_t q = 0; q < k; ++q)
    if (nodes[q] < 0 || nodes[q] >= n) return fail(AFC_EINVAL, "node %d out of range", nodes[q]);
  if (n > 4096) return fail(AFC_EUNSUPPORTED, "the envelopes take n <= 4096 (dense LU)");
  const size_t need = afc_robust_envelope_workspace(n, k);
  if (!workspace || workspace_bytes < need)
    return fail(AFC_ENOMEM, "workspace of %zu bytes given, %zu needed", workspace_bytes, need);
  cudaStream_t s = (cudaStream_t)stream;
  const uint32_t P = 2u * (uint32_t)k;
  unsigned char *ws = static_cast<unsigned char *>(workspace);
  uint32_t *status = reinterpret_cast<uint32_t *>(ws);
  unsigned char *h = ws + 256;
  uint32_t *d_active = reinterpret_cast<uint32_t *>(h);
  double *d_vsign = reinterpret_cast<double *>(h + 8 * (size_t)P);
  double *d_lambda = d_vsign + P;
  int32_t *d_node = reinterpret_cast<int32_t *>(d_lambda + P);
  double *d_diff = reinterpret_cast<double *>(d_node + 2 * (size_t)P);
  double *d_ratio = d_diff + P;
  const size_t nn = (size_t)n * n, vs = (al256h(8 * (size_t)n)) / 8;
  unsigned char *slab = ws + env_head_bytes(P);
  EnvBatch B{};
  B.Qs = reinterpret_cast<double *>(slab);
  B.A = B.Qs + P * (al256h(8 * nn) / 8);
  double *vec = B.A + P * (al256h(8 * nn) / 8);
  B.vstride = vs;
  B.V = vec;
  B.x = B.V + P * vs;
  B.T = B.x + P * vs;
  B.f = B.T + P * vs;
  B.piv = reinterpret_cast<int32_t *>(B.f + P * vs);
  B.active = d_active;
  B.vsign = d_vsign;
  B.lambda = d_lambda;
  B.node = d_node;
  B.diff = d_diff;
  B.ratio = d_ratio;
  // problem 2q: the supremum of b_v (the adversary maximises: vsign -1), 2q + 1: the infimum
  std::vector<uint32_t> dk(P, 1u), pi(P, 0u);
  std::vector<double> vsign(P), lambda(P, 0.0), diff(P), ratio(P), result(P, 0.0);
  std::vector<int32_t> node(2 * (size_t)P, 0), its(P, 0);
  for (uint32_t p = 0; p < P; ++p) {
    node[p] = nodes[p / 2];
    vsign[p] = (p % 2 == 0) ? -1.0 : 1.0;
  }
  AFC_CUDA(cudaMemsetAsync(status, 0, sizeof(uint32_t), s));
  AFC_CUDA(cudaMemcpyAsync(d_vsign, vsign.data(), 8 * (size_t)P, cudaMemcpyHostToDevice, s));
  AFC_CUDA(cudaMemcpyAsync(d_node, node.data(), 4 * (size_t)P, cudaMemcpyHostToDevice, s));
  auto check_status = [&]() -> int {
    uint32_t hs = 0;
    AFC_CUDA(cudaMemcpyAsync(&hs, status, sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
    AFC_CUDA(cudaStreamSynchronize(s));
    if (hs & kErrInput) return fail(AFC_EINVAL, "empty uncertainty set: a row's lower bounds exceed 1 - r_min");
    if (hs & kErrSolve) return fail(AFC_ESINGULAR, "zero pivot in I - Q*");
    return AFC_OK;
  };
  // Dinkelbach: lambda <- b_v of the kernel optimising s N (e_v - lambda 1) over the set, until
  // it stops moving (that optimum is then 0 and lambda the envelope)
  for (int outer = 0; outer < 60; ++outer) {
    if (std::find(dk.begin(), dk.end(), 1u) == dk.end()) break;
    AFC_CUDA(cudaMemcpyAsync(d_lambda, lambda.data(), 8 * (size_t)P, cudaMemcpyHostToDevice, s));
    AFC_CUDA(cudaMemcpyAsync(d_active, dk.data(), 4 * (size_t)P, cudaMemcpyHostToDevice, s));
    cudaError_t e = launch_env_reward(n, P, B, s);
    if (e != cudaSuccess) return cuda_fail(e, "envelope reward");
    // policy iteration of every problem still moving, in lockstep
    pi = dk;
    for (int it = 0; it < 100; ++it) {
      AFC_CUDA(cudaMemcpyAsync(d_active, pi.data(), 4 * (size_t)P, cudaMemcpyHostToDevice, s));
      e = launch_env_round(n, chain->realizations, chain->alpha, chain->absorb_floor, counts, eps,
                           r_min, support_only ? 1 : 0, P, B, status, s);
      if (e != cudaSuccess) return cuda_fail(e, "envelope round");
      AFC_CUDA(cudaMemcpyAsync(diff.data(), d_diff, 8 * (size_t)P, cudaMemcpyDeviceToHost, s));
      if (int rc = check_status()) return rc;
      bool any = false;
      for (uint32_t p = 0; p < P; ++p) {
        if (pi[p] && it > 0 && diff[p] <= 1e-13) pi[p] = 0;
        any = any || pi[p];
      }
      if (!any) break;
    }
    AFC_CUDA(cudaMemcpyAsync(d_active, dk.data(), 4 * (size_t)P, cudaMemcpyHostToDevice, s));
    e = launch_env_ratio(n, chain->s_init, P, B, s);
    if (e != cudaSuccess) return cuda_fail(e, "envelope ratio");
    AFC_CUDA(cudaMemcpyAsync(ratio.data(), d_ratio, 8 * (size_t)P, cudaMemcpyDeviceToHost, s));
    if (int rc = check_status()) return rc;
    for (uint32_t p = 0; p < P; ++p) {
      if (!dk[p]) continue;
      ++its[p];
      result[p] = ratio[p];
      if (std::fabs(ratio[p] - lambda[p]) <= 1e-13 * std::fabs(ratio[p])) dk[p] = 0;
      else lambda[p] = ratio[p];
    }
  }
  if (std::find(dk.begin(), dk.end(), 1u) != dk.end())
    return fail(AFC_EDEVICE, "envelope: the Dinkelbach iteration did not settle in 60 steps");
  for (int32_t q = 0; q < k; ++q) {
    b_hi[q] = result[2 * q];
    b_lo[q] = result[2 * q + 1];
    if (iterations) {
      iterations[2 * q] = its[2 * q];
      iterations[2 * q + 1] = its[2 * q + 1];
    }
  }
  return AFC_OK;
}

int afc_w1_graph(int32_t n, int64_t m, const int32_t *eu, const int32_t *ev, const double *x,
                 const double *y, int32_t count, double *out) {
  NvtxRange nvtx_range("afc.w1_graph");
  return guarded("afc_w1_graph", [&]() -> int {
    if (n < 1 || m < 0 || count < 0 || !x || !y || !out || (m > 0 && (!eu || !ev)))
      return fail(AFC_EINVAL, "bad arguments");
    std::vector<int32_t> rp((size_t)n + 1), col((size_t)std::max<int64_t>(2 * m, 1)),
        eid((size_t)std::max<int64_t>(2 * m, 1));
    int st = afc_csr_from_edges(n, m, eu, ev, rp.data(), col.data(), eid.data());
    if (st) return st;
    // rows are independent: spread them over the host's cores (a row whose solve fails to
    // allocate flags the call; threads that could not start leave their rows to this one)
    const int32_t nth = std::max(1, std::min<int32_t>(count, (int32_t)std::thread::hardware_concurrency()));
    std::atomic<int> failed{0};
    auto rows = [&](int32_t t0, int32_t step) {
      try {
        for (int32_t k = t0; k < count; k += step)
          out[k] = w1_graph_host(n, rp.data(), col.data(), eid.data(), x + (size_t)k * n, y);
      } catch (...) {
        failed = 1;
      }
    };
    std::vector<std::thread> pool;
    pool.reserve((size_t)nth);
    int32_t started = 0;
    try {
      for (; started < nth; ++started) pool.emplace_back(rows, started, nth);
    } catch (...) {
    }
    for (int32_t t = started; t < nth; ++t) rows(t, nth);
    for (auto &th : pool) th.join();
    if (failed) return fail(AFC_ENOMEM, "afc_w1_graph: host allocation failed");
    return AFC_OK;
  });
}

size_t afc_w1_batch_workspace(int32_t n, int64_t m, int32_t count) {
  if (n < 1 || m < 0 || count < 0) return 0;
  return 256 + w1_plan(n, m, count).slab;
}

int afc_w1_batch(int32_t n, int64_t m, const int32_t *row_ptr, const int32_t *col,
                 const int32_t *eid, const double *x, const double *y, int32_t count, double *out,
                 void *workspace, size_t workspace_bytes, void *stream) {
  NvtxRange nvtx_range("afc.w1_batch");
  if (n < 1 || m < 0 || count < 0 || !row_ptr || !y || (count > 0 && (!x || !out)) ||
      (m > 0 && (!col || !eid)))
    return fail(AFC_EINVAL, "bad arguments");
  if (m > 0x7FFFFFFFll / 2) return fail(AFC_EUNSUPPORTED, "more than 2^30 edges");
  const W1Plan p = w1_plan(n, m, count);
  if (!workspace || workspace_bytes < 256 + p.slab)
    return fail(AFC_ENOMEM, "workspace of %zu bytes given, %zu needed", workspace_bytes,
                256 + p.slab);
  if (count == 0) return AFC_OK;
  cudaStream_t s = (cudaStream_t)stream;
  unsigned char *ws = static_cast<unsigned char *>(workspace);
  uint32_t *status = reinterpret_cast<uint32_t *>(ws);
  AFC_CUDA(cudaMemsetAsync(status, 0, sizeof(uint32_t), s));
  cudaError_t e = launch_w1(n, m, row_ptr, col, eid, x, y, count, out, ws + 256, p.mode,
                            p.grid, status, s);
  if (e != cudaSuccess) return cuda_fail(e, "w1 launch");
  uint32_t h = 0;
  AFC_CUDA(cudaMemcpyAsync(&h, status, sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
  AFC_CUDA(cudaStreamSynchronize(s));
  if (h & 1u)
    return fail(AFC_EINVAL, "mass that reaches no deficit: x_k and y differ in total on some "
                            "connected component");
  if (h & 2u) return fail(AFC_EDEVICE, "w1: an iteration bound was hit");
  if (h & 4u) return fail(AFC_EDEVICE, "w1: a flow invariant failed");
  return AFC_OK;
}

int afc_rank_order(int32_t n, const double *b, double tie_rel, int32_t k, int32_t *rank,
                   int32_t *topk, void *stream) {
  if (n < 1 || !b || !rank || k < 0 || k > n || (k > 0 && !topk) || !(tie_rel >= 0.0))
    return fail(AFC_EINVAL, "bad arguments");
  cudaError_t e = launch_rank(n, b, tie_rel, k, rank, topk, (cudaStream_t)stream);
  return e == cudaSuccess ? AFC_OK : cuda_fail(e, "rank launch");
}

int afc_robust_summary(int32_t n, int32_t count, const double *b_rows, const double *b0,
                       const double *d1, const double *d2, int32_t *arg, double *b_low,
                       double *b_high, void *stream) {
  if (n < 1 || count < 0 || !b0 || (count > 0 && !b_rows && (b_low || b_high)) ||
      (arg && count > 0 && !d1 && !d2))
    return fail(AFC_EINVAL, "bad arguments");
  cudaError_t e = launch_robust_summary(n, count, b_rows, b0, d1, d2, arg, b_low, b_high,
                                        (cudaStream_t)stream);
  return e == cudaSuccess ? AFC_OK : cuda_fail(e, "robust summary launch");
}

}  // extern "C"
