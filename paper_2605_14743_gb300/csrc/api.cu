// api.cu -- query handles (afc_graph, afc_params, afc_result) over the end-to-end entry point,
// the sparse result layout, the solve's residual bound, the perturbation sweep of a result
// and the per-realization debug entry.  Host code; all device work runs in the library's
// kernels through the lower-level entry points.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "afc_internal.h"

struct afc_graph {
  int32_t n = 0;
  int64_t m = 0;
  std::vector<int32_t> eu, ev;
};

struct afc_result {
  int32_t n = 0;
  uint32_t R = 0;
  std::vector<int64_t> rp;
  std::vector<int32_t> col;
  std::vector<uint32_t> cnt, absorb;
  std::vector<double> b, mu;
  double expected_T = 0, b_f = 0, max_rowsum_N = 0, fp_err_bound = 0;
  int32_t c = 0;
  afc_mc_stats stats{};
  // chain parameters, for the perturbation sweep of the result
  double alpha = 0, eta = 0, tie_rel = 0;
  std::vector<double> s, f;
  void *stream = nullptr;
};

namespace afc {

// Result of one query from its dense counts [n][n+1] and solve outputs.
afc_result *build_result(int32_t n, uint32_t R, const uint32_t *dense, const double *b,
                         const double *mu, double expected_T, double b_f, double max_rowsum_N,
                         int32_t c, const afc_mc_stats &stats, double alpha, double eta,
                         const double *s, const double *f, double tie_rel, void *stream) {
  afc_result *r = new afc_result;
  r->n = n;
  r->R = R;
  const size_t w = (size_t)n + 1;
  r->rp.assign((size_t)n + 1, 0);
  r->absorb.resize((size_t)n);
  for (int32_t i = 0; i < n; ++i) {
    const uint32_t *row = dense + (size_t)i * w;
    for (int32_t j = 0; j < n; ++j)
      if (row[j]) {
        r->col.push_back(j);
        r->cnt.push_back(row[j]);
      }
    r->absorb[i] = row[n];
    r->rp[i + 1] = (int64_t)r->col.size();
  }
  r->b.assign(b, b + n);
  r->mu.assign(mu, mu + n);
  r->expected_T = expected_T;
  r->b_f = b_f;
  r->max_rowsum_N = max_rowsum_N;
  r->c = c;
  r->stats = stats;
  r->alpha = alpha;
  r->eta = eta;
  r->tie_rel = tie_rel;
  if (s) r->s.assign(s, s + n);
  if (f) r->f.assign(f, f + n);
  r->stream = stream;
  // residual of mu (I - Q) = s with the kernel assembled as the solve does (Q_ij =
  // (1 - alpha) counts_ij / R; a row that never absorbs gets the floor), in long double
  std::vector<long double> y((size_t)n, 0.0L);
  for (int32_t i = 0; i < n; ++i) {
    long double q_sum = 0.0L;
    for (int64_t k = r->rp[i]; k < r->rp[i + 1]; ++k)
      q_sum += (long double)(1.0 - alpha) * r->cnt[k] / (long double)R;
    const long double ri = (long double)alpha + (long double)(1.0 - alpha) * r->absorb[i] / R;
    const long double scale = (ri == 0.0L && q_sum > 0.0L) ? (1.0L - eta) / q_sum : 1.0L;
    for (int64_t k = r->rp[i]; k < r->rp[i + 1]; ++k)
      y[r->col[k]] += (long double)mu[i] * (1.0 - alpha) * r->cnt[k] / R * scale;
  }
  long double res = 0.0L, mass = 0.0L;
  for (int32_t j = 0; j < n; ++j) {
    const long double sj = s ? (long double)s[j] : 1.0L / n;
    res += fabsl(sj - ((long double)mu[j] - y[j]));
    mass += fabsl((long double)mu[j]);
  }
  r->fp_err_bound = mass > 0 ? (double)(2.0L * res * max_rowsum_N / mass) : 0.0;
  return r;
}

// Host query of a graph and parameters (arrays are borrowed from g and p).
afc_host_query host_query_of(const afc_graph *g, const afc_params *p, uint32_t n_perturb) {
  afc_host_query q{};
  q.n = g->n;
  q.m = g->m;
  q.eu = g->eu.data();
  q.ev = g->ev.data();
  q.p_survive = p->p_survive;
  q.p_survive_all = p->p_survive_all;
  q.w_lo = p->w_lo;
  q.w_hi = p->w_hi;
  q.w_lo_all = p->w_lo_all;
  q.w_hi_all = p->w_hi_all;
  q.seed = p->seed;
  q.graph_tag = p->graph_tag;
  q.realizations = p->realizations;
  q.k_min = p->k_min;
  q.alpha = p->alpha;
  q.absorb_floor = p->absorb_floor;
  q.s_init = p->s_init;
  q.reward = p->reward;
  q.candidates = p->candidates;
  q.n_candidates = p->n_candidates;
  q.top_k = p->top_k;
  q.tie_rel = p->tie_rel;
  q.precision = p->precision;
  q.recheck_margin = p->recheck_margin;
  q.n_perturb = n_perturb;
  return q;
}

}  // namespace afc

extern "C" {

int afc_graph_create(int32_t n, int64_t m, const int32_t *eu, const int32_t *ev, afc_graph **out) {
  if (!out) return afc::report_error(AFC_EINVAL, "null output");
  *out = nullptr;
  if (n < 1 || m < 0 || (m > 0 && (!eu || !ev))) return afc::report_error(AFC_EINVAL, "bad graph");
  // validation (ranges, self loops, duplicates) by the CSR builder
  std::vector<int32_t> rp((size_t)n + 1), col((size_t)std::max<int64_t>(2 * m, 1)), eid(col.size());
  const int st = afc_csr_from_edges(n, m, eu, ev, rp.data(), col.data(), eid.data());
  if (st) return st;
  afc_graph *g = new afc_graph;
  g->n = n;
  g->m = m;
  g->eu.assign(eu, eu + m);
  g->ev.assign(ev, ev + m);
  *out = g;
  return AFC_OK;
}

int afc_graph_create_csr(int32_t n, const int64_t *row_ptr, const int32_t *col, const int32_t *eid,
                         afc_graph **out) {
  if (!out) return afc::report_error(AFC_EINVAL, "null output");
  *out = nullptr;
  if (n < 1 || !row_ptr || row_ptr[0] != 0) return afc::report_error(AFC_EINVAL, "bad CSR");
  const int64_t arcs = row_ptr[n];
  if (arcs < 0 || (arcs & 1) || (arcs > 0 && (!col || !eid)))
    return afc::report_error(AFC_EINVAL, "CSR must hold an even number of arcs");
  const int64_t m = arcs / 2;
  std::vector<int32_t> eu((size_t)m, -1), ev((size_t)m, -1);
  std::vector<uint8_t> seen((size_t)m, 0);
  for (int32_t u = 0; u < n; ++u) {
    if (row_ptr[u + 1] < row_ptr[u]) return afc::report_error(AFC_EINVAL, "row_ptr not monotone");
    for (int64_t a = row_ptr[u]; a < row_ptr[u + 1]; ++a) {
      const int32_t v = col[a], e = eid[a];
      if (v < 0 || v >= n || e < 0 || e >= m) return afc::report_error(AFC_EINVAL, "arc out of range");
      if (seen[e] >= 2) return afc::report_error(AFC_EINVAL, "an edge id appears on more than two arcs");
      if (seen[e] == 0) {
        eu[e] = u;
        ev[e] = v;
      } else if (eu[e] != v || ev[e] != u) {
        return afc::report_error(AFC_EINVAL, "CSR is not symmetric");
      }
      seen[e]++;
    }
  }
  for (int64_t e = 0; e < m; ++e)
    if (seen[e] != 2) return afc::report_error(AFC_EINVAL, "an edge id is missing its reverse arc");
  return afc_graph_create(n, m, eu.data(), ev.data(), out);
}

int32_t afc_graph_nodes(const afc_graph *g) { return g ? g->n : 0; }
int64_t afc_graph_edges(const afc_graph *g) { return g ? g->m : 0; }
void afc_graph_destroy(afc_graph *g) { delete g; }

void afc_params_default(afc_params *p) {
  if (!p) return;
  std::memset(p, 0, sizeof(*p));
  p->p_survive_all = 1.0;
  p->w_lo_all = 1;
  p->w_hi_all = 1;
  p->k_min = 5;
  p->alpha = 0.15;
  p->absorb_floor = 1e-6;
  p->precision = AFC_FP64;
  p->recheck_margin = 1e-4;
  p->tie_rel = 1e-9;
}

int afc_run(const afc_graph *g, const afc_params *p, afc_result **out) {
  if (!g || !p || !out) return afc::report_error(AFC_EINVAL, "null argument");
  *out = nullptr;
  const int32_t n = g->n;
  afc_host_query q = afc::host_query_of(g, p, 0);
  std::vector<uint32_t> dense((size_t)n * ((size_t)n + 1));
  std::vector<double> b((size_t)n), mu((size_t)n);
  afc_host_result hr{};
  hr.counts = dense.data();
  hr.mu = mu.data();
  hr.b = b.data();
  const int st = afc_run_host(&q, &hr, p->cuda_stream);
  if (st) return st;
  *out = afc::build_result(n, p->realizations, dense.data(), b.data(), mu.data(), hr.expected_T,
                           hr.b_f, hr.max_rowsum_N, hr.c, hr.stats, p->alpha, p->absorb_floor,
                           p->s_init, p->reward, p->tie_rel, p->cuda_stream);
  return AFC_OK;
}

int afc_result_counts(const afc_result *r, const int64_t **row_ptr, const int32_t **col,
                      const uint32_t **cnt, const uint32_t **absorb) {
  if (!r) return afc::report_error(AFC_EINVAL, "null result");
  if (row_ptr) *row_ptr = r->rp.data();
  if (col) *col = r->col.data();
  if (cnt) *cnt = r->cnt.data();
  if (absorb) *absorb = r->absorb.data();
  return AFC_OK;
}

int afc_result_afc(const afc_result *r, const double **b, double *expected_T, double *b_reward) {
  if (!r) return afc::report_error(AFC_EINVAL, "null result");
  if (b) *b = r->b.data();
  if (expected_T) *expected_T = r->expected_T;
  if (b_reward) *b_reward = r->b_f;
  return AFC_OK;
}

int afc_result_diag(const afc_result *r, uint64_t *rechecked, double *fp_err_bound) {
  if (!r) return afc::report_error(AFC_EINVAL, "null result");
  if (rechecked) *rechecked = r->stats.rechecked;
  if (fp_err_bound) *fp_err_bound = r->fp_err_bound;
  return AFC_OK;
}

void afc_result_destroy(afc_result *r) { delete r; }

int afc_perturb(const afc_result *r, uint32_t n_perturb, double l1_radius, double r_min,
                uint64_t seed, uint32_t top_k, afc_perturb_stats *out) {
  if (!r || !out) return afc::report_error(AFC_EINVAL, "null argument");
  std::memset(out, 0, sizeof(*out));
  if (n_perturb == 0) return AFC_OK;
  if (top_k < 1 || top_k > 10) return afc::report_error(AFC_EINVAL, "top_k must be in [1, 10]");
  const int32_t n = r->n;
  cudaStream_t s = (cudaStream_t)r->stream;
  std::vector<uint32_t> dense((size_t)n * ((size_t)n + 1), 0);
  for (int32_t i = 0; i < n; ++i) {
    for (int64_t k = r->rp[i]; k < r->rp[i + 1]; ++k) dense[(size_t)i * (n + 1) + r->col[k]] = r->cnt[k];
    dense[(size_t)i * (n + 1) + n] = r->absorb[i];
  }
  std::vector<void *> allocs;
  auto dalloc = [&](size_t bytes) -> void * {
    void *p = nullptr;
    if (cudaMallocAsync(&p, std::max<size_t>(bytes, 16), s) != cudaSuccess) return nullptr;
    allocs.push_back(p);
    return p;
  };
  int rc = AFC_OK;
  do {
    uint32_t *counts = (uint32_t *)dalloc(4 * dense.size());
    int32_t *cidx = (int32_t *)dalloc(4 * (size_t)n);
    int32_t *clist = (int32_t *)dalloc(4 * (size_t)n);
    double *s_d = r->s.empty() ? nullptr : (double *)dalloc(8 * (size_t)n);
    double *f_d = r->f.empty() ? nullptr : (double *)dalloc(8 * (size_t)n);
    if (!counts || !cidx || !clist || (!r->s.empty() && !s_d) || (!r->f.empty() && !f_d)) {
      rc = afc::report_error(AFC_ENOMEM, "device allocation");
      break;
    }
    cudaMemcpyAsync(counts, dense.data(), 4 * dense.size(), cudaMemcpyHostToDevice, s);
    if (s_d) cudaMemcpyAsync(s_d, r->s.data(), 8 * (size_t)n, cudaMemcpyHostToDevice, s);
    if (f_d) cudaMemcpyAsync(f_d, r->f.data(), 8 * (size_t)n, cudaMemcpyHostToDevice, s);
    int32_t c = 0;
    rc = afc_observed_states(n, counts, cidx, clist, &c, s);
    if (rc) break;
    afc_chain ch{n, r->R, r->alpha, r->eta, s_d, f_d};
    const size_t wss = afc_solve_workspace(n, c);
    void *ws = dalloc(wss);
    double *mu = (double *)dalloc(8 * (size_t)n);
    double *b = (double *)dalloc(8 * (size_t)n);
    double *sc = (double *)dalloc(8 * 4);
    double *lu = (double *)dalloc(8 * (size_t)std::max(c, 1) * (size_t)std::max(c, 1));
    int32_t *piv = (int32_t *)dalloc(4 * (size_t)std::max(c, 1));
    uint64_t *pc = (uint64_t *)dalloc(8 * (3 + 100 + 16));
    double *pm = (double *)dalloc(8 * 3);
    if (!ws || !mu || !b || !sc || !lu || !piv || !pc || !pm) {
      rc = afc::report_error(AFC_ENOMEM, "device allocation");
      break;
    }
    rc = afc_absorbing_solve(&ch, counts, cidx, clist, c, mu, b, sc, lu, piv, ws, wss, s);
    if (rc) break;
    cudaMemsetAsync(pc, 0, 8 * (3 + 100 + 16), s);
    cudaMemsetAsync(pm, 0, 8 * 3, s);
    afc_perturb_params pp{0, n_perturb, l1_radius, r_min, seed, (int32_t)top_k, 10, 16, r->tie_rel};
    rc = afc_perturb_sweep(&ch, &pp, counts, cidx, clist, c, mu, b, lu, piv, pc, pc + 3, pc + 103,
                           pm, nullptr, ws, wss, s);
    if (rc) break;
    uint64_t h[3 + 100 + 16];
    double hm[3];
    cudaMemcpyAsync(h, pc, sizeof(h), cudaMemcpyDeviceToHost, s);
    cudaMemcpyAsync(hm, pm, sizeof(hm), cudaMemcpyDeviceToHost, s);
    const cudaError_t e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
      rc = afc::report_error(AFC_ECUDA, cudaGetErrorString(e));
      break;
    }
    out->top1_changes = h[0];
    out->topk_set_changes = h[1];
    out->topk_order_changes = h[2];
    std::memcpy(out->pair_flips, h + 3, sizeof(out->pair_flips));
    std::memcpy(out->shift_hist, h + 103, sizeof(out->shift_hist));
    out->max_shift_inf = hm[0];
    out->max_linear_err_inf = hm[1];
    out->max_rowsum_N = hm[2];
  } while (false);
  for (void *p : allocs) cudaFreeAsync(p, s);
  cudaStreamSynchronize(s);
  return rc;
}

int afc_debug_realization(const afc_graph *g, const afc_params *p, uint32_t r, int32_t src,
                          uint32_t *dist, uint64_t *sigma, double *B) {
  if (!g || !p) return afc::report_error(AFC_EINVAL, "null argument");
  const int32_t n = g->n;
  const int64_t m = g->m;
  if ((dist || sigma) && (src < 0 || src >= n)) return afc::report_error(AFC_EINVAL, "source out of range");
  cudaStream_t s = (cudaStream_t)p->cuda_stream;
  std::vector<int32_t> rp((size_t)n + 1), col((size_t)std::max<int64_t>(2 * m, 1)), eid(col.size());
  int rc = afc_csr_from_edges(n, m, g->eu.data(), g->ev.data(), rp.data(), col.data(), eid.data());
  if (rc) return rc;
  std::vector<uint64_t> th;
  if (p->p_survive) {
    th.resize((size_t)m);
    for (int64_t e = 0; e < m; ++e) th[e] = afc_survival_threshold(p->p_survive[e]);
  }
  std::vector<uint8_t> inw;
  if (p->candidates) {
    inw.assign((size_t)n, 0);
    for (int32_t k = 0; k < p->n_candidates; ++k) {
      if (p->candidates[k] < 0 || p->candidates[k] >= n) return afc::report_error(AFC_EINVAL, "candidate out of range");
      inw[p->candidates[k]] = 1;
    }
  }
  std::vector<void *> allocs;
  auto dalloc = [&](size_t bytes) -> void * {
    void *q = nullptr;
    if (cudaMallocAsync(&q, std::max<size_t>(bytes, 16), s) != cudaSuccess) return nullptr;
    allocs.push_back(q);
    return q;
  };
  do {
    int32_t *d_rp = (int32_t *)dalloc(4 * rp.size());
    int32_t *d_col = (int32_t *)dalloc(4 * col.size());
    int32_t *d_eid = (int32_t *)dalloc(4 * eid.size());
    uint64_t *d_th = th.empty() ? nullptr : (uint64_t *)dalloc(8 * th.size());
    uint32_t *d_wlo = p->w_lo ? (uint32_t *)dalloc(4 * (size_t)m) : nullptr;
    uint32_t *d_whi = p->w_hi ? (uint32_t *)dalloc(4 * (size_t)m) : nullptr;
    uint8_t *d_inw = inw.empty() ? nullptr : (uint8_t *)dalloc(inw.size());
    afc_mc_stats *d_stats = (afc_mc_stats *)dalloc(sizeof(afc_mc_stats));
    if (!d_rp || !d_col || !d_eid || !d_stats || (!th.empty() && !d_th) || (p->w_lo && !d_wlo) ||
        (p->w_hi && !d_whi) || (!inw.empty() && !d_inw)) {
      rc = afc::report_error(AFC_ENOMEM, "device allocation");
      break;
    }
    cudaMemcpyAsync(d_rp, rp.data(), 4 * rp.size(), cudaMemcpyHostToDevice, s);
    cudaMemcpyAsync(d_col, col.data(), 4 * col.size(), cudaMemcpyHostToDevice, s);
    cudaMemcpyAsync(d_eid, eid.data(), 4 * eid.size(), cudaMemcpyHostToDevice, s);
    if (d_th) cudaMemcpyAsync(d_th, th.data(), 8 * th.size(), cudaMemcpyHostToDevice, s);
    if (d_wlo) cudaMemcpyAsync(d_wlo, p->w_lo, 4 * (size_t)m, cudaMemcpyHostToDevice, s);
    if (d_whi) cudaMemcpyAsync(d_whi, p->w_hi, 4 * (size_t)m, cudaMemcpyHostToDevice, s);
    if (d_inw) cudaMemcpyAsync(d_inw, inw.data(), inw.size(), cudaMemcpyHostToDevice, s);
    cudaMemsetAsync(d_stats, 0, sizeof(afc_mc_stats), s);
    afc_mc_problem prob{};
    prob.n = n; prob.m = m; prob.row_ptr = d_rp; prob.col = d_col; prob.eid = d_eid;
    prob.seed = p->seed; prob.graph_tag = p->graph_tag;
    prob.thresh = d_th; prob.thresh_all = afc_survival_threshold(p->p_survive_all);
    prob.w_lo = d_wlo; prob.w_hi = d_whi; prob.w_lo_all = p->w_lo_all; prob.w_hi_all = p->w_hi_all;
    prob.k_min = p->k_min; prob.in_w = d_inw; prob.top_k = p->top_k; prob.tie_rel = p->tie_rel;
    prob.precision = p->precision; prob.recheck_margin = p->recheck_margin;
    if (dist || sigma) {
      uint32_t *d_dist = (uint32_t *)dalloc(4 * (size_t)n);
      uint64_t *d_sig = (uint64_t *)dalloc(8 * (size_t)n);
      int32_t *d_src = (int32_t *)dalloc(4);
      if (!d_dist || !d_sig || !d_src) { rc = afc::report_error(AFC_ENOMEM, "device allocation"); break; }
      cudaMemcpyAsync(d_src, &src, 4, cudaMemcpyHostToDevice, s);
      rc = afc_debug_sssp(&prob, r, d_src, 1, d_dist, d_sig, d_stats, s);
      if (rc) break;
      if (dist) cudaMemcpyAsync(dist, d_dist, 4 * (size_t)n, cudaMemcpyDeviceToHost, s);
      if (sigma) cudaMemcpyAsync(sigma, d_sig, 8 * (size_t)n, cudaMemcpyDeviceToHost, s);
    }
    if (B) {
      uint32_t *d_counts = (uint32_t *)dalloc(4 * (size_t)n * ((size_t)n + 1));
      double *d_bc = (double *)dalloc(8 * (size_t)n);
      const size_t wsb = afc_transition_counts_workspace(&prob);
      void *d_ws = dalloc(wsb);
      if (!d_counts || !d_bc || !d_ws || wsb == 0) { rc = afc::report_error(AFC_ENOMEM, "device allocation"); break; }
      cudaMemsetAsync(d_counts, 0, 4 * (size_t)n * ((size_t)n + 1), s);
      rc = afc_transition_counts(&prob, r, 1, d_counts, d_stats, d_bc, nullptr, d_ws, wsb, s);
      if (rc) break;
      cudaMemcpyAsync(B, d_bc, 8 * (size_t)n, cudaMemcpyDeviceToHost, s);
    }
    afc_mc_stats hs{};
    cudaMemcpyAsync(&hs, d_stats, sizeof(hs), cudaMemcpyDeviceToHost, s);
    const cudaError_t e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) { rc = afc::report_error(AFC_ECUDA, cudaGetErrorString(e)); break; }
    if (hs.device_error) { rc = afc::report_error(AFC_EDEVICE, "device consistency check failed"); break; }
  } while (false);
  for (void *q : allocs) cudaFreeAsync(q, s);
  cudaStreamSynchronize(s);
  return rc;
}

}  // extern "C"
