/*
 * afc_oracle.c -- plain, single-threaded CPU oracle for the absorbing-frequency-centrality
 * (AFC) path of "Betweenness-Central Nodes Under Uncertainty: An Absorbing Markov Chain
 * Approach" (Bao, Kontou, Vogiatzis).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the benchmark's CPU
 * baseline leg load this file's library.  It shares no code, header, table or helper with
 * the CUDA path.  Every routine is the plain definition (or the paper's algorithm in the
 * paper's order); nothing is blocked, fused or reordered for speed.  Floating point is FP64.
 *
 * Parity status of each routine (what pins it in the not-gpu tests):
 *   orc_philox4x32_10 / orc_philox4x64_10 : 4x64 checked against numpy.random.Philox;
 *                                           4x32 (multipliers included) checked block by
 *                                           block against PyTorch's header-only Philox
 *                                           engine; key schedule of both widths pinned to the
 *                                           golden-ratio and sqrt(3) Weyl increments;
 *                                           uniformity tests.
 *   orc_realize                           : survival frequency / weight histogram tests.
 *   orc_components                        : brute-force BFS comparison, invariants.
 *   orc_sssp / orc_brandes                : closed-form betweenness (path, star, cycle,
 *                                           complete, clique-bridge), brute-force shortest
 *                                           path enumeration, networkx cross-check.
 *   orc_select / orc_count_transitions    : crossroads example (Sec. 2.1) by exhaustive
 *                                           enumeration of failure patterns; row sums.
 *   orc_gauss_solve / orc_solve_*         : crossroads AFC and E[T]; Appendix B; canonical
 *                                           chain closed form (Prop. in App. A); constant-
 *                                           hazard discounted occupancy (Sec. 5.3).
 *   orc_certificates                      : Appendix B printed thresholds.
 *   orc_perturb_sweep                     : invariants; every perturbed solve against
 *                                           numpy's dense solve and the counters recounted
 *                                           from those solves; pair reversals never on a
 *                                           pair the Sec. 5.5 certificate protects (no
 *                                           printed values exist for these statistics).
 *   orc_topk_order / orc_count_rewards    : closed-form orderings (complete graph, star,
 *                                           path), rank-1 equals orc_select, the Top-1
 *                                           reward identity b_{1,f} = b.f - s.f / E[T],
 *                                           exhaustive failure patterns (Hoeffding bound).
 *   orc_select_ex (filter, fallback)      : exhaustive failure enumeration with networkx
 *                                           betweenness; identities between unconstrained,
 *                                           filtered and fallback counts (Sec. 7).
 *   orc_count_transitions, random ties    : exhaustive enumeration of the induced kernel on
 *                                           the crossroads example; label invariance.
 *   orc_weight_table_normal / _realize_law: scipy's normal distribution; realized histograms.
 *   orc_count_per_row (Alg. 2, r-hop)     : exhaustive enumeration; path and star closed
 *                                           forms; a radius covering the graph changes nothing.
 *   orc_bootstrap_weights                 : multinomial moments; coverage of the exact
 *                                           crossroads AFC.
 *   orc_perturb_row_mult                  : row validity, leak floor, KL of the sweep.
 * The robust inner problem, robust value and graph Wasserstein distance live in the Python
 * part of the oracle and are pinned in its tests (closed forms, brute-force value iteration,
 * an independent transport LP).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_OK 0
#define ORC_EINVAL 1
#define ORC_ENOMEM 2
#define ORC_EOVERFLOW 3
#define ORC_ESINGULAR 4

#define ORC_INF UINT64_MAX

/* ------------------------------------------------------------------------------------ */
/* Philox counter-based generator (Salmon, Moraes, Dror, Shaw, "Parallel random numbers:  */
/* as easy as 1, 2, 3", SC'11): 10 rounds of a multiply-hi/lo Feistel-like bijection on    */
/* a 4-word counter, with a Weyl-sequence key schedule.                                   */
/* ------------------------------------------------------------------------------------ */

/* `rounds` rounds of the bijection; the generator proper is rounds = 10.  Fewer rounds serve   */
/* the tests that pin the key schedule (10 rounds = 1 round, then 9 with the bumped key).      */
void orc_philox4x32_rounds(const uint32_t ctr[4], const uint32_t key[2], int32_t rounds,
                           uint32_t out[4]) {
  uint32_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
  uint32_t k0 = key[0], k1 = key[1];
  for (int round = 0; round < rounds; ++round) {
    if (round > 0) {
      k0 += 0x9E3779B9u;
      k1 += 0xBB67AE85u;
    }
    uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)x0;
    uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)x2;
    uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    uint32_t y0 = hi1 ^ x1 ^ k0;
    uint32_t y1 = lo1;
    uint32_t y2 = hi0 ^ x3 ^ k1;
    uint32_t y3 = lo0;
    x0 = y0; x1 = y1; x2 = y2; x3 = y3;
  }
  out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
  orc_philox4x32_rounds(ctr, key, 10, out);
}

void orc_philox4x64_rounds(const uint64_t ctr[4], const uint64_t key[2], int32_t rounds,
                           uint64_t out[4]) {
  uint64_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
  uint64_t k0 = key[0], k1 = key[1];
  for (int round = 0; round < rounds; ++round) {
    if (round > 0) {
      k0 += 0x9E3779B97F4A7C15ull;
      k1 += 0xBB67AE8584CAA73Bull;
    }
    unsigned __int128 p0 = (unsigned __int128)0xD2E7470EE14C6C93ull * x0;
    unsigned __int128 p1 = (unsigned __int128)0xCA5A826395121157ull * x2;
    uint64_t hi0 = (uint64_t)(p0 >> 64), lo0 = (uint64_t)p0;
    uint64_t hi1 = (uint64_t)(p1 >> 64), lo1 = (uint64_t)p1;
    uint64_t y0 = hi1 ^ x1 ^ k0;
    uint64_t y1 = lo1;
    uint64_t y2 = hi0 ^ x3 ^ k1;
    uint64_t y3 = lo0;
    x0 = y0; x1 = y1; x2 = y2; x3 = y3;
  }
  out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

void orc_philox4x64_10(const uint64_t ctr[4], const uint64_t key[2], uint64_t out[4]) {
  orc_philox4x64_rounds(ctr, key, 10, out);
}

/* ------------------------------------------------------------------------------------ */
/* Base graph: symmetric CSR built from an undirected simple edge list (Sec. 3.1: base    */
/* topology G(V, E)).  Arc a of row v goes to col[a] and belongs to undirected edge eid[a].*/
/* ------------------------------------------------------------------------------------ */

int orc_build_csr(int32_t n, int64_t m, const int32_t *eu, const int32_t *ev,
                  int64_t *row_ptr, int32_t *col, int32_t *eid) {
  if (n < 0 || m < 0) return ORC_EINVAL;
  for (int64_t e = 0; e < m; ++e) {
    if (eu[e] < 0 || eu[e] >= n || ev[e] < 0 || ev[e] >= n || eu[e] == ev[e]) return ORC_EINVAL;
  }
  for (int32_t v = 0; v <= n; ++v) row_ptr[v] = 0;
  for (int64_t e = 0; e < m; ++e) {
    row_ptr[eu[e] + 1]++;
    row_ptr[ev[e] + 1]++;
  }
  for (int32_t v = 0; v < n; ++v) row_ptr[v + 1] += row_ptr[v];
  int64_t *fill = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
  if (!fill) return ORC_ENOMEM;
  for (int32_t v = 0; v < n; ++v) fill[v] = row_ptr[v];
  for (int64_t e = 0; e < m; ++e) {
    int32_t a = eu[e], b = ev[e];
    col[fill[a]] = b; eid[fill[a]] = (int32_t)e; fill[a]++;
    col[fill[b]] = a; eid[fill[b]] = (int32_t)e; fill[b]++;
  }
  free(fill);
  /* reject duplicate edges: sort each row by neighbour (insertion sort; rows are short) */
  for (int32_t v = 0; v < n; ++v) {
    for (int64_t i = row_ptr[v] + 1; i < row_ptr[v + 1]; ++i) {
      int32_t c = col[i], d = eid[i];
      int64_t j = i - 1;
      while (j >= row_ptr[v] && col[j] > c) {
        col[j + 1] = col[j]; eid[j + 1] = eid[j]; --j;
      }
      col[j + 1] = c; eid[j + 1] = d;
    }
    for (int64_t i = row_ptr[v] + 1; i < row_ptr[v + 1]; ++i)
      if (col[i] == col[i - 1]) return ORC_EINVAL;
  }
  return ORC_OK;
}

/* ------------------------------------------------------------------------------------ */
/* One network realization (Sec. 3.1: network state Y -> working graph H).  Edge e of      */
/* realization r of graph g draws (u0, u1, -, -) = Philox4x32-10(ctr = (e, r, g, 0),       */
/* key = seed); it survives iff u0 < T_e with T_e = floor(p_e 2^32) (T_e = 2^32 for p=1),  */
/* and its length is w_e = lo_e + floor(u1 (hi_e - lo_e + 1) / 2^32).                     */
/* ------------------------------------------------------------------------------------ */

uint64_t orc_survival_threshold(double p) {
  if (!(p > 0.0)) return 0;
  if (p >= 1.0) return (uint64_t)1 << 32;
  return (uint64_t)floor(p * 4294967296.0);
}

/* With a weight table (wtab_ptr non-NULL) edge e's length is discrete with the law given by  */
/* its thresholds t_k = wtab[wtab_ptr[e] + k] (non-decreasing): lo + #{k : t_k <= u1},         */
/* capped at hi (the integer inverse-CDF draw of Sec. 9's rounded and clipped normal law).    */
void orc_realize_law(int64_t m, uint64_t seed, uint32_t graph_tag, uint32_t r,
                     const uint64_t *thresh, uint64_t thresh_all,
                     const uint32_t *w_lo, const uint32_t *w_hi, uint32_t w_lo_all,
                     uint32_t w_hi_all, const uint32_t *wtab_ptr, const uint32_t *wtab,
                     uint8_t *alive, uint32_t *w) {
  uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  for (int64_t e = 0; e < m; ++e) {
    uint32_t ctr[4] = {(uint32_t)e, r, graph_tag, 0u};
    uint32_t u[4];
    orc_philox4x32_10(ctr, key, u);
    uint64_t T = thresh ? thresh[e] : thresh_all;
    uint32_t lo = w_lo ? w_lo[e] : w_lo_all;
    uint32_t hi = w_hi ? w_hi[e] : w_hi_all;
    alive[e] = ((uint64_t)u[0] < T) ? 1 : 0;
    if (wtab_ptr) {
      uint32_t k = 0;
      for (uint32_t t = wtab_ptr[e]; t < wtab_ptr[e + 1]; ++t) k += (wtab[t] <= u[1]) ? 1u : 0u;
      w[e] = (lo + k < hi) ? lo + k : hi;
    } else {
      uint64_t span = (uint64_t)hi - (uint64_t)lo + 1u;
      w[e] = lo + (uint32_t)(((uint64_t)u[1] * span) >> 32);
    }
  }
}

void orc_realize(int64_t m, uint64_t seed, uint32_t graph_tag, uint32_t r,
                 const uint64_t *thresh, uint64_t thresh_all,
                 const uint32_t *w_lo, const uint32_t *w_hi, uint32_t w_lo_all, uint32_t w_hi_all,
                 uint8_t *alive, uint32_t *w) {
  orc_realize_law(m, seed, graph_tag, r, thresh, thresh_all, w_lo, w_hi, w_lo_all, w_hi_all,
                  NULL, NULL, alive, w);
}

/* Thresholds of the rounded and clipped normal length law (Sec. 9, Les Miserables setting):  */
/* x ~ N(mu_e, sigma_e^2), mu_e = w0_e + rho_mu (wmax - w0_e), sigma_e = rho_sigma (wmax -    */
/* w0_e), length = round(x) clipped to [w0_e, wmax].  Edge e gets wmax - w0_e thresholds       */
/* t_k = min(floor(2^32 F(w0_e + k)), 2^32 - 1), F(x) = Phi((x + 1/2 - mu_e) / sigma_e), the   */
/* probability that the clipped, rounded draw is at most x; ptr[e] indexes them.             */
void orc_weight_table_normal(int64_t m, const uint32_t *w0, uint32_t wmax, double rho_mu,
                             double rho_sigma, uint32_t *ptr, uint32_t *tab) {
  uint32_t o = 0;
  for (int64_t e = 0; e < m; ++e) {
    ptr[e] = o;
    const double span = (double)wmax - (double)w0[e];
    const double mu = (double)w0[e] + rho_mu * span, sigma = rho_sigma * span;
    for (uint32_t x = w0[e]; x < wmax; ++x) {
      double F;
      if (sigma > 0.0) F = 0.5 * erfc(-(((double)x + 0.5 - mu) / sigma) / sqrt(2.0));
      else F = ((double)x + 0.5 >= mu) ? 1.0 : 0.0;
      double t = floor(ldexp(F, 32));
      tab[o++] = t >= 4294967295.0 ? 0xFFFFFFFFu : (uint32_t)t;
    }
  }
  ptr[m] = o;
}

/* ------------------------------------------------------------------------------------ */
/* Components K(i; H) of the realized graph (Sec. 3.2).  comp[v] = smallest vertex id of  */
/* v's component; csize[v] = |K(v; H)|.  Plain BFS started from each unvisited vertex in  */
/* increasing id order.                                                                   */
/* ------------------------------------------------------------------------------------ */

int orc_components(int32_t n, const int64_t *row_ptr, const int32_t *col, const int32_t *eid,
                   const uint8_t *alive, int32_t *comp, int32_t *csize) {
  int32_t *queue = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
  if (!queue) return ORC_ENOMEM;
  for (int32_t v = 0; v < n; ++v) comp[v] = -1;
  for (int32_t s = 0; s < n; ++s) {
    if (comp[s] >= 0) continue;
    int32_t head = 0, tail = 0;
    queue[tail++] = s;
    comp[s] = s;
    while (head < tail) {
      int32_t v = queue[head++];
      for (int64_t a = row_ptr[v]; a < row_ptr[v + 1]; ++a) {
        if (!alive[eid[a]]) continue;
        int32_t u = col[a];
        if (comp[u] < 0) { comp[u] = s; queue[tail++] = u; }
      }
    }
    for (int32_t i = 0; i < tail; ++i) csize[queue[i]] = tail;
  }
  free(queue);
  return ORC_OK;
}

/* ------------------------------------------------------------------------------------ */
/* Weighted single-source shortest paths with path counting (Sec. 3.1: d_H(s,t) and       */
/* sigma_st(H)).  Textbook Dijkstra with a binary heap (lazy deletion).  sigma is counted  */
/* exactly in 64-bit integers; an overflow makes the call return ORC_EOVERFLOW.           */
/* order[] receives the settled vertices in non-decreasing distance; *n_settled its size.  */
/* ------------------------------------------------------------------------------------ */

typedef struct { uint64_t d; int32_t v; } heap_item;

static void heap_push(heap_item *h, int64_t *size, uint64_t d, int32_t v) {
  int64_t i = (*size)++;
  h[i].d = d; h[i].v = v;
  while (i > 0) {
    int64_t p = (i - 1) / 2;
    if (h[p].d < h[i].d || (h[p].d == h[i].d && h[p].v <= h[i].v)) break;
    heap_item t = h[p]; h[p] = h[i]; h[i] = t;
    i = p;
  }
}

static heap_item heap_pop(heap_item *h, int64_t *size) {
  heap_item top = h[0];
  h[0] = h[--(*size)];
  int64_t i = 0;
  for (;;) {
    int64_t l = 2 * i + 1, r = l + 1, b = i;
    if (l < *size && (h[l].d < h[b].d || (h[l].d == h[b].d && h[l].v < h[b].v))) b = l;
    if (r < *size && (h[r].d < h[b].d || (h[r].d == h[b].d && h[r].v < h[b].v))) b = r;
    if (b == i) break;
    heap_item t = h[b]; h[b] = h[i]; h[i] = t;
    i = b;
  }
  return top;
}

int orc_sssp(int32_t n, const int64_t *row_ptr, const int32_t *col, const int32_t *eid,
             const uint8_t *alive, const uint32_t *w, int32_t s,
             uint64_t *dist, uint64_t *sigma, int32_t *order, int32_t *n_settled) {
  int64_t arcs = row_ptr[n];
  heap_item *heap = (heap_item *)malloc(sizeof(heap_item) * (size_t)(arcs + 2));
  uint8_t *done = (uint8_t *)calloc((size_t)(n > 0 ? n : 1), 1);
  if (!heap || !done) { free(heap); free(done); return ORC_ENOMEM; }
  int status = ORC_OK;
  for (int32_t v = 0; v < n; ++v) { dist[v] = ORC_INF; sigma[v] = 0; }
  dist[s] = 0; sigma[s] = 1;
  int64_t hs = 0;
  int32_t ns = 0;
  heap_push(heap, &hs, 0, s);
  while (hs > 0) {
    heap_item it = heap_pop(heap, &hs);
    int32_t v = it.v;
    if (done[v] || it.d != dist[v]) continue;
    done[v] = 1;
    order[ns++] = v;
    for (int64_t a = row_ptr[v]; a < row_ptr[v + 1]; ++a) {
      int32_t e = eid[a];
      if (!alive[e]) continue;
      int32_t u = col[a];
      uint64_t nd = dist[v] + (uint64_t)w[e];
      if (nd < dist[u]) {
        dist[u] = nd;
        sigma[u] = sigma[v];
        heap_push(heap, &hs, nd, u);
      } else if (nd == dist[u]) {
        uint64_t t;
        if (__builtin_add_overflow(sigma[u], sigma[v], &t)) status = ORC_EOVERFLOW;
        sigma[u] = t;
      }
    }
  }
  *n_settled = ns;
  free(heap); free(done);
  return status;
}

/* ------------------------------------------------------------------------------------ */
/* Weighted betweenness B_v(H) over ordered pairs (Sec. 3.1, the non-normalised           */
/* definition: sum over s != t, s != v != t with t reachable of sigma_st(v) / sigma_st).   */
/* Computed with Brandes' dependency recursion: for each source s, in non-increasing       */
/* distance, delta_s(v) = sum over successors w of (sigma_v / sigma_w)(1 + delta_s(w)),    */
/* where w is a successor of v iff d(s,v) + len(v,w) = d(s,w); then B_v += delta_s(v).     */
/* Only sources with src_mask[s] != 0 are used (src_mask NULL = every source).            */
/* ------------------------------------------------------------------------------------ */

int orc_brandes(int32_t n, const int64_t *row_ptr, const int32_t *col, const int32_t *eid,
                const uint8_t *alive, const uint32_t *w, const uint8_t *src_mask, double *bc) {
  uint64_t *dist = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)(n > 0 ? n : 1));
  uint64_t *sigma = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)(n > 0 ? n : 1));
  int32_t *order = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
  double *delta = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
  if (!dist || !sigma || !order || !delta) {
    free(dist); free(sigma); free(order); free(delta);
    return ORC_ENOMEM;
  }
  int status = ORC_OK;
  for (int32_t v = 0; v < n; ++v) bc[v] = 0.0;
  for (int32_t s = 0; s < n; ++s) {
    if (src_mask && !src_mask[s]) continue;
    int32_t ns = 0;
    int st = orc_sssp(n, row_ptr, col, eid, alive, w, s, dist, sigma, order, &ns);
    if (st == ORC_ENOMEM) { status = st; break; }
    if (st != ORC_OK) status = st;
    for (int32_t i = 0; i < ns; ++i) delta[order[i]] = 0.0;
    for (int32_t i = ns - 1; i >= 0; --i) {
      int32_t v = order[i];
      double acc = 0.0;
      for (int64_t a = row_ptr[v]; a < row_ptr[v + 1]; ++a) {
        int32_t e = eid[a];
        if (!alive[e]) continue;
        int32_t x = col[a];
        if (dist[x] != ORC_INF && dist[v] + (uint64_t)w[e] == dist[x])
          acc += ((double)sigma[v] / (double)sigma[x]) * (1.0 + delta[x]);
      }
      delta[v] = acc;
      if (v != s) bc[v] += delta[v];
    }
  }
  free(dist); free(sigma); free(order); free(delta);
  return status;
}

/* ------------------------------------------------------------------------------------ */
/* Tie-broken local centre per component (Sec. 3.2 eq. local-center; Cor. on             */
/* deterministic tie-breaking; Sec. 7.1 constrained selector Sel_W).                      */
/*   valid component K: |K| >= k_min.  Candidate set X = K intersect W (W = V if absent).  */
/*   B* = max_X B, tau = tie_rel * B*, ties = {v in X : B_v >= B* - tau}, centre = min id. */
/*   With top_k > 0 the centre must also rank within the first top_k of K:                */
/*   rank = 1 + #{u in K : B_u > B_c + tauK, or |B_u - B_c| <= tauK and u < c},             */
/*   tauK = tie_rel * max_K B.  centre[root] = -1 encodes "no valid continuation".         */
/* ------------------------------------------------------------------------------------ */

/* With tie_random the centre is drawn uniformly from the tie set instead (Remark on        */
/* randomized tie-breaking, Sec. 4.1): u = Philox4x32-10(counter (root, r, graph_tag, 3),    */
/* key = seed)[0] with root the smallest id of K, the floor(u |ties| / 2^32)-th tied        */
/* candidate in ascending id order.                                                         */
void orc_select_ex(int32_t n, const int32_t *comp, const int32_t *csize, const double *bc,
                   uint32_t k_min, const uint8_t *in_w, uint32_t top_k, double tie_rel,
                   int32_t tie_random, uint64_t seed, uint32_t graph_tag, uint32_t r,
                   int32_t *centre);

void orc_select(int32_t n, const int32_t *comp, const int32_t *csize, const double *bc,
                uint32_t k_min, const uint8_t *in_w, uint32_t top_k, double tie_rel,
                int32_t *centre) {
  orc_select_ex(n, comp, csize, bc, k_min, in_w, top_k, tie_rel, 0, 0, 0, 0, centre);
}

void orc_select_ex(int32_t n, const int32_t *comp, const int32_t *csize, const double *bc,
                   uint32_t k_min, const uint8_t *in_w, uint32_t top_k, double tie_rel,
                   int32_t tie_random, uint64_t seed, uint32_t graph_tag, uint32_t r,
                   int32_t *centre) {
  for (int32_t v = 0; v < n; ++v) centre[v] = -1;
  for (int32_t root = 0; root < n; ++root) {
    if (comp[root] != root) continue;
    if ((uint32_t)csize[root] < k_min) continue;
    double bstar = -1.0, bmaxK = 0.0;
    for (int32_t v = 0; v < n; ++v) {
      if (comp[v] != root) continue;
      if (bc[v] > bmaxK) bmaxK = bc[v];
      if (in_w && !in_w[v]) continue;
      if (bc[v] > bstar) bstar = bc[v];
    }
    if (bstar < 0.0) continue; /* K has no candidate */
    double tau = tie_rel * bstar;
    int32_t c = -1;
    if (tie_random) {
      uint32_t ties = 0;
      for (int32_t v = 0; v < n; ++v)
        if (comp[v] == root && !(in_w && !in_w[v]) && bc[v] >= bstar - tau) ties++;
      const uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
      const uint32_t ctr[4] = {(uint32_t)root, r, graph_tag, 3u};
      uint32_t u[4];
      orc_philox4x32_10(ctr, key, u);
      uint32_t k = (uint32_t)(((uint64_t)u[0] * (uint64_t)ties) >> 32);
      for (int32_t v = 0; v < n && c < 0; ++v) {
        if (comp[v] != root || (in_w && !in_w[v]) || bc[v] < bstar - tau) continue;
        if (k == 0) c = v; else k--;
      }
    } else {
      for (int32_t v = 0; v < n && c < 0; ++v) {
        if (comp[v] != root || (in_w && !in_w[v])) continue;
        if (bc[v] >= bstar - tau) c = v;
      }
    }
    if (top_k > 0) {
      double tauK = tie_rel * bmaxK;
      uint32_t rank = 1;
      for (int32_t u = 0; u < n; ++u) {
        if (comp[u] != root || u == c) continue;
        double diff = bc[u] - bc[c];
        if (diff > tauK || (fabs(diff) <= tauK && u < c)) rank++;
      }
      if (rank > top_k) continue;
    }
    centre[root] = c;
  }
}

/* ------------------------------------------------------------------------------------ */
/* Monte Carlo transition counts (Alg. 1 SampleNext and Alg. 2 row-wise construction).    */
/* Realization r in [r_begin, r_begin + r_count) serves every anchor i at once (the row   */
/* law depends only on the law of H, Prop. on order/branch invariance):                   */
/*   next(i) = bottom if |K(i;H)| < k_min or K(i;H) has no admissible centre,             */
/*   next(i) = centre of K(i;H) otherwise;  counts[i*(n+1) + next(i)] += 1 (bottom = n).  */
/* Fallback selector Sel_{W,fb} (Sec. 7.3): with fb_node >= 0, a valid component whose    */
/* candidate set admits no centre reports fb_node instead of bottom, and fb_count[i]      */
/* (when given) counts those redirected draws; invalid components still absorb.           */
/* Only sources inside valid components enter the betweenness (a vertex's betweenness     */
/* only depends on sources of its own component).                                         */
/* stats[0] += realizations whose sigma overflowed 64 bits.                               */
/* ------------------------------------------------------------------------------------ */

int orc_count_transitions(int32_t n, int64_t m, const int64_t *row_ptr, const int32_t *col,
                          const int32_t *eid, uint64_t seed, uint32_t graph_tag,
                          uint32_t r_begin, uint32_t r_count,
                          const uint64_t *thresh, uint64_t thresh_all,
                          const uint32_t *w_lo, const uint32_t *w_hi,
                          uint32_t w_lo_all, uint32_t w_hi_all,
                          uint32_t k_min, const uint8_t *in_w, uint32_t top_k, double tie_rel,
                          uint32_t *counts, uint64_t *stats, int32_t fb_node,
                          uint32_t *fb_count, int32_t tie_random, const uint32_t *wtab_ptr,
                          const uint32_t *wtab) {
  size_t nn = (size_t)(n > 0 ? n : 1), mm = (size_t)(m > 0 ? m : 1);
  uint8_t *alive = (uint8_t *)malloc(mm);
  uint32_t *w = (uint32_t *)malloc(sizeof(uint32_t) * mm);
  int32_t *comp = (int32_t *)malloc(sizeof(int32_t) * nn);
  int32_t *csize = (int32_t *)malloc(sizeof(int32_t) * nn);
  int32_t *centre = (int32_t *)malloc(sizeof(int32_t) * nn);
  uint8_t *src = (uint8_t *)malloc(nn);
  double *bc = (double *)malloc(sizeof(double) * nn);
  int status = ORC_OK;
  if (!alive || !w || !comp || !csize || !centre || !src || !bc) { status = ORC_ENOMEM; goto out; }
  for (uint32_t k = 0; k < r_count; ++k) {
    uint32_t r = r_begin + k;
    orc_realize_law(m, seed, graph_tag, r, thresh, thresh_all, w_lo, w_hi, w_lo_all, w_hi_all,
                    wtab_ptr, wtab, alive, w);
    int st = orc_components(n, row_ptr, col, eid, alive, comp, csize);
    if (st != ORC_OK) { status = st; goto out; }
    /* sources: members of valid components that contain at least one candidate */
    for (int32_t v = 0; v < n; ++v) src[v] = 0;
    for (int32_t v = 0; v < n; ++v) {
      if ((uint32_t)csize[v] >= k_min && (!in_w || in_w[v])) src[comp[v]] = 1; /* mark root */
    }
    for (int32_t v = 0; v < n; ++v) src[v] = src[comp[v]];
    st = orc_brandes(n, row_ptr, col, eid, alive, w, src, bc);
    if (st == ORC_ENOMEM) { status = st; goto out; }
    if (st == ORC_EOVERFLOW) { if (stats) stats[0]++; status = ORC_EOVERFLOW; }
    orc_select_ex(n, comp, csize, bc, k_min, in_w, top_k, tie_rel, tie_random, seed, graph_tag,
                  r, centre);
    for (int32_t i = 0; i < n; ++i) {
      int32_t c = centre[comp[i]];
      size_t col_idx = (c < 0) ? (size_t)n : (size_t)c;
      if (c < 0 && fb_node >= 0 && (uint32_t)csize[comp[i]] >= k_min) {
        col_idx = (size_t)fb_node;
        if (fb_count) fb_count[i] += 1u;
      }
      counts[(size_t)i * (size_t)(n + 1) + col_idx] += 1u;
    }
  }
out:
  free(alive); free(w); free(comp); free(csize); free(centre); free(src); free(bc);
  return status;
}

/* ------------------------------------------------------------------------------------ */
/* Literal row-wise construction (Alg. 2 with M independent SampleNext(i) calls per row,   */
/* no realization shared between rows), optionally on anchor-dependent r-hop               */
/* neighbourhoods (Sec. 9 weighted-network experiment).  Draw m of row i uses realization  */
/* rho = m n + i.  With hop_radius > 0 the working graph is the realized graph induced on   */
/* S_r(i), the nodes within hop_radius hops of i in the base graph; K is i's component      */
/* there.  next(i) as in orc_count_transitions (fallback and randomised ties included,      */
/* with rho as the realization index of the tie draw).                                      */
/* ------------------------------------------------------------------------------------ */

int orc_count_per_row(int32_t n, int64_t m, const int64_t *row_ptr, const int32_t *col,
                      const int32_t *eid, uint64_t seed, uint32_t graph_tag, uint32_t r_begin,
                      uint32_t r_count, const uint64_t *thresh, uint64_t thresh_all,
                      const uint32_t *w_lo, const uint32_t *w_hi, uint32_t w_lo_all,
                      uint32_t w_hi_all, const uint32_t *wtab_ptr, const uint32_t *wtab,
                      uint32_t k_min, const uint8_t *in_w, uint32_t top_k, double tie_rel,
                      int32_t tie_random, int32_t fb_node, uint32_t hop_radius,
                      uint32_t *counts, uint32_t *fb_count, uint64_t *stats) {
  size_t nn = (size_t)(n > 0 ? n : 1), mm = (size_t)(m > 0 ? m : 1);
  uint8_t *alive = (uint8_t *)malloc(mm);
  uint32_t *w = (uint32_t *)malloc(sizeof(uint32_t) * mm);
  int32_t *comp = (int32_t *)malloc(sizeof(int32_t) * nn);
  int32_t *csize = (int32_t *)malloc(sizeof(int32_t) * nn);
  int32_t *centre = (int32_t *)malloc(sizeof(int32_t) * nn);
  uint8_t *src = (uint8_t *)malloc(nn);
  double *bc = (double *)malloc(sizeof(double) * nn);
  int32_t *hop = (int32_t *)malloc(sizeof(int32_t) * nn);
  int32_t *queue = (int32_t *)malloc(sizeof(int32_t) * nn);
  int status = ORC_OK;
  if (!alive || !w || !comp || !csize || !centre || !src || !bc || !hop || !queue) {
    status = ORC_ENOMEM;
    goto out;
  }
  for (uint32_t k = 0; k < r_count; ++k) {
    for (int32_t i = 0; i < n; ++i) {
      const uint32_t rho = (r_begin + k) * (uint32_t)n + (uint32_t)i;
      orc_realize_law(m, seed, graph_tag, rho, thresh, thresh_all, w_lo, w_hi, w_lo_all,
                      w_hi_all, wtab_ptr, wtab, alive, w);
      if (hop_radius > 0) {
        /* S_r(i): breadth-first search of the base graph from i, hop_radius levels */
        for (int32_t v = 0; v < n; ++v) hop[v] = -1;
        int32_t head = 0, tail = 0;
        hop[i] = 0;
        queue[tail++] = i;
        while (head < tail) {
          const int32_t v = queue[head++];
          if ((uint32_t)hop[v] == hop_radius) continue;
          for (int64_t a = row_ptr[v]; a < row_ptr[v + 1]; ++a)
            if (hop[col[a]] < 0) { hop[col[a]] = hop[v] + 1; queue[tail++] = col[a]; }
        }
        for (int32_t v = 0; v < n; ++v)
          for (int64_t a = row_ptr[v]; a < row_ptr[v + 1]; ++a)
            if (hop[v] < 0 || hop[col[a]] < 0) alive[eid[a]] = 0;
      }
      int st = orc_components(n, row_ptr, col, eid, alive, comp, csize);
      if (st != ORC_OK) { status = st; goto out; }
      const int32_t root = comp[i];
      int has_cand = 0;
      for (int32_t v = 0; v < n; ++v) {
        src[v] = (comp[v] == root) ? 1 : 0;
        if (src[v] && (!in_w || in_w[v])) has_cand = 1;
      }
      size_t col_idx = (size_t)n;
      if ((uint32_t)csize[i] >= k_min && has_cand) {
        st = orc_brandes(n, row_ptr, col, eid, alive, w, src, bc);
        if (st == ORC_ENOMEM) { status = st; goto out; }
        if (st == ORC_EOVERFLOW) { if (stats) stats[0]++; status = ORC_EOVERFLOW; }
        orc_select_ex(n, comp, csize, bc, k_min, in_w, top_k, tie_rel, tie_random, seed,
                      graph_tag, rho, centre);
        if (centre[root] >= 0) col_idx = (size_t)centre[root];
      }
      if (col_idx == (size_t)n && fb_node >= 0 && (uint32_t)csize[i] >= k_min) {
        col_idx = (size_t)fb_node;
        if (fb_count) fb_count[i] += 1u;
      }
      counts[(size_t)i * (size_t)(n + 1) + col_idx] += 1u;
    }
  }
out:
  free(alive); free(w); free(comp); free(csize); free(centre); free(src); free(bc); free(hop);
  free(queue);
  return status;
}

/* ------------------------------------------------------------------------------------ */
/* Realization-level bootstrap weights (Sec. 8: nonparametric bootstrap of b by resampling */
/* the draws with replacement; with realization sharing the draws of all anchors come from */
/* the same realizations, so whole realizations are resampled).  Replicate b draws R       */
/* indices k = 0 .. R-1: u = Philox4x32-10(counter (k, b, 0, 2), key = seed)[0], index =     */
/* floor(u R / 2^32); w[r] = how often r was drawn (sum w = R).                             */
/* ------------------------------------------------------------------------------------ */

void orc_bootstrap_weights(uint32_t R, uint32_t b, uint64_t seed, uint32_t *w) {
  const uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  for (uint32_t r = 0; r < R; ++r) w[r] = 0;
  for (uint32_t k = 0; k < R; ++k) {
    const uint32_t ctr[4] = {k, b, 0u, 2u};
    uint32_t out[4];
    orc_philox4x32_10(ctr, key, out);
    w[(uint32_t)(((uint64_t)out[0] * (uint64_t)R) >> 32)] += 1u;
  }
}

/* ------------------------------------------------------------------------------------ */
/* Ordered local Top-k of every valid component (Sec. 2.3: the component-wise top-k set   */
/* of eq. topk-comp, the local top-k of Def. local-topk, and the rank-r centre of the      */
/* remark after the Prop. on set-valued states).  The ordering pi of K repeats the          */
/* tie-broken centre rule on what is left of K: pi(1) is the centre of K (candidates =     */
/* K), pi(t) the centre of K minus {pi(1), ..., pi(t-1)}: B* = max over the remaining      */
/* nodes, ties = {v : B_v >= B* - tie_rel * B*}, smallest id.                              */
/* order[root * k + t] = pi(t + 1) for t < min(k, |K|) on valid roots (|K| >= k_min),       */
/* -1 elsewhere.  taken: scratch of n bytes.                                              */
/* ------------------------------------------------------------------------------------ */

void orc_topk_order(int32_t n, const int32_t *comp, const int32_t *csize, const double *bc,
                    uint32_t k_min, uint32_t k, double tie_rel, int32_t *order,
                    uint8_t *taken) {
  for (size_t q = 0; q < (size_t)n * k; ++q) order[q] = -1;
  for (int32_t v = 0; v < n; ++v) taken[v] = 0;
  for (int32_t root = 0; root < n; ++root) {
    if (comp[root] != root || (uint32_t)csize[root] < k_min) continue;
    for (uint32_t t = 0; t < k; ++t) {
      double bstar = -1.0;
      for (int32_t v = 0; v < n; ++v)
        if (comp[v] == root && !taken[v] && bc[v] > bstar) bstar = bc[v];
      if (bstar < 0.0) break; /* K exhausted */
      const double tau = tie_rel * bstar;
      int32_t pick = -1;
      for (int32_t v = 0; v < n && pick < 0; ++v)
        if (comp[v] == root && !taken[v] && bc[v] >= bstar - tau) pick = v;
      taken[pick] = 1;
      order[(size_t)root * k + t] = pick;
    }
  }
}

/* ------------------------------------------------------------------------------------ */
/* Transition counts with a rank-r report and the valued local Top-k step reward          */
/* (Sec. 6.2 ell^(k,gamma)_i = sum of gamma_v over the local Top-k set of anchor i, and     */
/* Sec. 6.3 its pool-restricted form over Top-k intersect W_pool).  Per realization and     */
/* anchor i with a valid component K = K(i):                                               */
/*   next(i) = pi_K(report_rank) if |K| >= report_rank, else bottom (report_rank = 1 is the  */
/*   tie-broken centre of orc_select with no candidate pool and no rank cutoff);            */
/*   psi_sum[i] += sum_{t < min(reward_k, |K|)} gamma[pi_K(t+1)] * [pi_K(t+1) in pool]      */
/* (gamma NULL: 1; pool NULL: every node); an anchor of an invalid component adds nothing   */
/* and moves to bottom.  counts and psi_sum may each be NULL; both are accumulated.         */
/* ------------------------------------------------------------------------------------ */

int orc_count_rewards(int32_t n, int64_t m, const int64_t *row_ptr, const int32_t *col,
                      const int32_t *eid, uint64_t seed, uint32_t graph_tag,
                      uint32_t r_begin, uint32_t r_count,
                      const uint64_t *thresh, uint64_t thresh_all,
                      const uint32_t *w_lo, const uint32_t *w_hi,
                      uint32_t w_lo_all, uint32_t w_hi_all,
                      uint32_t k_min, double tie_rel, uint32_t reward_k, const double *gamma,
                      const uint8_t *pool, uint32_t report_rank, uint32_t *counts,
                      double *psi_sum) {
  if (report_rank < 1) return ORC_EINVAL;
  const uint32_t k = reward_k > report_rank ? reward_k : report_rank;
  size_t nn = (size_t)(n > 0 ? n : 1), mm = (size_t)(m > 0 ? m : 1);
  uint8_t *alive = (uint8_t *)malloc(mm);
  uint32_t *w = (uint32_t *)malloc(sizeof(uint32_t) * mm);
  int32_t *comp = (int32_t *)malloc(sizeof(int32_t) * nn);
  int32_t *csize = (int32_t *)malloc(sizeof(int32_t) * nn);
  uint8_t *src = (uint8_t *)malloc(nn);
  double *bc = (double *)malloc(sizeof(double) * nn);
  int32_t *order = (int32_t *)malloc(sizeof(int32_t) * nn * k);
  int status = ORC_OK;
  if (!alive || !w || !comp || !csize || !src || !bc || !order) { status = ORC_ENOMEM; goto out; }
  for (uint32_t q = 0; q < r_count; ++q) {
    uint32_t r = r_begin + q;
    orc_realize(m, seed, graph_tag, r, thresh, thresh_all, w_lo, w_hi, w_lo_all, w_hi_all, alive, w);
    int st = orc_components(n, row_ptr, col, eid, alive, comp, csize);
    if (st != ORC_OK) { status = st; goto out; }
    for (int32_t v = 0; v < n; ++v) src[v] = (uint32_t)csize[comp[v]] >= k_min ? 1 : 0;
    st = orc_brandes(n, row_ptr, col, eid, alive, w, src, bc);
    if (st == ORC_ENOMEM) { status = st; goto out; }
    if (st == ORC_EOVERFLOW) status = ORC_EOVERFLOW;
    orc_topk_order(n, comp, csize, bc, k_min, k, tie_rel, order, src);
    for (int32_t i = 0; i < n; ++i) {
      const int32_t *pi = order + (size_t)comp[i] * k;
      if (counts) {
        const int32_t c = pi[report_rank - 1];
        counts[(size_t)i * (size_t)(n + 1) + (c < 0 ? (size_t)n : (size_t)c)] += 1u;
      }
      if (psi_sum) {
        double ell = 0.0;
        for (uint32_t t = 0; t < reward_k; ++t) {
          const int32_t v = pi[t];
          if (v < 0) break;
          if (pool && !pool[v]) continue;
          ell += gamma ? gamma[v] : 1.0;
        }
        psi_sum[i] += ell;
      }
    }
  }
out:
  free(alive); free(w); free(comp); free(csize); free(src); free(bc); free(order);
  return status;
}

/* ------------------------------------------------------------------------------------ */
/* Dense Gaussian elimination with partial pivoting: solves A x = b in place (A is n x n  */
/* row-major and is destroyed; b is overwritten by x).                                    */
/* ------------------------------------------------------------------------------------ */

int orc_gauss_solve(int32_t n, double *A, double *b, int32_t nrhs) {
  for (int32_t k = 0; k < n; ++k) {
    int32_t piv = k;
    double best = fabs(A[(size_t)k * n + k]);
    for (int32_t i = k + 1; i < n; ++i) {
      double a = fabs(A[(size_t)i * n + k]);
      if (a > best) { best = a; piv = i; }
    }
    if (best == 0.0) return ORC_ESINGULAR;
    if (piv != k) {
      for (int32_t j = 0; j < n; ++j) {
        double t = A[(size_t)k * n + j]; A[(size_t)k * n + j] = A[(size_t)piv * n + j]; A[(size_t)piv * n + j] = t;
      }
      for (int32_t q = 0; q < nrhs; ++q) {
        double t = b[(size_t)k * nrhs + q]; b[(size_t)k * nrhs + q] = b[(size_t)piv * nrhs + q]; b[(size_t)piv * nrhs + q] = t;
      }
    }
    for (int32_t i = k + 1; i < n; ++i) {
      double f = A[(size_t)i * n + k] / A[(size_t)k * n + k];
      if (f == 0.0) continue;
      for (int32_t j = k; j < n; ++j) A[(size_t)i * n + j] -= f * A[(size_t)k * n + j];
      for (int32_t q = 0; q < nrhs; ++q) b[(size_t)i * nrhs + q] -= f * b[(size_t)k * nrhs + q];
    }
  }
  for (int32_t i = n - 1; i >= 0; --i) {
    for (int32_t q = 0; q < nrhs; ++q) {
      double acc = b[(size_t)i * nrhs + q];
      for (int32_t j = i + 1; j < n; ++j) acc -= A[(size_t)i * n + j] * b[(size_t)j * nrhs + q];
      b[(size_t)i * nrhs + q] = acc / A[(size_t)i * n + i];
    }
  }
  return ORC_OK;
}

/* ------------------------------------------------------------------------------------ */
/* Kernel assembly from counts (Alg. 2 plus stabilisation, Sec. 8.2, and the analytic     */
/* exogenous stop alpha, Sec. 4):                                                         */
/*   Q_ij = (1 - alpha) counts_ij / R,   r_i = alpha + (1 - alpha) counts_i,bottom / R.   */
/*   If r_i == 0 (possible only for alpha = 0): r_i = eta and row i's transient part is   */
/*   rescaled to sum 1 - eta.                                                              */
/* Q is written densely (n x n row-major), r as a vector.                                 */
/* ------------------------------------------------------------------------------------ */

void orc_assemble_q(int32_t n, const uint32_t *counts, uint32_t R, double alpha, double eta,
                    double *Q, double *r) {
  for (int32_t i = 0; i < n; ++i) {
    const uint32_t *row = counts + (size_t)i * (size_t)(n + 1);
    double tsum = 0.0;
    for (int32_t j = 0; j < n; ++j) {
      Q[(size_t)i * n + j] = (1.0 - alpha) * (double)row[j] / (double)R;
      tsum += Q[(size_t)i * n + j];
    }
    r[i] = alpha + (1.0 - alpha) * (double)row[n] / (double)R;
    if (r[i] == 0.0) {
      r[i] = eta;
      if (tsum > 0.0)
        for (int32_t j = 0; j < n; ++j) Q[(size_t)i * n + j] *= (1.0 - eta) / tsum;
    }
  }
}

/* ------------------------------------------------------------------------------------ */
/* AFC from a transient block (Sec. 4 eqs. fundamental, visits, expected-length, afc-def, */
/* Sec. 6.4 eq. mr-inner-product):  mu = s N with N = (I - Q)^-1, i.e. (I - Q)^T mu^T =    */
/* s^T;  E_s[T] = mu 1;  b = mu / E_s[T];  b_f = b . f.  Full n x n solve.                */
/* ------------------------------------------------------------------------------------ */

int orc_afc_from_q(int32_t n, const double *Q, const double *s, const double *f,
                   double *mu, double *b, double *expected_T, double *b_f) {
  double *A = (double *)malloc(sizeof(double) * (size_t)n * (size_t)n);
  if (!A) return ORC_ENOMEM;
  for (int32_t i = 0; i < n; ++i)
    for (int32_t j = 0; j < n; ++j)
      A[(size_t)i * n + j] = (i == j ? 1.0 : 0.0) - Q[(size_t)j * n + i]; /* (I - Q)^T */
  for (int32_t i = 0; i < n; ++i) mu[i] = s ? s[i] : 1.0 / (double)n;
  int st = orc_gauss_solve(n, A, mu, 1);
  free(A);
  if (st != ORC_OK) return st;
  double T = 0.0;
  for (int32_t i = 0; i < n; ++i) T += mu[i];
  *expected_T = T;
  double bf = 0.0;
  for (int32_t i = 0; i < n; ++i) {
    b[i] = mu[i] / T;
    if (f) bf += b[i] * f[i];
  }
  if (b_f) *b_f = f ? bf : 0.0;
  return ORC_OK;
}

/* counts -> Q -> AFC, full solve.  Also returns r (absorption probabilities). */
int orc_solve_full(int32_t n, const uint32_t *counts, uint32_t R, double alpha, double eta,
                   const double *s, const double *f, double *mu, double *b, double *expected_T,
                   double *b_f) {
  double *Q = (double *)malloc(sizeof(double) * (size_t)n * (size_t)n);
  double *r = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
  if (!Q || !r) { free(Q); free(r); return ORC_ENOMEM; }
  orc_assemble_q(n, counts, R, alpha, eta, Q, r);
  int st = orc_afc_from_q(n, Q, s, f, mu, b, expected_T, b_f);
  free(Q); free(r);
  return st;
}

/* ------------------------------------------------------------------------------------ */
/* Reduced solve on the observed centre states.  C = {j : some count_ij > 0, j in V},     */
/* U = V \ C.  The columns of Q on U are zero, so with (U, C) block order                 */
/*   mu_U = s_U,   mu_C (I - Q_CC) = s_C + s_U Q_UC.                                       */
/* This is an exact rewriting of mu = s N, used where the full n x n system is too large. */
/* c_out receives |C|.                                                                     */
/* ------------------------------------------------------------------------------------ */

int orc_solve_reduced(int32_t n, const uint32_t *counts, uint32_t R, double alpha, double eta,
                      const double *s, const double *f, double *mu, double *b,
                      double *expected_T, double *b_f, int32_t *c_out) {
  size_t nn = (size_t)(n > 0 ? n : 1);
  int32_t *pos = (int32_t *)malloc(sizeof(int32_t) * nn);
  int32_t *cl = (int32_t *)malloc(sizeof(int32_t) * nn);
  double *qrow = (double *)malloc(sizeof(double) * nn);
  if (!pos || !cl || !qrow) { free(pos); free(cl); free(qrow); return ORC_ENOMEM; }
  int32_t c = 0;
  for (int32_t j = 0; j < n; ++j) {
    pos[j] = -1;
    for (int32_t i = 0; i < n; ++i)
      if (counts[(size_t)i * (size_t)(n + 1) + j] > 0) { pos[j] = c; cl[c++] = j; break; }
  }
  *c_out = c;
  double *A = (double *)calloc((size_t)(c > 0 ? c : 1) * (size_t)(c > 0 ? c : 1), sizeof(double));
  double *y = (double *)calloc((size_t)(c > 0 ? c : 1), sizeof(double));
  if (!A || !y) { free(pos); free(cl); free(qrow); free(A); free(y); return ORC_ENOMEM; }
  for (int32_t k = 0; k < c; ++k) A[(size_t)k * c + k] = 1.0; /* A = (I - Q_CC)^T */
  for (int32_t i = 0; i < n; ++i) {
    const uint32_t *row = counts + (size_t)i * (size_t)(n + 1);
    double tsum = 0.0;
    for (int32_t j = 0; j < n; ++j) { qrow[j] = (1.0 - alpha) * (double)row[j] / (double)R; tsum += qrow[j]; }
    double ri = alpha + (1.0 - alpha) * (double)row[n] / (double)R;
    if (ri == 0.0 && tsum > 0.0)
      for (int32_t j = 0; j < n; ++j) qrow[j] *= (1.0 - eta) / tsum;
    double si = s ? s[i] : 1.0 / (double)n;
    if (pos[i] >= 0) {
      for (int32_t k = 0; k < c; ++k) A[(size_t)k * c + pos[i]] -= qrow[cl[k]];
      y[pos[i]] += si;
    } else {
      for (int32_t k = 0; k < c; ++k) y[k] += si * qrow[cl[k]];
    }
  }
  int st = orc_gauss_solve(c, A, y, 1);
  if (st == ORC_OK) {
    for (int32_t i = 0; i < n; ++i) mu[i] = (pos[i] >= 0) ? y[pos[i]] : (s ? s[i] : 1.0 / (double)n);
    double T = 0.0;
    for (int32_t i = 0; i < n; ++i) T += mu[i];
    *expected_T = T;
    double bf = 0.0;
    for (int32_t i = 0; i < n; ++i) { b[i] = mu[i] / T; if (f) bf += b[i] * f[i]; }
    if (b_f) *b_f = f ? bf : 0.0;
  }
  free(pos); free(cl); free(qrow); free(A); free(y);
  return st;
}

/* ------------------------------------------------------------------------------------ */
/* Ranking of AFC scores: u precedes v iff b_u - b_v > tau, or |b_u - b_v| <= tau and     */
/* u < v, with tau = tie_rel * max b.  rank[v] = #{u : u precedes v} (0 = first).          */
/* ------------------------------------------------------------------------------------ */

static int precedes(const double *b, int32_t u, int32_t v, double tau) {
  double d = b[u] - b[v];
  return d > tau || (fabs(d) <= tau && u < v);
}

void orc_rank(int32_t n, const double *b, double tie_rel, int32_t *rank) {
  double bmax = 0.0;
  for (int32_t v = 0; v < n; ++v) if (b[v] > bmax) bmax = b[v];
  double tau = tie_rel * bmax;
  for (int32_t v = 0; v < n; ++v) {
    int32_t r = 0;
    for (int32_t u = 0; u < n; ++u) if (u != v && precedes(b, u, v, tau)) r++;
    rank[v] = r;
  }
}

/* ------------------------------------------------------------------------------------ */
/* Ranking certificates (Sec. 5.5): visit gap G_uv = mu_u - mu_v (eq. pm-gap); crude     */
/* threshold 2 eps / r^2; sharpened threshold (eps / r) max_i |N_iu - N_iv| (eq.          */
/* sharp-gap).  Q is the dense n x n nominal transient block; pairs (u[k], v[k]).         */
/* Outputs per pair: gap[k], crude (same for all pairs), sharp[k].                        */
/* ------------------------------------------------------------------------------------ */

int orc_certificates(int32_t n, const double *Q, const double *s, double eps_bar, double r_min,
                     int32_t npairs, const int32_t *pu, const int32_t *pv,
                     double *gap, double *crude, double *sharp) {
  double *mu = (double *)malloc(sizeof(double) * (size_t)n);
  double *b = (double *)malloc(sizeof(double) * (size_t)n);
  double *A = (double *)malloc(sizeof(double) * (size_t)n * (size_t)n);
  double *Nm = (double *)malloc(sizeof(double) * (size_t)n * (size_t)n);
  if (!mu || !b || !A || !Nm) { free(mu); free(b); free(A); free(Nm); return ORC_ENOMEM; }
  double T = 0.0;
  int st = orc_afc_from_q(n, Q, s, NULL, mu, b, &T, NULL);
  if (st == ORC_OK) {
    /* N = (I - Q)^-1: solve (I - Q) N = I */
    for (int32_t i = 0; i < n; ++i)
      for (int32_t j = 0; j < n; ++j) {
        A[(size_t)i * n + j] = (i == j ? 1.0 : 0.0) - Q[(size_t)i * n + j];
        Nm[(size_t)i * n + j] = (i == j ? 1.0 : 0.0);
      }
    st = orc_gauss_solve(n, A, Nm, n);
  }
  if (st == ORC_OK) {
    *crude = 2.0 * eps_bar / (r_min * r_min);
    for (int32_t k = 0; k < npairs; ++k) {
      int32_t u = pu[k], v = pv[k];
      gap[k] = mu[u] - mu[v];
      double mx = 0.0;
      for (int32_t i = 0; i < n; ++i) {
        double d = fabs(Nm[(size_t)i * n + u] - Nm[(size_t)i * n + v]);
        if (d > mx) mx = d;
      }
      sharp[k] = eps_bar / r_min * mx;
    }
  }
  free(mu); free(b); free(A); free(Nm);
  return st;
}

/* ------------------------------------------------------------------------------------ */
/* Row-wise perturbation sweep (Sec. 5.1 row-wise uncertainty; Sec. 5.4 first-order      */
/* sensitivity; Sec. 5.5 ranking reversals).  For p = 0..P-1 every row i of the nominal   */
/* kernel is perturbed on its support J_i = {j : Q_ij > 0} plus the absorbing column:      */
/*   z_j = 2 u_j - 1, u_j = Philox4x32-10(ctr = (j, i, p, 1), key = seed)[0] / 2^32       */
/*   (j = n for the absorbing column);  d = z - mean(z);  d <- radius d / ||d||_1;         */
/*   q' = max(q + d, 0);  q' <- q' / sum(q');  if q'_abs < r_min the transient part is     */
/*   rescaled to 1 - r_min and q'_abs = r_min.                                             */
/* Then mu' = s N', b' = mu' / mu' 1 (full solve), ranked with orc_rank.  Against the      */
/* nominal ranking the sweep counts:                                                       */
/*   out_counts[0] top-1 changes; [1] top-k set changes; [2] top-k order changes.          */
/*   pair_flips[a*K2+b] (a<b<K2): perturbations where nominal ranks a and b swap order.     */
/*   shift_hist[h]: |rank' - rank0| over the nominal top-K2 nodes, h clipped to H-1.       */
/*   out_f64[0] = max ||b' - b0||_inf; [1] = max ||b' - (b0 + db_lin)||_inf with the       */
/*   first-order prediction db_lin = x/T0 - b0 (x 1)/T0, x = mu0 E N0, E = Q' - Q0;         */
/*   [2] = max over p of max_i (N' 1)_i (uniform transience bound, eq. pm-N-bound).        */
/* Q0 is dense n x n; r0 its absorption vector.                                             */
/* ------------------------------------------------------------------------------------ */

static double perturb_uniform(uint64_t seed, uint32_t j, uint32_t i, uint32_t p) {
  uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  uint32_t ctr[4] = {j, i, p, 1u};
  uint32_t u[4];
  orc_philox4x32_10(ctr, key, u);
  return (double)u[0] / 4294967296.0;
}

void orc_perturb_row(int32_t n, const double *q0, double r0, uint64_t seed, uint32_t i,
                     uint32_t p, double radius, double r_min, double *q, double *r) {
  int32_t supp = 1;
  for (int32_t j = 0; j < n; ++j) if (q0[j] > 0.0) supp++;
  double zsum = 0.0;
  for (int32_t j = 0; j < n; ++j) if (q0[j] > 0.0) zsum += 2.0 * perturb_uniform(seed, (uint32_t)j, i, p) - 1.0;
  double zabs = 2.0 * perturb_uniform(seed, (uint32_t)n, i, p) - 1.0;
  zsum += zabs;
  double mean = zsum / (double)supp;
  double l1 = 0.0;
  for (int32_t j = 0; j < n; ++j)
    if (q0[j] > 0.0) l1 += fabs((2.0 * perturb_uniform(seed, (uint32_t)j, i, p) - 1.0) - mean);
  l1 += fabs(zabs - mean);
  double scale = (l1 > 0.0) ? radius / l1 : 0.0;
  double tot = 0.0;
  for (int32_t j = 0; j < n; ++j) {
    if (q0[j] > 0.0) {
      double d = ((2.0 * perturb_uniform(seed, (uint32_t)j, i, p) - 1.0) - mean) * scale;
      q[j] = q0[j] + d;
      if (q[j] < 0.0) q[j] = 0.0;
      tot += q[j];
    } else {
      q[j] = 0.0;
    }
  }
  double ra = r0 + (zabs - mean) * scale;
  if (ra < 0.0) ra = 0.0;
  tot += ra;
  double ts = 0.0;
  for (int32_t j = 0; j < n; ++j) { q[j] /= tot; ts += q[j]; }
  ra /= tot;
  if (ra < r_min) {
    double f = (ts > 0.0) ? (1.0 - r_min) / ts : 0.0;
    for (int32_t j = 0; j < n; ++j) q[j] *= f;
    ra = r_min;
  }
  *r = ra;
}

/* Multiplicative row perturbation (Sec. 9 robust experiment): every transient entry with  */
/* q0_j > 0 becomes min(max(q0_j (1 + rel z_j), 0), 1), z_j = 2u - 1 with u from counter   */
/* (j, i, p, 1); if the transient sum exceeds 1 - r_min it is scaled to 1 - r_min; the     */
/* absorption is the remainder 1 - sum_j q_j.  (r0 is not used: absorption is implied.)    */
void orc_perturb_row_mult(int32_t n, const double *q0, uint64_t seed, uint32_t i, uint32_t p,
                          double rel, double r_min, double *q, double *r) {
  double ts = 0.0;
  for (int32_t j = 0; j < n; ++j) {
    q[j] = 0.0;
    if (q0[j] > 0.0) {
      double z = 2.0 * perturb_uniform(seed, (uint32_t)j, i, p) - 1.0;
      double v = q0[j] * (1.0 + rel * z);
      if (v < 0.0) v = 0.0;
      if (v > 1.0) v = 1.0;
      q[j] = v;
      ts += v;
    }
  }
  if (ts > 1.0 - r_min) {
    double f = (1.0 - r_min) / ts;
    ts = 0.0;
    for (int32_t j = 0; j < n; ++j) { q[j] *= f; ts += q[j]; }
  }
  *r = 1.0 - ts;
}

/* model 0: the l1 row model of orc_perturb_row (radius = l1 radius); model 1: the          */
/* multiplicative model of orc_perturb_row_mult (radius = relative radius).  kl_out[k]     */
/* (optional) = KL(b' || b0) = sum_v b'_v log(b'_v / b0_v) of perturbation p_begin + k.     */
int orc_perturb_sweep(int32_t n, const double *Q0, const double *r0, const double *s,
                      uint32_t p_begin, uint32_t p_count, double radius, double r_min,
                      uint64_t seed, int32_t top_k, int32_t K2, int32_t H, double tie_rel,
                      uint64_t *out_counts, uint64_t *pair_flips, uint64_t *shift_hist,
                      double *out_f64, double *b_out, int32_t *rank_out, int32_t model,
                      double *kl_out) {
  size_t nn = (size_t)n;
  double *Qp = (double *)malloc(sizeof(double) * nn * nn);
  double *rp = (double *)malloc(sizeof(double) * nn);
  double *mu0 = (double *)malloc(sizeof(double) * nn);
  double *b0 = (double *)malloc(sizeof(double) * nn);
  double *mu = (double *)malloc(sizeof(double) * nn);
  double *b = (double *)malloc(sizeof(double) * nn);
  double *x = (double *)malloc(sizeof(double) * nn);
  double *A = (double *)malloc(sizeof(double) * nn * nn);
  double *ones = (double *)malloc(sizeof(double) * nn);
  int32_t *rank0 = (int32_t *)malloc(sizeof(int32_t) * nn);
  int32_t *rank = (int32_t *)malloc(sizeof(int32_t) * nn);
  int32_t *byrank0 = (int32_t *)malloc(sizeof(int32_t) * nn);
  int st = ORC_OK;
  if (!Qp || !rp || !mu0 || !b0 || !mu || !b || !x || !A || !ones || !rank0 || !rank || !byrank0) {
    st = ORC_ENOMEM; goto out;
  }
  double T0 = 0.0;
  st = orc_afc_from_q(n, Q0, s, NULL, mu0, b0, &T0, NULL);
  if (st != ORC_OK) goto out;
  orc_rank(n, b0, tie_rel, rank0);
  for (int32_t v = 0; v < n; ++v) byrank0[rank0[v]] = v;
  out_counts[0] = out_counts[1] = out_counts[2] = 0;
  out_f64[0] = out_f64[1] = out_f64[2] = 0.0;
  for (int32_t a = 0; a < K2 * K2; ++a) pair_flips[a] = 0;
  for (int32_t h = 0; h < H; ++h) shift_hist[h] = 0;
  for (uint32_t k = 0; k < p_count; ++k) {
    uint32_t p = p_begin + k;
    for (int32_t i = 0; i < n; ++i) {
      if (model == 1)
        orc_perturb_row_mult(n, Q0 + (size_t)i * nn, seed, (uint32_t)i, p, radius, r_min,
                             Qp + (size_t)i * nn, rp + i);
      else
        orc_perturb_row(n, Q0 + (size_t)i * nn, r0[i], seed, (uint32_t)i, p, radius, r_min,
                        Qp + (size_t)i * nn, rp + i);
    }
    double T = 0.0;
    st = orc_afc_from_q(n, Qp, s, NULL, mu, b, &T, NULL);
    if (st != ORC_OK) goto out;
    if (kl_out) {
      double kl = 0.0;
      for (int32_t v = 0; v < n; ++v)
        if (b[v] > 0.0) kl += b[v] * log(b[v] / b0[v]);
      kl_out[k] = kl;
    }
    /* first-order prediction: x = mu0 E, then y = x N0 (solve (I - Q0)^T y^T = x^T) */
    for (int32_t j = 0; j < n; ++j) {
      double acc = 0.0;
      for (int32_t i = 0; i < n; ++i) acc += mu0[i] * (Qp[(size_t)i * nn + j] - Q0[(size_t)i * nn + j]);
      x[j] = acc;
    }
    for (int32_t i = 0; i < n; ++i)
      for (int32_t j = 0; j < n; ++j)
        A[(size_t)i * nn + j] = (i == j ? 1.0 : 0.0) - Q0[(size_t)j * nn + i];
    st = orc_gauss_solve(n, A, x, 1);
    if (st != ORC_OK) goto out;
    double y1 = 0.0;
    for (int32_t j = 0; j < n; ++j) y1 += x[j];
    double dmax = 0.0, lmax = 0.0;
    for (int32_t v = 0; v < n; ++v) {
      double lin = b0[v] + x[v] / T0 - b0[v] * y1 / T0;
      if (fabs(b[v] - b0[v]) > dmax) dmax = fabs(b[v] - b0[v]);
      if (fabs(b[v] - lin) > lmax) lmax = fabs(b[v] - lin);
    }
    if (dmax > out_f64[0]) out_f64[0] = dmax;
    if (lmax > out_f64[1]) out_f64[1] = lmax;
    /* uniform transience: max_i (N' 1)_i, solve (I - Q') t = 1 */
    for (int32_t i = 0; i < n; ++i) {
      ones[i] = 1.0;
      for (int32_t j = 0; j < n; ++j) A[(size_t)i * nn + j] = (i == j ? 1.0 : 0.0) - Qp[(size_t)i * nn + j];
    }
    st = orc_gauss_solve(n, A, ones, 1);
    if (st != ORC_OK) goto out;
    for (int32_t i = 0; i < n; ++i) if (ones[i] > out_f64[2]) out_f64[2] = ones[i];
    /* ranking statistics against the nominal ranking */
    orc_rank(n, b, tie_rel, rank);
    if (b_out) for (int32_t v = 0; v < n; ++v) b_out[(size_t)k * nn + v] = b[v];
    if (rank_out) for (int32_t v = 0; v < n; ++v) rank_out[(size_t)k * nn + v] = rank[v];
    int32_t kk = top_k < n ? top_k : n;
    int top1 = (rank[byrank0[0]] != 0);
    int set_changed = 0, order_changed = 0;
    for (int32_t a = 0; a < kk; ++a) {
      int32_t v = byrank0[a];
      if (rank[v] >= kk) set_changed = 1;
      if (rank[v] != a) order_changed = 1;
    }
    out_counts[0] += (uint64_t)top1;
    out_counts[1] += (uint64_t)set_changed;
    out_counts[2] += (uint64_t)order_changed;
    int32_t k2 = K2 < n ? K2 : n;
    for (int32_t a = 0; a < k2; ++a)
      for (int32_t c = a + 1; c < k2; ++c)
        if (rank[byrank0[a]] > rank[byrank0[c]]) pair_flips[a * K2 + c]++;
    for (int32_t a = 0; a < k2; ++a) {
      int32_t sh = abs(rank[byrank0[a]] - a);
      if (sh > H - 1) sh = H - 1;
      shift_hist[sh]++;
    }
  }
out:
  free(Qp); free(rp); free(mu0); free(b0); free(mu); free(b); free(x); free(A); free(ones);
  free(rank0); free(rank); free(byrank0);
  return st;
}
