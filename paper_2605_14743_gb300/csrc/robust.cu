// robust.cu -- host side of the sampled robust search (Sec. 9 robust sensitivity experiment):
// the Wasserstein-1 distance between two node distributions under the base graph's hop metric.
//
// W1 on a graph metric is an uncapacitated transshipment problem on the graph itself (each
// unit of mass moved across an edge costs 1).  It is solved exactly by successive shortest
// paths: node potentials keep the reduced arc costs non-negative, each round runs a
// multi-source Dijkstra from every node with excess mass and stops at the first node with a
// deficit, then pushes as much as the path allows (the source's excess, the sink's deficit,
// the flow on any arc the path cancels).  Costs are integers, so distances and potentials are
// exact; the masses are doubles and are settled to within a relative 1e-14.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <functional>
#include <limits>
#include <queue>
#include <utility>
#include <vector>

#include "afc_internal.h"

namespace afc {

double w1_graph_host(int32_t n, const int32_t *rp, const int32_t *col, const int32_t *eid,
                     const double *x, const double *y) {
  const int32_t arcs = rp[n];
  // partner arc of every arc (the other direction of the same edge)
  std::vector<int32_t> first(std::max<int32_t>(arcs, 1), -1), rev(std::max<int32_t>(arcs, 1), -1);
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
