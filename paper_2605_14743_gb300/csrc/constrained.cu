// constrained.cu -- summaries of the set-constrained kernels (Sec. 7) and the 3-clique target
// pools of the structure-constrained experiment (Sec. 9).
//
//   feasibility_kernel  xi_i = sum_{j in W} P^W_ij (Sec. 7.1 eq. settopk-xi) on the kernel the
//                       solve assembles from the counts: the row's transient mass times the
//                       share of its non-absorbed draws that reached W directly (warp per row)
//   pool_kernel         m_W = sum_{v in W} b_v (Sec. 7.2 eq. settopk-bPsi), the within-pool
//                       profile, c_fb = sum_{u not in V_fb} b_u and the censored profile
//                       (Sec. 7.4); one CTA, fixed-order reductions
//   clique_pool         host: every triangle of the base graph, scored by its base degree sum,
//                       the S best (ties by the ascending node triple), their union and v_fb
#include <algorithm>
#include <cstdint>
#include <vector>

#include <cuda_runtime.h>

#include "afc_internal.h"
#include "linalg.cuh"

namespace afc {

namespace {

__global__ void feasibility_kernel(int32_t n, uint32_t R, double alpha, double eta,
                                   const uint32_t *counts, const uint32_t *fb_count, double *xi) {
  const uint32_t lane = threadIdx.x & 31u;
  const uint32_t warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const uint32_t nwarps = (gridDim.x * blockDim.x) >> 5;
  const size_t stride = (size_t)n + 1;
  for (uint32_t i = warp; i < (uint32_t)n; i += nwarps) {
    const uint32_t *row = counts + (size_t)i * stride;
    unsigned long long all = 0;
    for (uint32_t j = lane; j < (uint32_t)n; j += 32u) all += row[j];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) all += __shfl_xor_sync(0xFFFFFFFFu, all, o);
    if (lane == 0) {
      // the row scale of the assembled kernel: (1 - alpha) / R, and where no absorption was
      // observed (r_i = 0) the transient part rescaled to 1 - eta
      const double q_sum = (1.0 - alpha) * (double)all / (double)R;
      const double r_i = alpha + (1.0 - alpha) * (double)row[n] / (double)R;
      const double scale = (r_i == 0.0 && q_sum > 0.0) ? (1.0 - eta) / q_sum : 1.0;
      const unsigned long long fb = fb_count ? fb_count[i] : 0u;
      const unsigned long long direct = all >= fb ? all - fb : 0ull;
      xi[i] = (1.0 - alpha) * (double)direct / (double)R * scale;
    }
  }
}

__global__ void __launch_bounds__(1024) pool_kernel(int32_t n, const double *b,
                                                    const uint8_t *in_w, const uint8_t *fb_set,
                                                    double *b_pool, double *b_censored,
                                                    double *mass) {
  __shared__ double red[33];
  double pw = 0.0, pc = 0.0;
  for (int32_t v = threadIdx.x; v < n; v += blockDim.x) {
    if (in_w[v]) pw += b[v];
    if (!(fb_set && fb_set[v])) pc += b[v];
  }
  const double m_w = block_sum(pw, red);
  const double c_fb = block_sum(pc, red);
  for (int32_t v = threadIdx.x; v < n; v += blockDim.x) {
    if (b_pool) b_pool[v] = (m_w > 0.0 && in_w[v]) ? b[v] / m_w : 0.0;
    if (b_censored) b_censored[v] = (c_fb > 0.0 && !(fb_set && fb_set[v])) ? b[v] / c_fb : 0.0;
  }
  if (threadIdx.x == 0) {
    mass[0] = m_w;
    mass[1] = c_fb;
  }
}

}  // namespace

cudaError_t launch_feasibility(int32_t n, uint32_t R, double alpha, double eta,
                               const uint32_t *counts, const uint32_t *fb_count, double *xi,
                               cudaStream_t stream) {
  const int grid = (int)std::min<int64_t>(((int64_t)n + 7) / 8, 1024);
  feasibility_kernel<<<grid, 256, 0, stream>>>(n, R, alpha, eta, counts, fb_count, xi);
  return cudaGetLastError();
}

cudaError_t launch_pool_summaries(int32_t n, const double *b, const uint8_t *in_w,
                                  const uint8_t *fb_set, double *b_pool, double *b_censored,
                                  double *mass, cudaStream_t stream) {
  pool_kernel<<<1, 1024, 0, stream>>>(n, b, in_w, fb_set, b_pool, b_censored, mass);
  return cudaGetLastError();
}

// Triangles u < v < w of a graph given as sorted adjacency rows; kept: the S with the largest
// base degree sum, ties by (u, v, w) ascending.
void clique_pool_host(int32_t n, const int32_t *row_ptr, const int32_t *col, int32_t S,
                      std::vector<int32_t> &out) {
  struct Tri { int64_t score; int32_t u, v, w; };
  std::vector<Tri> tri;
  for (int32_t u = 0; u < n; ++u)
    for (int32_t a = row_ptr[u]; a < row_ptr[u + 1]; ++a) {
      const int32_t v = col[a];
      if (v <= u) continue;
      // common neighbours w > v of u and v: merge of the two sorted rows
      int32_t x = row_ptr[u], y = row_ptr[v];
      while (x < row_ptr[u + 1] && y < row_ptr[v + 1]) {
        if (col[x] < col[y]) { ++x; continue; }
        if (col[y] < col[x]) { ++y; continue; }
        const int32_t w = col[x];
        if (w > v) {
          const int64_t sc = (int64_t)(row_ptr[u + 1] - row_ptr[u]) + (row_ptr[v + 1] - row_ptr[v]) +
                             (row_ptr[w + 1] - row_ptr[w]);
          tri.push_back({sc, u, v, w});
        }
        ++x; ++y;
      }
    }
  const size_t keep = std::min<size_t>(tri.size(), (size_t)std::max(0, S));
  auto better = [](const Tri &a, const Tri &b) {
    if (a.score != b.score) return a.score > b.score;
    if (a.u != b.u) return a.u < b.u;
    if (a.v != b.v) return a.v < b.v;
    return a.w < b.w;
  };
  std::partial_sort(tri.begin(), tri.begin() + keep, tri.end(), better);
  out.clear();
  for (size_t k = 0; k < keep; ++k) {
    out.push_back(tri[k].u);
    out.push_back(tri[k].v);
    out.push_back(tri[k].w);
  }
}

}  // namespace afc
