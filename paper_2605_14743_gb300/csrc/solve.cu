// solve.cu -- A8 on the GPU: kernel assembly from the transition counts and the reduced
// FP64 absorbing-chain solve on the observed centre states C (Sec. 4 eqs. fundamental,
// visits, expected-length, afc-def; Sec. 6.4 eq. mr-inner-product; Sec. 8.2 floor), plus the
// visit-gap certificates of Sec. 5.5 (eqs. pm-gap, sharp-gap).
//
// With the columns of U = V \ C zero, N = (I - Q)^-1 has the block form [[I, Q_UC N_CC],
// [0, N_CC]] in (U, C) order, so mu_U = s_U and mu_C (I - Q_CC) = s_C + s_U Q_UC.
#include <algorithm>
#include <cstdint>
#include <cuda_runtime.h>

#include "afc_internal.h"
#include "linalg.cuh"

namespace afc {

// ---- observed states --------------------------------------------------------------------
__global__ void column_flags_kernel(int32_t n, const uint32_t *counts, uint32_t *flags) {
  const int32_t j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  const size_t stride = (size_t)n + 1;
  uint32_t any = 0;
  for (int32_t i = blockIdx.y; i < n; i += gridDim.y) any |= counts[(size_t)i * stride + j];
  if (any) flags[j] = 1u;
}

__global__ void compact_states_kernel(int32_t n, const uint32_t *flags, int32_t *c_index,
                                      int32_t *c_list, int32_t *c_out) {
  __shared__ int32_t warp_tot[32];
  __shared__ int32_t base;
  if (threadIdx.x == 0) base = 0;
  __syncthreads();
  const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
  for (int32_t start = 0; start < n; start += blockDim.x) {
    const int32_t j = start + threadIdx.x;
    const bool f = j < n && flags[j];
    const uint32_t ball = __ballot_sync(0xFFFFFFFFu, f);
    if (lane == 0) warp_tot[warp] = __popc(ball);
    __syncthreads();
    int32_t off = 0;
    for (uint32_t w = 0; w < warp; ++w) off += warp_tot[w];
    const int32_t pos = base + off + __popc(ball & ((1u << lane) - 1u));
    if (j < n) {
      c_index[j] = f ? pos : -1;
      if (f) c_list[pos] = j;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      int32_t t = 0;
      for (uint32_t w = 0; w < (blockDim.x + 31u) / 32u; ++w) t += warp_tot[w];
      base += t;
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) *c_out = base;
}

cudaError_t launch_observed_states(int32_t n, const uint32_t *counts, int32_t *c_index,
                                   int32_t *c_list, int32_t *c_dev, cudaStream_t stream) {
  // c_list first holds the column flags; the in-order compaction then overwrites its prefix
  // [0, |C|) (a chunk's flags are read before any of that chunk's writes, and every write
  // position is at most the flag position it comes from).
  uint32_t *flags = reinterpret_cast<uint32_t *>(c_list);
  cudaMemsetAsync(flags, 0, sizeof(uint32_t) * (size_t)n, stream);
  dim3 grid((n + 255) / 256, (unsigned)min(n, 64));
  column_flags_kernel<<<grid, 256, 0, stream>>>(n, counts, flags);
  compact_states_kernel<<<1, 1024, 0, stream>>>(n, flags, c_index, c_list, c_dev);
  return cudaGetLastError();
}

// ---- workspace ----------------------------------------------------------------------------
SolveWs solve_ws_layout(int32_t n, int32_t c, size_t nnz_cap, uint32_t perturb_slabs,
                        size_t slab_bytes, size_t csc_cap) {
  auto al = [](size_t x) { return (x + 255) & ~size_t(255); };
  SolveWs L{};
  size_t o = 0;
  const size_t cc = (size_t)(c > 0 ? c : 1);
  L.off_y = o;        o = al(o + 8 * cc);
  L.off_t = o;        o = al(o + 8 * cc);
  L.off_rowscale = o; o = al(o + 8 * 2 * (size_t)n);         // per row: scale, r_i
  L.off_nzptr = o;    o = al(o + 4 * ((size_t)n + 1));
  L.off_nzcol = o;    o = al(o + 4 * nnz_cap);
  L.off_nzval = o;    o = al(o + 8 * nnz_cap);
  L.off_flags = o;    o = al(o + 4 * (size_t)n + 64);
  L.off_tmp = o;      o = al(o + 8 * (4 * (size_t)n + 4 * cc + 64));
  L.off_csc = o;      o = al(o + (csc_cap ? 4 * ((cc + 1 + 63) & ~size_t(63)) + 8 * csc_cap : 0));
  L.csc_cap = csc_cap;
  L.off_slab = o;     o = al(o + (size_t)perturb_slabs * slab_bytes);
  L.total = o;
  L.nnz_cap = nnz_cap;
  return L;
}

// ---- kernel assembly ---------------------------------------------------------------------
// Per row i: transient count sum, the scale that maps counts to Q, r_i, and the row's
// nonzero count (transient columns plus the absorbing column, always present).
__global__ void row_prep_kernel(ChainDev C, double *rowscale, int32_t *nnz_row) {
  const int32_t n = C.n;
  const size_t stride = (size_t)n + 1;
  const uint32_t warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31u;
  const uint32_t nwarps = (gridDim.x * blockDim.x) >> 5;
  for (int32_t i = warp; i < n; i += nwarps) {
    const uint32_t *row = C.counts + (size_t)i * stride;
    unsigned long long tsum = 0;
    int32_t nz = 0;
    for (int32_t j = lane; j < n; j += 32) {
      const uint32_t v = row[j];
      tsum += v;
      nz += v ? 1 : 0;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      tsum += __shfl_down_sync(0xFFFFFFFFu, tsum, o);
      nz += __shfl_down_sync(0xFFFFFFFFu, nz, o);
    }
    if (lane == 0) {
      double scale = (1.0 - C.alpha) / (double)C.R;
      double r = C.alpha + (1.0 - C.alpha) * (double)row[n] / (double)C.R;
      if (r == 0.0) {
        // floor: r_i = eta, transient part rescaled to 1 - eta
        const double qsum = (1.0 - C.alpha) * (double)tsum / (double)C.R;
        r = C.eta;
        if (qsum > 0.0) scale *= (1.0 - C.eta) / qsum;
      }
      rowscale[2 * i] = scale;
      rowscale[2 * i + 1] = r;
      nnz_row[i] = nz + 1;
    }
  }
}

__global__ void exclusive_scan_kernel(int32_t n, const int32_t *in, int32_t *out) {
  __shared__ int32_t warp_tot[32];
  __shared__ int32_t base;
  if (threadIdx.x == 0) base = 0;
  __syncthreads();
  const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
  for (int32_t start = 0; start < n; start += blockDim.x) {
    const int32_t i = start + threadIdx.x;
    const int32_t x = i < n ? in[i] : 0;
    int32_t inc = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int32_t y = __shfl_up_sync(0xFFFFFFFFu, inc, o);
      if ((int)lane >= o) inc += y;
    }
    if (lane == 31) warp_tot[warp] = inc;
    __syncthreads();
    int32_t off = base;
    for (uint32_t w = 0; w < warp; ++w) off += warp_tot[w];
    if (i < n) out[i] = off + inc - x;
    __syncthreads();
    if (threadIdx.x == 0) {
      int32_t t = 0;
      for (uint32_t w = 0; w < (blockDim.x + 31u) / 32u; ++w) t += warp_tot[w];
      base += t;
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) out[n] = base;
}

// Writes the sparse rows (C positions ascending, then the absorbing column as position c)
// and scatters A = I - Q_CC and y = s_C + s_U Q_UC.
__global__ void row_fill_kernel(ChainDev C, const double *rowscale, const int32_t *nzptr,
                                int32_t *nzcol, double *nzval, double *A, double *y) {
  const int32_t n = C.n, c = C.c;
  const size_t stride = (size_t)n + 1;
  const uint32_t warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31u;
  const uint32_t nwarps = (gridDim.x * blockDim.x) >> 5;
  for (int32_t i = warp; i < n; i += nwarps) {
    const uint32_t *row = C.counts + (size_t)i * stride;
    const double scale = rowscale[2 * i], r = rowscale[2 * i + 1];
    const double si = C.s ? C.s[i] : 1.0 / (double)n;
    const int32_t pi = C.c_index[i];
    int32_t out = nzptr[i];
    for (int32_t j0 = 0; j0 < n; j0 += 32) {
      const int32_t j = j0 + lane;
      const uint32_t v = j < n ? row[j] : 0u;
      const uint32_t ball = __ballot_sync(0xFFFFFFFFu, v != 0);
      if (v) {
        const int32_t pos = out + __popc(ball & ((1u << lane) - 1u));
        const int32_t pj = C.c_index[j];
        const double q = scale * (double)v;
        nzcol[pos] = pj;
        nzval[pos] = q;
        if (pi >= 0) A[(size_t)pi * c + pj] -= q;  // distinct (pi, pj) per lane: no race
        else atomicAdd(&y[pj], si * q);
      }
      out += __popc(ball);
    }
    if (lane == 0) {
      nzcol[out] = c;  // absorbing column
      nzval[out] = r;
      if (pi >= 0) atomicAdd(&y[pi], si);
    }
  }
}

__global__ void identity_kernel(double *A, int32_t c) {
  const size_t total = (size_t)c * c;
  for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < total;
       k += (size_t)gridDim.x * blockDim.x)
    A[k] = (k / c == k % c) ? 1.0 : 0.0;
}

// ---- factor + solves + finalise (one CTA) -----------------------------------------------------
__global__ void __launch_bounds__(1024, 1)
chain_solve_kernel(ChainDev C, double *A, int32_t *piv, double *y, double *t,
                   const double *rowscale, const int32_t *nzptr, const int32_t *nzcol,
                   const double *nzval, double *mu, double *b, double *scalars,
                   uint32_t *status) {
  __shared__ double sval[33];
  __shared__ int32_t sidx[32];
  __shared__ double sb[2];
  __shared__ int32_t sflag[1];
  __shared__ double red[33];
  LinScratch ls{sval, sidx, sb, sflag};
  const int32_t n = C.n, c = C.c;
  bool ok = true;
  if (c > 0) {
    ok = lu_factor(A, c, c, piv, ls);
    if (ok) {
      lu_solve_transposed(A, c, c, piv, y, ls);                  // mu_C
      for (int32_t k = threadIdx.x; k < c; k += blockDim.x) t[k] = 1.0;
      __syncthreads();
      lu_solve(A, c, c, piv, t, ls);                             // (N 1) on C
    }
  }
  if (!ok) {
    if (threadIdx.x == 0) *status |= kErrSolve;
    return;
  }
  // mu, E[T], b, b_f; max (N 1) including the U rows: 1 + sum_j Q_ij (N 1)_j
  double part = 0.0, tmax = 0.0;
  for (int32_t i = threadIdx.x; i < n; i += blockDim.x) {
    const int32_t pi = C.c_index[i];
    const double m = pi >= 0 ? y[pi] : (C.s ? C.s[i] : 1.0 / (double)n);
    mu[i] = m;
    part += m;
    double ti;
    if (pi >= 0) {
      ti = t[pi];
    } else {
      ti = 1.0;
      for (int32_t e = nzptr[i]; e < nzptr[i + 1]; ++e)
        if (nzcol[e] < c) ti += nzval[e] * t[nzcol[e]];
    }
    tmax = fmax(tmax, ti);
  }
  const double T = block_sum(part, red);
  tmax = block_max(tmax, red);
  double bf = 0.0;
  for (int32_t i = threadIdx.x; i < n; i += blockDim.x) {
    const double bi = mu[i] / T;
    b[i] = bi;
    if (C.f) bf += bi * C.f[i];
  }
  bf = block_sum(bf, red);
  if (threadIdx.x == 0) {
    scalars[0] = T;
    scalars[1] = C.f ? bf : 0.0;
    scalars[2] = tmax;
    scalars[3] = (double)c;
  }
  (void)rowscale;
}

cudaError_t launch_solve(const ChainDev &C, double *mu, double *b, double *scalars, double *lu,
                         int32_t *piv, unsigned char *ws, const SolveWs &L, uint32_t *status_dev,
                         cudaStream_t stream) {
  const int32_t n = C.n, c = C.c;
  double *y = reinterpret_cast<double *>(ws + L.off_y);
  double *t = reinterpret_cast<double *>(ws + L.off_t);
  double *rowscale = reinterpret_cast<double *>(ws + L.off_rowscale);
  int32_t *nzptr = reinterpret_cast<int32_t *>(ws + L.off_nzptr);
  int32_t *nzcol = reinterpret_cast<int32_t *>(ws + L.off_nzcol);
  double *nzval = reinterpret_cast<double *>(ws + L.off_nzval);
  int32_t *nnz_row = reinterpret_cast<int32_t *>(ws + L.off_flags);
  const int64_t want_blocks = ((int64_t)n * 32 + 255) / 256;
  const int blocks = (int)(want_blocks < 2048 ? want_blocks : 2048);
  const int64_t want_id = ((int64_t)c * c + 255) / 256;
  const int id_blocks = (int)(want_id < 4096 ? want_id : 4096);
  row_prep_kernel<<<blocks, 256, 0, stream>>>(C, rowscale, nnz_row);
  exclusive_scan_kernel<<<1, 1024, 0, stream>>>(n, nnz_row, nzptr);
  if (c > 0) identity_kernel<<<id_blocks, 256, 0, stream>>>(lu, c);
  cudaMemsetAsync(y, 0, sizeof(double) * (size_t)(c > 0 ? c : 1), stream);
  row_fill_kernel<<<blocks, 256, 0, stream>>>(C, rowscale, nzptr, nzcol, nzval, lu, y);
  chain_solve_kernel<<<1, 1024, 0, stream>>>(C, lu, piv, y, t, rowscale, nzptr, nzcol, nzval, mu,
                                             b, scalars, status_dev);
  return cudaGetLastError();
}

// ---- certificates (one CTA per pair) ---------------------------------------------------------
__global__ void __launch_bounds__(512)
certificates_kernel(ChainDev C, const double *mu0, const double *lu0, const int32_t *piv0,
                    double scale, int32_t npairs, const int32_t *pu, const int32_t *pv,
                    double *gap, double *sharp, const int32_t *nzptr, const int32_t *nzcol,
                    const double *nzval, double *tmp) {
  __shared__ double sval[33];
  __shared__ int32_t sidx[32];
  __shared__ double sb[2];
  __shared__ int32_t sflag[1];
  __shared__ double red[33];
  LinScratch ls{sval, sidx, sb, sflag};
  const int32_t n = C.n, c = C.c;
  for (int32_t k = blockIdx.x; k < npairs; k += gridDim.x) {
    const int32_t u = pu[k], v = pv[k];
    double *x = tmp + (size_t)blockIdx.x * (c > 0 ? c : 1);
    // x_C solves (I - Q_CC) x_C = (e_u - e_v)_C; x_U = (e_u - e_v)_U + Q_UC x_C
    for (int32_t j = threadIdx.x; j < c; j += blockDim.x) x[j] = 0.0;
    __syncthreads();
    if (threadIdx.x == 0) {
      if (u >= 0 && u < n && C.c_index[u] >= 0) x[C.c_index[u]] += 1.0;
      if (v >= 0 && v < n && C.c_index[v] >= 0) x[C.c_index[v]] -= 1.0;
    }
    __syncthreads();
    if (c > 0) lu_solve(lu0, c, c, piv0, x, ls);
    double mx = 0.0;
    for (int32_t i = threadIdx.x; i < n; i += blockDim.x) {
      const int32_t pi = C.c_index[i];
      double xi;
      if (pi >= 0) {
        xi = x[pi];
      } else {
        xi = (i == u ? 1.0 : 0.0) - (i == v ? 1.0 : 0.0);
        for (int32_t e = nzptr[i]; e < nzptr[i + 1]; ++e)
          if (nzcol[e] < c) xi += nzval[e] * x[nzcol[e]];
      }
      mx = fmax(mx, fabs(xi));
    }
    mx = block_max(mx, red);
    if (threadIdx.x == 0) {
      gap[k] = mu0[u] - mu0[v];
      sharp[k] = scale * mx;
    }
    __syncthreads();
  }
}

// Reward-AFC of the Top-k and switching rewards (warp per count row, partial sums added to
// out with atomics): out[0] += b_i (1 - alpha) psi_sum_i / R, out[1] += b_i sum_{j != i} Q_ij.
__global__ void reward_afc_kernel(int32_t n, uint32_t R, double alpha, double eta,
                                  const uint32_t *counts, const double *b, const double *psi_sum,
                                  double *out) {
  __shared__ double red0[33], red1[33];
  const uint32_t lane = threadIdx.x & 31u;
  const uint32_t warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const uint32_t nwarps = (gridDim.x * blockDim.x) >> 5;
  const size_t stride = (size_t)n + 1;
  double p0 = 0.0, p1 = 0.0;
  for (uint32_t i = warp; i < (uint32_t)n; i += nwarps) {
    const uint32_t *row = counts + (size_t)i * stride;
    unsigned long long all = 0, self = 0;
    for (uint32_t j = lane; j < (uint32_t)n; j += 32u) {
      const uint32_t c = row[j];
      all += c;
      if (j == i) self = c;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      all += __shfl_xor_sync(0xFFFFFFFFu, all, o);
      self += __shfl_xor_sync(0xFFFFFFFFu, self, o);
    }
    if (lane == 0) {
      const double q_sum = (1.0 - alpha) * (double)all / (double)R;
      const double r_i = alpha + (1.0 - alpha) * (double)row[n] / (double)R;
      const double scale = (r_i == 0.0 && q_sum > 0.0) ? (1.0 - eta) / q_sum : 1.0;
      p1 += b[i] * (1.0 - alpha) * (double)(all - self) / (double)R * scale;
      if (psi_sum) p0 += b[i] * (1.0 - alpha) * psi_sum[i] / (double)R;
    }
  }
  const double s0 = block_sum(p0, red0);
  const double s1 = block_sum(p1, red1);
  if (threadIdx.x == 0) {
    atomicAdd(&out[0], s0);
    atomicAdd(&out[1], s1);
  }
}

cudaError_t launch_reward_afc(int32_t n, uint32_t R, double alpha, double eta,
                              const uint32_t *counts, const double *b, const double *psi_sum,
                              double *out, cudaStream_t stream) {
  cudaError_t e = cudaMemsetAsync(out, 0, 2 * sizeof(double), stream);
  if (e != cudaSuccess) return e;
  const int grid = (int)std::min<int64_t>(((int64_t)n + 7) / 8, 1024);
  reward_afc_kernel<<<grid, 256, 0, stream>>>(n, R, alpha, eta, counts, b, psi_sum, out);
  return cudaGetLastError();
}

cudaError_t launch_certificates(const ChainDev &C, const double *mu0, const double *lu0,
                                const int32_t *piv0, double eps_bar, double r_min, int32_t npairs,
                                const int32_t *pu, const int32_t *pv, double *gap, double *sharp,
                                unsigned char *ws, const SolveWs &L, cudaStream_t stream) {
  if (npairs <= 0) return cudaSuccess;
  const int32_t *nzptr = reinterpret_cast<const int32_t *>(ws + L.off_nzptr);
  const int32_t *nzcol = reinterpret_cast<const int32_t *>(ws + L.off_nzcol);
  const double *nzval = reinterpret_cast<const double *>(ws + L.off_nzval);
  double *tmp = reinterpret_cast<double *>(ws + L.off_slab);
  const int grid = min(npairs, 64);
  certificates_kernel<<<grid, 512, 0, stream>>>(C, mu0, lu0, piv0, eps_bar / r_min, npairs, pu, pv,
                                                gap, sharp, nzptr, nzcol, nzval, tmp);
  return cudaGetLastError();
}

}  // namespace afc
