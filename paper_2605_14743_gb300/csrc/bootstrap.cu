// bootstrap.cu -- realization-level bootstrap of the AFC vector b (Sec. 8: nonparametric
// bootstrap over resampled draws; with realization sharing every anchor's draws come from the
// same realizations, so whole realizations are resampled).
//
// One 256-thread CTA per replicate at a time (persistent over replicates, two per SM):
//   (1) weights: R draws with replacement, u = Philox4x32-10(counter (k, b, 0, 2))[0],
//       index floor(u R / 2^32), w[index] += 1
//   (2) one pass over the next-state records [R][n] of the nominal run: per anchor the
//       re-weighted absorbed count and the re-weighted counts into the observed states C
//   (3) the reduced system of the solve: A = I - Q_CC, y = s_C + s_U Q_UC with the same row
//       scale rule as the kernel assembly (exact integer counts, then one scale per row; the
//       U-row sums run per column in ascending row order, so the result is deterministic)
//   (4) FP64 LU with partial pivoting (blocked when the matrix is in the device slab),
//       A^T mu_C = y, E[T] and b for every node
// A second kernel takes, per node, the replicates at the two sorted positions of the
// percentile interval (rank by value, ties by replicate index).
#include <algorithm>
#include <cmath>
#include <cstdint>

#include <cuda_runtime.h>

#include "afc_device.cuh"
#include "afc_internal.h"
#include "linalg.cuh"

namespace afc {

namespace {

constexpr int kBootThreads = 256;
constexpr int kBootCtasPerSm = 2;

__host__ __device__ inline size_t al256(size_t x) { return (x + 255u) & ~size_t(255); }

struct BootSlab {
  size_t off_w, off_abs, off_cnt, off_a, off_y, off_piv, bytes;
};

__host__ __device__ inline BootSlab boot_slab(int32_t n, int32_t c, uint32_t R, bool a_in_smem) {
  BootSlab s{};
  const size_t cc = (size_t)(c > 0 ? c : 1);
  size_t o = 0;
  s.off_w = o;   o += al256(4ull * R);
  s.off_abs = o; o += al256(4ull * (size_t)n);
  s.off_cnt = o; o += al256(4ull * (size_t)n * cc);     // [n][c] re-weighted counts into C
  s.off_a = o;   o += a_in_smem ? 0 : al256(8ull * cc * cc);
  s.off_y = o;   o += al256(8ull * cc);
  s.off_piv = o; o += al256(4ull * cc);
  s.bytes = o;
  return s;
}

__global__ void __launch_bounds__(kBootThreads, kBootCtasPerSm)
bootstrap_kernel(ChainDev C, const int32_t *__restrict__ rec, uint32_t R, uint32_t B,
                 uint32_t k0, uint32_t k1, unsigned char *slabs, size_t slab_bytes, int a_in_smem,
                 double *b_rep, double *T_rep, uint32_t *status) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ double sval[33];
  __shared__ int32_t sidx[32];
  __shared__ double sb[2];
  __shared__ int32_t sflag[1];
  __shared__ double red[33];
  LinScratch ls{sval, sidx, sb, sflag};
  const int32_t n = C.n, c = C.c;
  const double s_unif = 1.0 / (double)n;
  unsigned char *slab = slabs + (size_t)blockIdx.x * slab_bytes;
  const BootSlab L = boot_slab(n, c, R, a_in_smem != 0);
  uint32_t *w = reinterpret_cast<uint32_t *>(slab + L.off_w);
  uint32_t *rabs = reinterpret_cast<uint32_t *>(slab + L.off_abs);
  uint32_t *cnt = reinterpret_cast<uint32_t *>(slab + L.off_cnt);
  double *A = a_in_smem ? reinterpret_cast<double *>(smem) : reinterpret_cast<double *>(slab + L.off_a);
  double *y = reinterpret_cast<double *>(slab + L.off_y);
  int32_t *piv = reinterpret_cast<int32_t *>(slab + L.off_piv);
  const size_t ncc = (size_t)n * (size_t)c;
  // row scale of the assembled kernel: (1 - alpha) / R, or where no absorption was seen the
  // transient part rescaled to 1 - eta
  auto row_scale = [&](uint32_t absorbed) {
    const double q_sum = (1.0 - C.alpha) * (double)(R - absorbed) / (double)R;
    const double r_i = C.alpha + (1.0 - C.alpha) * (double)absorbed / (double)R;
    double scale = (1.0 - C.alpha) / (double)R;
    if (r_i == 0.0 && q_sum > 0.0) scale *= (1.0 - C.eta) / q_sum;
    return scale;
  };
  for (uint32_t b = blockIdx.x; b < B; b += gridDim.x) {
    // (1) weights, cleared accumulators
    for (uint32_t r = threadIdx.x; r < R; r += blockDim.x) w[r] = 0u;
    for (int32_t i = threadIdx.x; i < n; i += blockDim.x) rabs[i] = 0u;
    for (size_t k = threadIdx.x; k < ncc; k += blockDim.x) cnt[k] = 0u;
    __syncthreads();
    for (uint32_t k = threadIdx.x; k < R; k += blockDim.x) {
      const uint4 u = philox4x32_10(make_uint4(k, b, 0u, 2u), k0, k1);
      atomicAdd(&w[(uint32_t)(((uint64_t)u.x * (uint64_t)R) >> 32)], 1u);
    }
    __syncthreads();
    // (2) one pass over the records of the drawn realizations
    for (uint32_t r = 0; r < R; ++r) {
      const uint32_t wr = w[r];
      if (wr == 0u) continue;   // uniform across the CTA
      const int32_t *row = rec + (size_t)r * (size_t)n;
      for (int32_t i = threadIdx.x; i < n; i += blockDim.x) {
        const int32_t j = row[i];
        if (j == n) {
          atomicAdd(&rabs[i], wr);
        } else {
          const int32_t pj = (j >= 0 && j < n) ? C.c_index[j] : -1;
          if (pj < 0) { atomicOr(status, kErrInput); continue; }
          atomicAdd(&cnt[(size_t)i * c + pj], wr);
        }
      }
    }
    __syncthreads();
    // (3) A = I - Q_CC and y = s_C + s_U Q_UC
    for (size_t k = threadIdx.x; k < (size_t)c * c; k += blockDim.x) {
      const int32_t pi = (int32_t)(k / c), pj = (int32_t)(k % c);
      const int32_t i = C.c_list[pi];
      A[k] = (pi == pj ? 1.0 : 0.0) - row_scale(rabs[i]) * (double)cnt[(size_t)i * c + pj];
    }
    for (int32_t pj = threadIdx.x; pj < c; pj += blockDim.x) {
      double acc = C.s ? C.s[C.c_list[pj]] : s_unif;
      for (int32_t i = 0; i < n; ++i) {
        if (C.c_index[i] >= 0) continue;
        const uint32_t k = cnt[(size_t)i * c + pj];
        if (k) acc += (C.s ? C.s[i] : s_unif) * row_scale(rabs[i]) * (double)k;
      }
      y[pj] = acc;
    }
    __syncthreads();
    // (4) solve, E[T], b
    bool ok = true;
    if (c > 0) {
      // on chip: the column-by-column LU; in the device slab: the blocked LU, its tiles in
      // the dynamic shared memory the matrix does not use
      ok = a_in_smem ? lu_factor(A, c, c, piv, ls)
                     : lu_factor_blocked(A, c, c, piv, ls, reinterpret_cast<double *>(smem));
      if (ok) lu_solve_transposed(A, c, c, piv, y, ls);
    }
    if (!ok) {
      if (threadIdx.x == 0) atomicOr(status, kErrSolve);
      continue;
    }
    double part = 0.0;
    for (int32_t v = threadIdx.x; v < n; v += blockDim.x) {
      const int32_t pv = C.c_index[v];
      part += pv >= 0 ? y[pv] : (C.s ? C.s[v] : s_unif);
    }
    const double T = block_sum(part, red);
    for (int32_t v = threadIdx.x; v < n; v += blockDim.x) {
      const int32_t pv = C.c_index[v];
      b_rep[(size_t)b * n + v] = (pv >= 0 ? y[pv] : (C.s ? C.s[v] : s_unif)) / T;
    }
    if (threadIdx.x == 0 && T_rep) T_rep[b] = T;
    __syncthreads();
  }
}

// Per node (a warp each): the replicates at sorted positions k_lo and k_hi, replicates ordered
// by value, ties by replicate index.
__global__ void quantile_kernel(int32_t n, uint32_t B, const double *b_rep, uint32_t k_lo,
                                uint32_t k_hi, double *lo, double *hi) {
  const uint32_t lane = threadIdx.x & 31u;
  const uint32_t warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const uint32_t nwarps = (gridDim.x * blockDim.x) >> 5;
  for (uint32_t v = warp; v < (uint32_t)n; v += nwarps) {
    for (uint32_t t = lane; t < B; t += 32u) {
      const double x = b_rep[(size_t)t * n + v];
      uint32_t rank = 0;
      for (uint32_t u = 0; u < B; ++u) {
        const double xu = b_rep[(size_t)u * n + v];
        rank += (xu < x || (xu == x && u < t)) ? 1u : 0u;
      }
      if (rank == k_lo) lo[v] = x;
      if (rank == k_hi) hi[v] = x;
    }
  }
}

}  // namespace

size_t bootstrap_slab_bytes(int32_t n, int32_t c, uint32_t R) {
  return boot_slab(n, c, R, false).bytes;
}

cudaError_t launch_bootstrap(const ChainDev &C, const int32_t *rec, uint32_t R, uint32_t B,
                             uint64_t seed, double level, double *b_rep, double *T_rep,
                             double *lo, double *hi, unsigned char *slabs, size_t slab_space,
                             uint32_t *status, int num_sms, cudaStream_t stream) {
  const int32_t n = C.n, c = C.c;
  int max_optin = 0, dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&max_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  const size_t a_bytes = 8ull * (size_t)std::max(c, 1) * (size_t)std::max(c, 1);
  // A on chip when two CTAs per SM still fit (the LU's rank-1 updates then stay in shared memory)
  const bool a_smem = a_bytes + 16 * 1024 <= (size_t)max_optin / 2;
  const size_t slab = boot_slab(n, c, R, a_smem).bytes;
  size_t grid = slab_space / std::max<size_t>(slab, 1);
  grid = std::min<size_t>({grid, (size_t)B, (size_t)num_sms * kBootCtasPerSm});
  if (grid == 0) return cudaErrorMemoryAllocation;
  const uint32_t dyn = a_smem ? (uint32_t)a_bytes
                              : (uint32_t)(sizeof(double) * lu_blocked_smem_doubles());
  cudaFuncSetAttribute(bootstrap_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, dyn);
  bootstrap_kernel<<<(unsigned)grid, kBootThreads, dyn, stream>>>(
      C, rec, R, B, (uint32_t)seed, (uint32_t)(seed >> 32), slabs, slab, a_smem ? 1 : 0, b_rep,
      T_rep, status);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess || !lo || !hi) return e;
  const double q = (1.0 - level) / 2.0;
  const uint32_t k_lo = (uint32_t)std::floor(q * (double)(B - 1));
  const uint32_t k_hi = (uint32_t)std::ceil((1.0 - q) * (double)(B - 1));
  const int qgrid = (int)std::min<int64_t>(((int64_t)n + 7) / 8, 1024);
  quantile_kernel<<<qgrid, 256, 0, stream>>>(n, B, b_rep, k_lo, k_hi, lo, hi);
  return cudaGetLastError();
}

}  // namespace afc
