// linalg.cuh -- CTA-cooperative FP64 dense LU with partial pivoting and triangular solves.
// The matrix may live in shared memory or global memory (generic pointers); all threads of
// the CTA must call these functions together.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace afc {

struct LinScratch {
  double *val;   // [32]
  int32_t *idx;  // [32]
  double *bcast; // [2]
  int32_t *flag; // [1]
};

// argmax |x| over rows [k, c) of column k, ties to the smallest row
__device__ __forceinline__ int32_t pivot_search(const double *A, int32_t c, int32_t lda, int32_t k,
                                                LinScratch s) {
  double best = -1.0;
  int32_t bi = k;
  for (int32_t i = k + (int32_t)threadIdx.x; i < c; i += blockDim.x) {
    const double a = fabs(A[(size_t)i * lda + k]);
    if (a > best) { best = a; bi = i; }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const double ob = __shfl_down_sync(0xFFFFFFFFu, best, o);
    const int32_t oi = __shfl_down_sync(0xFFFFFFFFu, bi, o);
    if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
  }
  const uint32_t warp = threadIdx.x >> 5, lane = threadIdx.x & 31u;
  if (lane == 0) { s.val[warp] = best; s.idx[warp] = bi; }
  __syncthreads();
  if (warp == 0) {
    const uint32_t nw = (blockDim.x + 31u) >> 5;
    best = lane < nw ? s.val[lane] : -1.0;
    bi = lane < nw ? s.idx[lane] : 0x7FFFFFFF;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const double ob = __shfl_down_sync(0xFFFFFFFFu, best, o);
      const int32_t oi = __shfl_down_sync(0xFFFFFFFFu, bi, o);
      if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
    }
    if (lane == 0) { s.idx[0] = bi; s.val[0] = best; }
  }
  __syncthreads();
  const int32_t p = s.idx[0];
  const double pv = s.val[0];
  __syncthreads();
  return pv > 0.0 ? p : -1;
}

// In-place PA = LU (unit lower L below the diagonal, U on and above).  piv[k] = row swapped
// with row k at step k.  Returns false if a pivot column is exactly zero.
__device__ inline bool lu_factor(double *A, int32_t c, int32_t lda, int32_t *piv, LinScratch s) {
  const uint32_t warp = threadIdx.x >> 5, lane = threadIdx.x & 31u;
  const uint32_t nw = blockDim.x >> 5;
  for (int32_t k = 0; k < c; ++k) {
    const int32_t p = pivot_search(A, c, lda, k, s);
    if (p < 0) return false;
    if (threadIdx.x == 0) piv[k] = p;
    if (p != k) {
      for (int32_t j = threadIdx.x; j < c; j += blockDim.x) {
        const double t = A[(size_t)k * lda + j];
        A[(size_t)k * lda + j] = A[(size_t)p * lda + j];
        A[(size_t)p * lda + j] = t;
      }
      __syncthreads();
    }
    const double inv = 1.0 / A[(size_t)k * lda + k];
    for (int32_t i = k + 1 + threadIdx.x; i < c; i += blockDim.x) A[(size_t)i * lda + k] *= inv;
    __syncthreads();
    for (int32_t i = k + 1 + warp; i < c; i += nw) {
      const double l = A[(size_t)i * lda + k];
      if (l == 0.0) continue;
      for (int32_t j = k + 1 + lane; j < c; j += 32)
        A[(size_t)i * lda + j] = fma(-l, A[(size_t)k * lda + j], A[(size_t)i * lda + j]);
    }
    __syncthreads();
  }
  return true;
}

// Blocked right-looking form of lu_factor for matrices in device memory (same factors, same
// pivot rule, same piv format): a panel of kLuB columns is factored with full-row swaps and
// rank-1 updates inside the panel, then U12 = L11^-1 A12 by forward substitution (a column
// per thread), then the trailing matrix takes A22 -= L21 U12 in 64 x 64 tiles staged through
// shared memory (each thread a 4 x 4 register tile).  The trailing matrix is read and written
// once per panel instead of once per column, which is what bounds lu_factor on large c.
// Needs blockDim.x == 256 and lu_blocked_smem_doubles() doubles of shared memory at tile.
constexpr int kLuB = 32;
constexpr int kLuT = 64;
__host__ __device__ constexpr int lu_blocked_smem_doubles() { return kLuT * (kLuB + 1) + kLuB * (kLuT + 1); }

__device__ inline bool lu_factor_blocked(double *A, int32_t c, int32_t lda, int32_t *piv,
                                         LinScratch s, double *tile) {
  if (blockDim.x != 256u) return lu_factor(A, c, lda, piv, s);   // the tile mapping needs 256
  const uint32_t tid = threadIdx.x;
  double *Lt = tile;                          // [kLuT][kLuB + 1]
  double *Ut = tile + kLuT * (kLuB + 1);      // [kLuB][kLuT + 1]
  for (int32_t kb = 0; kb < c; kb += kLuB) {
    const int32_t nb = min(kLuB, c - kb), ke = kb + nb;
    // (1) panel: columns kb .. ke-1, rows kb .. c-1
    for (int32_t k = kb; k < ke; ++k) {
      const int32_t p = pivot_search(A, c, lda, k, s);
      if (p < 0) return false;
      if (tid == 0) piv[k] = p;
      if (p != k) {
        for (int32_t j = tid; j < c; j += blockDim.x) {
          const double t = A[(size_t)k * lda + j];
          A[(size_t)k * lda + j] = A[(size_t)p * lda + j];
          A[(size_t)p * lda + j] = t;
        }
        __syncthreads();
      }
      const double inv = 1.0 / A[(size_t)k * lda + k];
      for (int32_t i = k + 1 + tid; i < c; i += blockDim.x) A[(size_t)i * lda + k] *= inv;
      __syncthreads();
      const int32_t w = ke - (k + 1);         // panel columns right of k
      if (w > 0) {
        const int64_t tot = (int64_t)(c - (k + 1)) * w;
        for (int64_t q = tid; q < tot; q += blockDim.x) {
          const int32_t i = k + 1 + (int32_t)(q / w), j = k + 1 + (int32_t)(q % w);
          A[(size_t)i * lda + j] = fma(-A[(size_t)i * lda + k], A[(size_t)k * lda + j], A[(size_t)i * lda + j]);
        }
      }
      __syncthreads();
    }
    if (ke >= c) break;
    // (2) U12 = L11^-1 A12 (L11 unit lower), a column per thread
    for (int32_t j = ke + tid; j < c; j += blockDim.x)
      for (int32_t r = 1; r < nb; ++r) {
        double acc = A[(size_t)(kb + r) * lda + j];
        for (int32_t t = 0; t < r; ++t)
          acc = fma(-A[(size_t)(kb + r) * lda + kb + t], A[(size_t)(kb + t) * lda + j], acc);
        A[(size_t)(kb + r) * lda + j] = acc;
      }
    __syncthreads();
    // (3) A22 -= L21 U12 in kLuT x kLuT tiles
    const uint32_t ty = tid / 16u, tx = tid % 16u;
    for (int32_t i0 = ke; i0 < c; i0 += kLuT)
      for (int32_t j0 = ke; j0 < c; j0 += kLuT) {
        for (uint32_t q = tid; q < (uint32_t)(kLuT * kLuB); q += blockDim.x) {
          const int32_t r = (int32_t)(q / kLuB), t = (int32_t)(q % kLuB);
          Lt[r * (kLuB + 1) + t] = (i0 + r < c && t < nb) ? A[(size_t)(i0 + r) * lda + kb + t] : 0.0;
          const int32_t t2 = (int32_t)(q / kLuT), col = (int32_t)(q % kLuT);
          Ut[t2 * (kLuT + 1) + col] = (j0 + col < c && t2 < nb) ? A[(size_t)(kb + t2) * lda + j0 + col] : 0.0;
        }
        __syncthreads();
        double acc[4][4];
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
          for (int b = 0; b < 4; ++b) acc[a][b] = 0.0;
        for (int32_t t = 0; t < nb; ++t) {
          double l[4], u[4];
#pragma unroll
          for (int a = 0; a < 4; ++a) l[a] = Lt[(ty * 4 + a) * (kLuB + 1) + t];
#pragma unroll
          for (int b = 0; b < 4; ++b) u[b] = Ut[t * (kLuT + 1) + tx * 4 + b];
#pragma unroll
          for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int b = 0; b < 4; ++b) acc[a][b] = fma(l[a], u[b], acc[a][b]);
        }
#pragma unroll
        for (int a = 0; a < 4; ++a) {
          const int32_t i = i0 + (int32_t)ty * 4 + a;
          if (i >= c) continue;
#pragma unroll
          for (int b = 0; b < 4; ++b) {
            const int32_t j = j0 + (int32_t)tx * 4 + b;
            if (j < c) A[(size_t)i * lda + j] -= acc[a][b];
          }
        }
        __syncthreads();
      }
  }
  return true;
}

// ---------------------------------------------------------------------------------------
// Mixed precision: the same blocked factorisation on a copy of the matrix in another type
// (FP32 here), and triangular solves that apply those factors to FP64 vectors, so that FP64
// iterative refinement (residual with the FP64 matrix, correction with the FP32 factors)
// reaches the FP64 solution.  Same pivot rule and piv format as lu_factor.
// ---------------------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ int32_t pivot_search_t(const T *A, int32_t c, int32_t lda, int32_t k,
                                                  LinScratch s) {
  double best = -1.0;
  int32_t bi = k;
  for (int32_t i = k + (int32_t)threadIdx.x; i < c; i += blockDim.x) {
    const double a = fabs((double)A[(size_t)i * lda + k]);
    if (a > best) { best = a; bi = i; }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const double ob = __shfl_down_sync(0xFFFFFFFFu, best, o);
    const int32_t oi = __shfl_down_sync(0xFFFFFFFFu, bi, o);
    if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
  }
  const uint32_t warp = threadIdx.x >> 5, lane = threadIdx.x & 31u;
  if (lane == 0) { s.val[warp] = best; s.idx[warp] = bi; }
  __syncthreads();
  if (warp == 0) {
    const uint32_t nw = (blockDim.x + 31u) >> 5;
    best = lane < nw ? s.val[lane] : -1.0;
    bi = lane < nw ? s.idx[lane] : 0x7FFFFFFF;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const double ob = __shfl_down_sync(0xFFFFFFFFu, best, o);
      const int32_t oi = __shfl_down_sync(0xFFFFFFFFu, bi, o);
      if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
    }
    if (lane == 0) { s.idx[0] = bi; s.val[0] = best; }
  }
  __syncthreads();
  const int32_t p = s.idx[0];
  const double pv = s.val[0];
  __syncthreads();
  return pv > 0.0 ? p : -1;
}

template <typename T>
__host__ __device__ constexpr int lu_blocked_smem_elems() { return kLuT * (kLuB + 1) + kLuB * (kLuT + 1); }

// lu_factor_blocked on a matrix of T (256 threads; lu_blocked_smem_elems<T>() elements of T at
// tile).
template <typename T>
__device__ inline bool lu_factor_blocked_t(T *A, int32_t c, int32_t lda, int32_t *piv,
                                           LinScratch s, T *tile) {
  const uint32_t tid = threadIdx.x;
  if (blockDim.x != 256u) return false;
  T *Lt = tile;
  T *Ut = tile + kLuT * (kLuB + 1);
  for (int32_t kb = 0; kb < c; kb += kLuB) {
    const int32_t nb = min(kLuB, c - kb), ke = kb + nb;
    for (int32_t k = kb; k < ke; ++k) {
      const int32_t p = pivot_search_t(A, c, lda, k, s);
      if (p < 0) return false;
      if (tid == 0) piv[k] = p;
      if (p != k) {
        for (int32_t j = tid; j < c; j += blockDim.x) {
          const T t = A[(size_t)k * lda + j];
          A[(size_t)k * lda + j] = A[(size_t)p * lda + j];
          A[(size_t)p * lda + j] = t;
        }
        __syncthreads();
      }
      const T inv = (T)1 / A[(size_t)k * lda + k];
      for (int32_t i = k + 1 + tid; i < c; i += blockDim.x) A[(size_t)i * lda + k] *= inv;
      __syncthreads();
      const int32_t w = ke - (k + 1);
      if (w > 0) {
        const int64_t tot = (int64_t)(c - (k + 1)) * w;
        for (int64_t q = tid; q < tot; q += blockDim.x) {
          const int32_t i = k + 1 + (int32_t)(q / w), j = k + 1 + (int32_t)(q % w);
          A[(size_t)i * lda + j] = fma(-A[(size_t)i * lda + k], A[(size_t)k * lda + j], A[(size_t)i * lda + j]);
        }
      }
      __syncthreads();
    }
    if (ke >= c) break;
    for (int32_t j = ke + tid; j < c; j += blockDim.x)
      for (int32_t r = 1; r < nb; ++r) {
        T acc = A[(size_t)(kb + r) * lda + j];
        for (int32_t t = 0; t < r; ++t)
          acc = fma(-A[(size_t)(kb + r) * lda + kb + t], A[(size_t)(kb + t) * lda + j], acc);
        A[(size_t)(kb + r) * lda + j] = acc;
      }
    __syncthreads();
    const uint32_t ty = tid / 16u, tx = tid % 16u;
    for (int32_t i0 = ke; i0 < c; i0 += kLuT)
      for (int32_t j0 = ke; j0 < c; j0 += kLuT) {
        for (uint32_t q = tid; q < (uint32_t)(kLuT * kLuB); q += blockDim.x) {
          const int32_t r = (int32_t)(q / kLuB), t = (int32_t)(q % kLuB);
          Lt[r * (kLuB + 1) + t] = (i0 + r < c && t < nb) ? A[(size_t)(i0 + r) * lda + kb + t] : (T)0;
          const int32_t t2 = (int32_t)(q / kLuT), col = (int32_t)(q % kLuT);
          Ut[t2 * (kLuT + 1) + col] = (j0 + col < c && t2 < nb) ? A[(size_t)(kb + t2) * lda + j0 + col] : (T)0;
        }
        __syncthreads();
        T acc[4][4];
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
          for (int b = 0; b < 4; ++b) acc[a][b] = (T)0;
        for (int32_t t = 0; t < nb; ++t) {
          T l[4], u[4];
#pragma unroll
          for (int a = 0; a < 4; ++a) l[a] = Lt[(ty * 4 + a) * (kLuB + 1) + t];
#pragma unroll
          for (int b = 0; b < 4; ++b) u[b] = Ut[t * (kLuT + 1) + tx * 4 + b];
#pragma unroll
          for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int b = 0; b < 4; ++b) acc[a][b] = fma(l[a], u[b], acc[a][b]);
        }
#pragma unroll
        for (int a = 0; a < 4; ++a) {
          const int32_t i = i0 + (int32_t)ty * 4 + a;
          if (i >= c) continue;
#pragma unroll
          for (int b = 0; b < 4; ++b) {
            const int32_t j = j0 + (int32_t)tx * 4 + b;
            if (j < c) A[(size_t)i * lda + j] -= acc[a][b];
          }
        }
        __syncthreads();
      }
  }
  return true;
}

// A x = b with factors of type F (lu_factor_blocked_t), b and x in FP64 (in place).
template <typename F>
__device__ inline void lu_solve_t(const F *LU, int32_t c, int32_t lda, const int32_t *piv,
                                  double *b, LinScratch s) {
  if (threadIdx.x == 0)
    for (int32_t k = 0; k < c; ++k) {
      const int32_t p = piv[k];
      if (p != k) { const double t = b[k]; b[k] = b[p]; b[p] = t; }
    }
  __syncthreads();
  for (int32_t k = 0; k < c; ++k) {
    const double yk = b[k];
    for (int32_t i = k + 1 + threadIdx.x; i < c; i += blockDim.x)
      b[i] = fma(-(double)LU[(size_t)i * lda + k], yk, b[i]);
    __syncthreads();
  }
  for (int32_t k = c - 1; k >= 0; --k) {
    if (threadIdx.x == 0) s.bcast[0] = b[k] / (double)LU[(size_t)k * lda + k];
    __syncthreads();
    const double xk = s.bcast[0];
    for (int32_t i = threadIdx.x; i < k; i += blockDim.x)
      b[i] = fma(-(double)LU[(size_t)i * lda + k], xk, b[i]);
    if (threadIdx.x == 0) b[k] = xk;
    __syncthreads();
  }
}

// A^T x = b with factors of type F, FP64 vectors (in place).
template <typename F>
__device__ inline void lu_solve_transposed_t(const F *LU, int32_t c, int32_t lda,
                                             const int32_t *piv, double *b, LinScratch s) {
  for (int32_t k = 0; k < c; ++k) {
    if (threadIdx.x == 0) s.bcast[0] = b[k] / (double)LU[(size_t)k * lda + k];
    __syncthreads();
    const double zk = s.bcast[0];
    for (int32_t i = k + 1 + threadIdx.x; i < c; i += blockDim.x)
      b[i] = fma(-(double)LU[(size_t)k * lda + i], zk, b[i]);
    if (threadIdx.x == 0) b[k] = zk;
    __syncthreads();
  }
  for (int32_t k = c - 1; k >= 0; --k) {
    const double wk = b[k];
    for (int32_t i = threadIdx.x; i < k; i += blockDim.x)
      b[i] = fma(-(double)LU[(size_t)k * lda + i], wk, b[i]);
    __syncthreads();
  }
  if (threadIdx.x == 0)
    for (int32_t k = c - 1; k >= 0; --k) {
      const int32_t p = piv[k];
      if (p != k) { const double t = b[k]; b[k] = b[p]; b[p] = t; }
    }
  __syncthreads();
}

// Blocked triangular solves with factors of type F on FP64 vectors (in place), for factors in
// device memory: per 32-row block, warp 0 solves the diagonal block with shuffles, then the
// CTA updates the remaining rows with the block's solution.  Two barriers per block instead
// of one per row.  Same results as lu_solve_t / lu_solve_transposed_t up to rounding order.
template <typename F>
__device__ inline void lu_solve_blocked_t(const F *LU, int32_t c, int32_t lda, const int32_t *piv,
                                          double *b) {
  const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
  if (threadIdx.x == 0)
    for (int32_t k = 0; k < c; ++k) {
      const int32_t p = piv[k];
      if (p != k) { const double t = b[k]; b[k] = b[p]; b[p] = t; }
    }
  __syncthreads();
  for (int32_t kb = 0; kb < c; kb += 32) {          // L y = P b, L unit lower
    const int32_t nb = min(32, c - kb), ke = kb + nb;
    if (warp == 0) {
      double v = (int32_t)lane < nb ? b[kb + lane] : 0.0;
      for (int32_t i = 0; i < nb; ++i) {
        const double xi = __shfl_sync(0xFFFFFFFFu, v, i);
        if ((int32_t)lane > i && (int32_t)lane < nb) v = fma(-(double)LU[(size_t)(kb + lane) * lda + kb + i], xi, v);
      }
      if ((int32_t)lane < nb) b[kb + lane] = v;
    }
    __syncthreads();
    for (int32_t i = ke + threadIdx.x; i < c; i += blockDim.x) {
      double acc = b[i];
      for (int32_t t = 0; t < nb; ++t) acc = fma(-(double)LU[(size_t)i * lda + kb + t], b[kb + t], acc);
      b[i] = acc;
    }
    __syncthreads();
  }
  for (int32_t kb = ((c - 1) / 32) * 32; kb >= 0; kb -= 32) {   // U x = y
    const int32_t nb = min(32, c - kb);
    if (warp == 0) {
      double v = (int32_t)lane < nb ? b[kb + lane] : 0.0;
      for (int32_t i = nb - 1; i >= 0; --i) {
        double xi = (int32_t)lane == i ? v / (double)LU[(size_t)(kb + i) * lda + kb + i] : 0.0;
        xi = __shfl_sync(0xFFFFFFFFu, xi, i);
        if ((int32_t)lane == i) v = xi;
        else if ((int32_t)lane < i) v = fma(-(double)LU[(size_t)(kb + lane) * lda + kb + i], xi, v);
      }
      if ((int32_t)lane < nb) b[kb + lane] = v;
    }
    __syncthreads();
    for (int32_t i = threadIdx.x; i < kb; i += blockDim.x) {
      double acc = b[i];
      for (int32_t t = 0; t < nb; ++t) acc = fma(-(double)LU[(size_t)i * lda + kb + t], b[kb + t], acc);
      b[i] = acc;
    }
    __syncthreads();
  }
}

template <typename F>
__device__ inline void lu_solve_transposed_blocked_t(const F *LU, int32_t c, int32_t lda,
                                                     const int32_t *piv, double *b) {
  const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
  for (int32_t kb = 0; kb < c; kb += 32) {          // U^T z = b (lower, with diagonal)
    const int32_t nb = min(32, c - kb), ke = kb + nb;
    if (warp == 0) {
      double v = (int32_t)lane < nb ? b[kb + lane] : 0.0;
      for (int32_t i = 0; i < nb; ++i) {
        double zi = (int32_t)lane == i ? v / (double)LU[(size_t)(kb + i) * lda + kb + i] : 0.0;
        zi = __shfl_sync(0xFFFFFFFFu, zi, i);
        if ((int32_t)lane == i) v = zi;
        else if ((int32_t)lane > i && (int32_t)lane < nb) v = fma(-(double)LU[(size_t)(kb + i) * lda + kb + lane], zi, v);
      }
      if ((int32_t)lane < nb) b[kb + lane] = v;
    }
    __syncthreads();
    for (int32_t i = ke + threadIdx.x; i < c; i += blockDim.x) {
      double acc = b[i];
      for (int32_t t = 0; t < nb; ++t) acc = fma(-(double)LU[(size_t)(kb + t) * lda + i], b[kb + t], acc);
      b[i] = acc;
    }
    __syncthreads();
  }
  for (int32_t kb = ((c - 1) / 32) * 32; kb >= 0; kb -= 32) {   // L^T w = z (unit upper)
    const int32_t nb = min(32, c - kb);
    if (warp == 0) {
      double v = (int32_t)lane < nb ? b[kb + lane] : 0.0;
      for (int32_t i = nb - 1; i >= 0; --i) {
        const double wi = __shfl_sync(0xFFFFFFFFu, v, i);
        if ((int32_t)lane < i) v = fma(-(double)LU[(size_t)(kb + i) * lda + kb + lane], wi, v);
      }
      if ((int32_t)lane < nb) b[kb + lane] = v;
    }
    __syncthreads();
    for (int32_t i = threadIdx.x; i < kb; i += blockDim.x) {
      double acc = b[i];
      for (int32_t t = 0; t < nb; ++t) acc = fma(-(double)LU[(size_t)(kb + t) * lda + i], b[kb + t], acc);
      b[i] = acc;
    }
    __syncthreads();
  }
  if (threadIdx.x == 0)
    for (int32_t k = c - 1; k >= 0; --k) {
      const int32_t p = piv[k];
      if (p != k) { const double t = b[k]; b[k] = b[p]; b[p] = t; }
    }
  __syncthreads();
}

// Solves A x = b in place (b -> x) with the factors of lu_factor.
__device__ inline void lu_solve(const double *LU, int32_t c, int32_t lda, const int32_t *piv, double *b,
                         LinScratch s) {
  if (threadIdx.x == 0)
    for (int32_t k = 0; k < c; ++k) {
      const int32_t p = piv[k];
      if (p != k) { const double t = b[k]; b[k] = b[p]; b[p] = t; }
    }
  __syncthreads();
  for (int32_t k = 0; k < c; ++k) {  // L y = P b
    const double yk = b[k];
    for (int32_t i = k + 1 + threadIdx.x; i < c; i += blockDim.x)
      b[i] = fma(-LU[(size_t)i * lda + k], yk, b[i]);
    __syncthreads();
  }
  for (int32_t k = c - 1; k >= 0; --k) {  // U x = y
    if (threadIdx.x == 0) s.bcast[0] = b[k] / LU[(size_t)k * lda + k];
    __syncthreads();
    const double xk = s.bcast[0];
    for (int32_t i = threadIdx.x; i < k; i += blockDim.x) b[i] = fma(-LU[(size_t)i * lda + k], xk, b[i]);
    if (threadIdx.x == 0) b[k] = xk;
    __syncthreads();
  }
}

// Solves A^T x = b in place (b -> x): U^T z = b, L^T w = z, x = P^T w.
__device__ inline void lu_solve_transposed(const double *LU, int32_t c, int32_t lda, const int32_t *piv,
                                    double *b, LinScratch s) {
  for (int32_t k = 0; k < c; ++k) {  // U^T z = b (forward; column k of U^T = row k of U)
    if (threadIdx.x == 0) s.bcast[0] = b[k] / LU[(size_t)k * lda + k];
    __syncthreads();
    const double zk = s.bcast[0];
    for (int32_t i = k + 1 + threadIdx.x; i < c; i += blockDim.x) b[i] = fma(-LU[(size_t)k * lda + i], zk, b[i]);
    if (threadIdx.x == 0) b[k] = zk;
    __syncthreads();
  }
  for (int32_t k = c - 1; k >= 0; --k) {  // L^T w = z (backward, unit diagonal)
    const double wk = b[k];
    for (int32_t i = threadIdx.x; i < k; i += blockDim.x) b[i] = fma(-LU[(size_t)k * lda + i], wk, b[i]);
    __syncthreads();
  }
  if (threadIdx.x == 0)
    for (int32_t k = c - 1; k >= 0; --k) {
      const int32_t p = piv[k];
      if (p != k) { const double t = b[k]; b[k] = b[p]; b[p] = t; }
    }
  __syncthreads();
}

// Block reductions of doubles (result broadcast to every thread).
__device__ __forceinline__ double block_sum(double x, double *tmp) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xFFFFFFFFu, x, o);
  const uint32_t warp = threadIdx.x >> 5, lane = threadIdx.x & 31u;
  __syncthreads();
  if (lane == 0) tmp[warp] = x;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (uint32_t w = 0; w < (blockDim.x + 31u) / 32u; ++w) t += tmp[w];
    tmp[32] = t;
  }
  __syncthreads();
  return tmp[32];
}

__device__ __forceinline__ double block_max(double x, double *tmp) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x = fmax(x, __shfl_down_sync(0xFFFFFFFFu, x, o));
  const uint32_t warp = threadIdx.x >> 5, lane = threadIdx.x & 31u;
  __syncthreads();
  if (lane == 0) tmp[warp] = x;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = tmp[0];
    for (uint32_t w = 1; w < (blockDim.x + 31u) / 32u; ++w) t = fmax(t, tmp[w]);
    tmp[32] = t;
  }
  __syncthreads();
  return tmp[32];
}

}  // namespace afc
