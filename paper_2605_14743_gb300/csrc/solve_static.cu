// solve_static.cu -- allocation-free variant of the absorbing-chain solve.
//
// For callers that cannot allocate device memory themselves (for example code running inside
// a host framework whose device memory is all handed out up front, or a plugin that may only
// use buffers it is given): the whole workspace of the solve lives in one file-scope device
// array of fixed size, so a call needs nothing but its inputs and outputs.
//
// Limits: n <= kStaticMaxN nodes and at most kStaticMaxC observed centre states.  The array is
// shared by every call on a device and keeps the last call's contents; calls whose work
// overlaps on the GPU (different streams, or different host threads) race on it.
#include <cstdint>
#include <mutex>

#include <cuda_runtime.h>

#include "afc_internal.h"
#include "linalg.cuh"

namespace afc {

constexpr int32_t kStaticMaxN = 4096;
constexpr int32_t kStaticMaxC = 256;

// Scratch layout (bytes): c_index, c_list, c, status | row scale and absorption | y, t | A, piv
constexpr size_t kOffCIndex = 0;
constexpr size_t kOffCList = kOffCIndex + 4 * kStaticMaxN;
constexpr size_t kOffCount = kOffCList + 4 * kStaticMaxN;          // int32 c, u32 status
constexpr size_t kOffRow = kOffCount + 256;                        // f64 [2 n]
constexpr size_t kOffY = kOffRow + 16 * kStaticMaxN;               // f64 [c]
constexpr size_t kOffT = kOffY + 8 * kStaticMaxC;                  // f64 [c]
constexpr size_t kOffPiv = kOffT + 8 * kStaticMaxC;                // i32 [c]
constexpr size_t kOffA = kOffPiv + 4 * kStaticMaxC;                // f64 [c c]
constexpr size_t kStaticBytes = kOffA + 8 * (size_t)kStaticMaxC * kStaticMaxC;

static __device__ __align__(256) unsigned char g_static_scratch[kStaticBytes];

constexpr uint32_t kStatusTooManyStates = 1u;
constexpr uint32_t kStatusSingular = 2u;

// Row scales (Q_ij = scale_i counts_ij) and absorption r_i, as in the workspace solve.
__global__ void static_rows_kernel(int32_t n, uint32_t R, double alpha, double eta,
                                   const uint32_t *counts, double *row) {
  const size_t stride = (size_t)n + 1;
  const uint32_t warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31u;
  const uint32_t nwarps = (gridDim.x * blockDim.x) >> 5;
  for (int32_t i = warp; i < n; i += nwarps) {
    const uint32_t *rowc = counts + (size_t)i * stride;
    unsigned long long tsum = 0;
    for (int32_t j = lane; j < n; j += 32) tsum += rowc[j];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) tsum += __shfl_down_sync(0xFFFFFFFFu, tsum, o);
    if (lane == 0) {
      double scale = (1.0 - alpha) / (double)R;
      double r = alpha + (1.0 - alpha) * (double)rowc[n] / (double)R;
      if (r == 0.0) {
        const double qsum = (1.0 - alpha) * (double)tsum / (double)R;
        r = eta;
        if (qsum > 0.0) scale *= (1.0 - eta) / qsum;
      }
      row[2 * i] = scale;
      row[2 * i + 1] = r;
    }
  }
}

// A = I - Q_CC and y = s_C + s_U Q_UC from the dense counts (c read on the device).
__global__ void static_assemble_kernel(int32_t n, const uint32_t *counts, const double *s,
                                       unsigned char *scr) {
  const int32_t c = *reinterpret_cast<const int32_t *>(scr + kOffCount);
  if (c > kStaticMaxC) return;
  const int32_t *c_index = reinterpret_cast<const int32_t *>(scr + kOffCIndex);
  const double *row = reinterpret_cast<const double *>(scr + kOffRow);
  double *y = reinterpret_cast<double *>(scr + kOffY);
  double *A = reinterpret_cast<double *>(scr + kOffA);
  const size_t stride = (size_t)n + 1;
  const uint32_t warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31u;
  const uint32_t nwarps = (gridDim.x * blockDim.x) >> 5;
  for (int32_t i = warp; i < n; i += nwarps) {
    const uint32_t *rowc = counts + (size_t)i * stride;
    const double scale = row[2 * i];
    const double si = s ? s[i] : 1.0 / (double)n;
    const int32_t pi = c_index[i];
    for (int32_t j = lane; j < n; j += 32) {
      const uint32_t v = rowc[j];
      if (!v) continue;
      const int32_t pj = c_index[j];
      const double q = scale * (double)v;
      if (pi >= 0) A[(size_t)pi * c + pj] -= q;
      else atomicAdd(&y[pj], si * q);
    }
    if (lane == 0 && pi >= 0) atomicAdd(&y[pi], si);
  }
}

__global__ void static_reset_kernel(unsigned char *scr) {
  const int32_t c = *reinterpret_cast<const int32_t *>(scr + kOffCount);
  uint32_t *status = reinterpret_cast<uint32_t *>(scr + kOffCount + 4);
  if (c > kStaticMaxC) {
    if (blockIdx.x == 0 && threadIdx.x == 0) *status = kStatusTooManyStates;
    return;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) *status = 0u;
  double *A = reinterpret_cast<double *>(scr + kOffA);
  double *y = reinterpret_cast<double *>(scr + kOffY);
  const size_t total = (size_t)c * c;
  for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < total;
       k += (size_t)gridDim.x * blockDim.x)
    A[k] = (k / c == k % c) ? 1.0 : 0.0;
  for (int32_t k = blockIdx.x * blockDim.x + threadIdx.x; k < c; k += gridDim.x * blockDim.x)
    y[k] = 0.0;
}

// Factor, mu_C, (N 1)_C, and the C part of the outputs (one CTA).
__global__ void __launch_bounds__(1024, 1)
static_solve_kernel(int32_t n, const double *s, const double *f, unsigned char *scr, double *mu,
                    double *b, double *scalars) {
  __shared__ double sval[33];
  __shared__ int32_t sidx[32];
  __shared__ double sb[2];
  __shared__ int32_t sflag[1];
  __shared__ double red[33];
  LinScratch ls{sval, sidx, sb, sflag};
  const int32_t c = *reinterpret_cast<const int32_t *>(scr + kOffCount);
  uint32_t *status = reinterpret_cast<uint32_t *>(scr + kOffCount + 4);
  if (c > kStaticMaxC) return;
  const int32_t *c_index = reinterpret_cast<const int32_t *>(scr + kOffCIndex);
  double *y = reinterpret_cast<double *>(scr + kOffY);
  double *t = reinterpret_cast<double *>(scr + kOffT);
  int32_t *piv = reinterpret_cast<int32_t *>(scr + kOffPiv);
  double *A = reinterpret_cast<double *>(scr + kOffA);
  if (c > 0) {
    if (!lu_factor(A, c, c, piv, ls)) {
      if (threadIdx.x == 0) *status = kStatusSingular;
      return;
    }
    lu_solve_transposed(A, c, c, piv, y, ls);
    for (int32_t k = threadIdx.x; k < c; k += blockDim.x) t[k] = 1.0;
    __syncthreads();
    lu_solve(A, c, c, piv, t, ls);
  }
  double part = 0.0, tmax = 0.0;
  for (int32_t i = threadIdx.x; i < n; i += blockDim.x) {
    const int32_t pi = c_index[i];
    const double m = pi >= 0 ? y[pi] : (s ? s[i] : 1.0 / (double)n);
    mu[i] = m;
    part += m;
    if (pi >= 0) tmax = fmax(tmax, t[pi]);
  }
  const double T = block_sum(part, red);
  tmax = block_max(tmax, red);
  double bf = 0.0;
  for (int32_t i = threadIdx.x; i < n; i += blockDim.x) {
    const double bi = mu[i] / T;
    b[i] = bi;
    if (f) bf += bi * f[i];
  }
  bf = block_sum(bf, red);
  if (threadIdx.x == 0) {
    scalars[0] = T;
    scalars[1] = f ? bf : 0.0;
    scalars[2] = tmax;
    scalars[3] = (double)c;
  }
}

// (N 1)_i = 1 + sum_j Q_ij (N 1)_j for the rows outside C; folded into scalars[2].
__global__ void static_rowsum_kernel(int32_t n, const uint32_t *counts, unsigned char *scr,
                                     double *scalars) {
  const int32_t c = *reinterpret_cast<const int32_t *>(scr + kOffCount);
  const uint32_t status = *reinterpret_cast<const uint32_t *>(scr + kOffCount + 4);
  if (c > kStaticMaxC || status) return;
  const int32_t *c_index = reinterpret_cast<const int32_t *>(scr + kOffCIndex);
  const double *row = reinterpret_cast<const double *>(scr + kOffRow);
  const double *t = reinterpret_cast<const double *>(scr + kOffT);
  const size_t stride = (size_t)n + 1;
  const uint32_t warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31u;
  const uint32_t nwarps = (gridDim.x * blockDim.x) >> 5;
  for (int32_t i = warp; i < n; i += nwarps) {
    if (c_index[i] >= 0) continue;
    const uint32_t *rowc = counts + (size_t)i * stride;
    double acc = 0.0;
    for (int32_t j = lane; j < n; j += 32) {
      const uint32_t v = rowc[j];
      if (v) acc += row[2 * i] * (double)v * t[c_index[j]];
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xFFFFFFFFu, acc, o);
    if (lane == 0)
      atomicMax(reinterpret_cast<unsigned long long *>(&scalars[2]),
                (unsigned long long)__double_as_longlong(1.0 + acc));
  }
}

namespace {
std::mutex g_static_mu;
unsigned char *g_static_ptr[64] = {nullptr};
}  // namespace

// Device address of the scratch array on the current device (looked up once per device).
static cudaError_t static_scratch(unsigned char **out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_static_mu);
  if (!g_static_ptr[dev]) {
    void *p = nullptr;
    e = cudaGetSymbolAddress(&p, g_static_scratch);
    if (e != cudaSuccess) return e;
    g_static_ptr[dev] = static_cast<unsigned char *>(p);
  }
  *out = g_static_ptr[dev];
  return cudaSuccess;
}

cudaError_t launch_solve_static(int32_t n, uint32_t R, double alpha, double eta, const double *s,
                                const double *f, const uint32_t *counts, double *mu, double *b,
                                double *scalars, uint32_t *status_host, int32_t *c_host,
                                cudaStream_t stream) {
  unsigned char *scr = nullptr;
  cudaError_t e = static_scratch(&scr);
  if (e != cudaSuccess) return e;
  int32_t *c_index = reinterpret_cast<int32_t *>(scr + kOffCIndex);
  int32_t *c_list = reinterpret_cast<int32_t *>(scr + kOffCList);
  int32_t *c_dev = reinterpret_cast<int32_t *>(scr + kOffCount);
  uint32_t *status = reinterpret_cast<uint32_t *>(scr + kOffCount + 4);
  e = launch_observed_states(n, counts, c_index, c_list, c_dev, stream);
  if (e != cudaSuccess) return e;
  const int blocks = (int)((n * 32 + 255) / 256 < 1024 ? (n * 32 + 255) / 256 : 1024);
  static_reset_kernel<<<256, 256, 0, stream>>>(scr);
  static_rows_kernel<<<blocks, 256, 0, stream>>>(n, R, alpha, eta, counts,
                                                 reinterpret_cast<double *>(scr + kOffRow));
  static_assemble_kernel<<<blocks, 256, 0, stream>>>(n, counts, s, scr);
  static_solve_kernel<<<1, 1024, 0, stream>>>(n, s, f, scr, mu, b, scalars);
  static_rowsum_kernel<<<blocks, 256, 0, stream>>>(n, counts, scr, scalars);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  e = cudaMemcpyAsync(status_host, status, sizeof(uint32_t), cudaMemcpyDeviceToHost, stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(c_host, c_dev, sizeof(int32_t), cudaMemcpyDeviceToHost, stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
  return e;
}

size_t solve_static_bytes() { return kStaticBytes; }

}  // namespace afc
