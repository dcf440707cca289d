// diag.cu -- a measurement of the GPU's FMA throughput in FP64 and FP32, the denominators of
// the FP64-bound kernels' rooflines (the absorbing solve and the perturbation sweep's LU).
// Every thread runs 8 independent FMA chains in registers for a fixed number of steps; the
// result is written so the compiler keeps the work.  Grid: 4 CTAs of 256 threads per SM.
#include <cstdint>

#include <cuda_runtime.h>

#include "abi_util.h"

using namespace afc;

namespace {

template <typename T>
__global__ void __launch_bounds__(256) fma_kernel(int32_t steps, T a, T b, T *sink) {
  T x[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) x[k] = (T)(threadIdx.x + k) * (T)1e-3;
  for (int32_t s = 0; s < steps; ++s) {
#pragma unroll
    for (int k = 0; k < 8; ++k) x[k] = fma(x[k], a, b);
  }
  T acc = 0;
#pragma unroll
  for (int k = 0; k < 8; ++k) acc += x[k];
  if (acc == (T)12345.678) sink[0] = acc;   // practically never true: keeps the chains live
}

template <typename T>
int measure(int32_t steps, double *tflops, cudaStream_t s) {
  const afc::DevInfo d = afc::dev_info();
  const int grid = 4 * (d.sms > 0 ? d.sms : 1);
  T *sink = nullptr;
  AFC_CUDA(cudaMallocAsync(&sink, sizeof(T), s));
  fma_kernel<T><<<grid, 256, 0, s>>>(steps / 8 + 1, (T)0.999999, (T)1e-7, sink);   // warm-up
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  cudaEventRecord(e0, s);
  fma_kernel<T><<<grid, 256, 0, s>>>(steps, (T)0.999999, (T)1e-7, sink);
  cudaEventRecord(e1, s);
  cudaError_t e = cudaEventSynchronize(e1);
  float ms = 0.f;
  cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFreeAsync(sink, s);
  cudaStreamSynchronize(s);
  if (e != cudaSuccess) return afc::cuda_fail(e, "fma measurement");
  const double flops = 2.0 * 8.0 * (double)steps * 256.0 * (double)grid;
  *tflops = ms > 0.f ? flops / ((double)ms * 1e-3) / 1e12 : 0.0;
  return AFC_OK;
}

}  // namespace

extern "C" int afc_measure_fma_rate(int32_t fp64, double *tflops, void *stream) {
  afc::NvtxRange nvtx_range("afc.measure_fma_rate");
  if (!tflops) return afc::fail(AFC_EINVAL, "null output");
  cudaStream_t s = (cudaStream_t)stream;
  return fp64 ? measure<double>(1 << 16, tflops, s) : measure<float>(1 << 18, tflops, s);
}
