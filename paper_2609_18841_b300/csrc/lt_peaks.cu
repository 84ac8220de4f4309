// Roofline denominators of the SIMT pipes: a microbenchmark of independent
// fused multiply-add chains (registers only, no memory traffic in the timed
// loop), timed with CUDA events.  The single-precision kernel issues packed
// pairs (__ffma2_rn), the form the bond kernel's hot loops use; the
// double-precision kernel issues scalar FMAs.
#include <cuda_runtime.h>

#include "lindtebd.h"

namespace {

constexpr int kChains = 8;
constexpr int kThreads = 256;

__global__ void __launch_bounds__(kThreads) peak_ffma2_kernel(int iters, float seed, float* sink) {
  float2 acc[kChains];
#pragma unroll
  for (int i = 0; i < kChains; ++i) acc[i] = make_float2(seed + i, seed - i);
  const float2 a = make_float2(0.999999f, 0.999998f), b = make_float2(1e-7f, 2e-7f);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int u = 0; u < 16; ++u)
#pragma unroll
      for (int i = 0; i < kChains; ++i) acc[i] = __ffma2_rn(acc[i], a, b);
  }
  float s = 0.f;
#pragma unroll
  for (int i = 0; i < kChains; ++i) s += acc[i].x + acc[i].y;
  if (s == 12345.678f) sink[threadIdx.x] = s;  // keeps the chains live
}

__global__ void __launch_bounds__(kThreads) peak_dfma_kernel(int iters, double seed, double* sink) {
  double acc[kChains];
#pragma unroll
  for (int i = 0; i < kChains; ++i) acc[i] = seed + i;
  const double a = 0.9999999999, b = 1e-12;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int u = 0; u < 16; ++u)
#pragma unroll
      for (int i = 0; i < kChains; ++i) acc[i] = fma(acc[i], a, b);
  }
  double s = 0.0;
#pragma unroll
  for (int i = 0; i < kChains; ++i) s += acc[i];
  if (s == 12345.678) sink[threadIdx.x] = s;
}

}  // namespace

extern "C" lt_status lt_pipe_peaks(double* out) {
  if (!out) return LT_ERR_ARG;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return LT_ERR_CUDA;
  cudaStream_t st = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  void* sink = nullptr;
  lt_status rc = LT_OK;
  if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess ||
      cudaMalloc(&sink, kThreads * sizeof(double)) != cudaSuccess) {
    rc = LT_ERR_CUDA;
  } else {
    const int grid = 4 * sms;  // four resident CTAs of 256 threads per SM
    for (int pass = 0; pass < 2 && rc == LT_OK; ++pass) {
      // single precision: iters x 16 x 8 packed FMAs of 4 flops per thread
      const int it32 = 40000, it64 = 1500;
      float ms = 0.f;
      for (int rep = 0; rep < 2; ++rep) {  // the first launch warms the clocks up
        cudaEventRecord(e0, st);
        if (pass == 0) peak_ffma2_kernel<<<grid, kThreads, 0, st>>>(it32, 1.0f, (float*)sink);
        else peak_dfma_kernel<<<grid, kThreads, 0, st>>>(it64, 1.0, (double*)sink);
        cudaEventRecord(e1, st);
        if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
          rc = LT_ERR_CUDA;
          break;
        }
      }
      if (rc != LT_OK || ms <= 0.f) break;
      const double per_thread = pass == 0 ? (double)it32 * 16 * kChains * 4 : (double)it64 * 16 * kChains * 2;
      out[pass] = per_thread * grid * kThreads / (ms * 1e-3) / 1e12;
    }
    int clk = 0;
    cudaDeviceGetAttribute(&clk, cudaDevAttrClockRate, dev);
    out[2] = clk / 1000.0;
    out[3] = sms;
  }
  if (sink) cudaFree(sink);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (st) cudaStreamDestroy(st);
  return rc;
}
