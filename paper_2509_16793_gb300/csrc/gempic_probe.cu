// FP32 FMA throughput probe: the measured denominator of the ALU roofline the particle push is
// reported against (gempic_probe_fp32_fma, include/gempic.h).  The paper has no counterpart.
//
// Every thread runs 16 independent FMA chains (enough to hide the FMA latency at 16 warps per
// SM) for `iters` iterations; the grid holds 4 CTAs of 512 threads per SM.  The result is kept
// alive by a store that depends on it and is never taken in practice; the sink is a file-scope
// device array, so the probe allocates nothing.
#include <cuda_runtime.h>

#include <cstdint>

#include "../../include/gempic.h"

namespace {

constexpr int kChains = 16;
constexpr int kThreads = 512;

__device__ float g_probe_sink[kThreads];

__global__ void __launch_bounds__(kThreads) fma_probe_kernel(int iters, float a, float b) {
  float x[kChains];
#pragma unroll
  for (int i = 0; i < kChains; ++i) x[i] = (float)(threadIdx.x + i) * 1e-3f;
  for (int k = 0; k < iters; ++k) {
#pragma unroll
    for (int i = 0; i < kChains; ++i) x[i] = fmaf(x[i], a, b);
  }
  float s = 0.0f;
#pragma unroll
  for (int i = 0; i < kChains; ++i) s += x[i];
  if (s == -1.0f) g_probe_sink[threadIdx.x] = s;
}

}  // namespace

extern "C" gempic_status gempic_probe_fp32_fma(void* cuda_stream, int32_t iters, double* tflops,
                                               double* ms) {
  if (iters < 1 || !tflops) return GEMPIC_EINVAL;
  cudaStream_t s = (cudaStream_t)cuda_stream;
  int dev = 0, nsm = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return GEMPIC_ECUDA;
  const int blocks = 4 * nsm;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  // warm-up launch (clocks ramp, code loaded), then the timed one
  if (e == cudaSuccess) {
    fma_probe_kernel<<<blocks, kThreads, 0, s>>>(iters / 8 + 1, 0.999999f, 1e-6f);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaEventRecord(e0, s);
  if (e == cudaSuccess) {
    fma_probe_kernel<<<blocks, kThreads, 0, s>>>(iters, 0.999999f, 1e-6f);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaEventRecord(e1, s);
  if (e == cudaSuccess) e = cudaEventSynchronize(e1);
  float t = 0.0f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&t, e0, e1);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (e != cudaSuccess) return GEMPIC_ECUDA;
  const double flop = 2.0 * kChains * (double)iters * (double)blocks * kThreads;
  *tflops = flop / (t * 1e-3) / 1e12;
  if (ms) *ms = t;
  return GEMPIC_OK;
}
