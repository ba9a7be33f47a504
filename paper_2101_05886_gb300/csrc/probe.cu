// probe.cu - measured arithmetic peaks of the device the library runs on (C ABI in
// include/fp.h: fp_probe_peaks).  The roofline of the sweep divides by these: FP32 fused
// multiply-add issued as scalar FFMA and as packed FFMA2, and FP64 DFMA.
//
// Each thread runs kChains independent multiply-add chains (enough to cover the pipe
// latency) for `iters` iterations on values that stay bounded (x <- x a + b with |a| < 1),
// and the sum of the chains is stored so that nothing can be removed.  The grid fills every
// SM with several CTAs.  flops = 2 x chains x iterations x threads (x 2 for FFMA2).
#include <cuda_runtime.h>

#include <algorithm>

#include "../../include/fp.h"
#include "fp_internal.h"

namespace {

constexpr int kChains = 8;
constexpr int kProbeThreads = 256;

__global__ void __launch_bounds__(kProbeThreads) k_ffma(float *out, int iters, float a, float b) {
  float x[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) x[c] = 1e-3f * (threadIdx.x + c);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = fmaf(x[c], a, b);
  }
  float s = 0.f;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += x[c];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void __launch_bounds__(kProbeThreads) k_ffma2(float *out, int iters, float a, float b) {
  float2 x[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) x[c] = make_float2(1e-3f * (threadIdx.x + c), 2e-3f * (threadIdx.x + c));
  const float2 a2 = make_float2(a, a), b2 = make_float2(b, b);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = __ffma2_rn(x[c], a2, b2);
  }
  float s = 0.f;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += x[c].x + x[c].y;
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void __launch_bounds__(kProbeThreads) k_dfma(double *out, int iters, double a, double b) {
  double x[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) x[c] = 1e-3 * (threadIdx.x + c);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = fma(x[c], a, b);
  }
  double s = 0.0;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += x[c];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// best of `reps` timed launches (after one warm-up) of `launch`, in milliseconds
template <typename F>
cudaError_t best_ms(F launch, cudaStream_t s, int reps, float *ms) {
  cudaEvent_t e0, e1;
  cudaError_t e = cudaEventCreate(&e0);
  if (e != cudaSuccess) return e;
  e = cudaEventCreate(&e1);
  if (e != cudaSuccess) { cudaEventDestroy(e0); return e; }
  launch();
  float best = 1e30f;
  for (int r = 0; r < reps && e == cudaSuccess; ++r) {
    e = cudaEventRecord(e0, s);
    launch();
    if (e == cudaSuccess) e = cudaEventRecord(e1, s);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float t = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&t, e0, e1);
    if (e == cudaSuccess) best = std::min(best, t);
  }
  if (e == cudaSuccess) e = cudaGetLastError();
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  *ms = best;
  return e;
}

}  // namespace

extern "C" int fp_probe_peaks(double *fp32_tflops, double *fp32x2_tflops, double *fp64_tflops,
                              void *stream) {
  if (!fp32_tflops || !fp32x2_tflops || !fp64_tflops) return FP_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  int dev = 0, nsm = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return FP_ERR_CUDA;
  const int grid = nsm * 8;                      // 8 CTAs of 256 threads per SM: 64 warps
  const double threads = (double)grid * kProbeThreads;
  void *buf = nullptr;
  e = fpk::dev_malloc(&buf, (size_t)grid * kProbeThreads * sizeof(double));
  if (e != cudaSuccess) return e == cudaErrorMemoryAllocation ? FP_ERR_OOM : FP_ERR_CUDA;
  const int it32 = 1 << 16, it64 = 1 << 11;     // tens of milliseconds per launch on one GB300
  float ms32 = 0.f, ms32x2 = 0.f, ms64 = 0.f;
  e = best_ms([&] { k_ffma<<<grid, kProbeThreads, 0, s>>>((float *)buf, it32, 0.999f, 1e-4f); }, s, 3, &ms32);
  if (e == cudaSuccess)
    e = best_ms([&] { k_ffma2<<<grid, kProbeThreads, 0, s>>>((float *)buf, it32, 0.999f, 1e-4f); }, s, 3, &ms32x2);
  if (e == cudaSuccess)
    e = best_ms([&] { k_dfma<<<grid, kProbeThreads, 0, s>>>((double *)buf, it64, 0.999, 1e-4); }, s, 3, &ms64);
  cudaFree(buf);
  if (e != cudaSuccess) return FP_ERR_CUDA;
  *fp32_tflops = 2.0 * kChains * (double)it32 * threads / (ms32 * 1e-3) / 1e12;
  *fp32x2_tflops = 4.0 * kChains * (double)it32 * threads / (ms32x2 * 1e-3) / 1e12;
  *fp64_tflops = 2.0 * kChains * (double)it64 * threads / (ms64 * 1e-3) / 1e12;
  return FP_OK;
}
