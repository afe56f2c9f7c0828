// Measured arithmetic rates of the device (igabem_measure_peaks): the denominators of the roofline
// fractions of the ALU-bound kernels (FP64 singular quadrature, FP32 kernel samples of the M2L).
//
// Each probe is a grid of 8 blocks of 256 threads per SM; every thread runs NCHAIN independent
// dependency chains of the probed operation (enough independent work per warp to cover the
// pipeline latency) for `iters` rounds, and the result is stored only under a condition that never
// holds at run time, so the compiler keeps the arithmetic.  The rate is operations / CUDA-event time
// of the launch on the context's stream, best of several launches after a warm-up.  Nothing here
// changes a setting of the GPU: the clocks are whatever the GPU runs at.
#include <algorithm>
#include <cmath>

#include "internal.h"

namespace igabem {

namespace {

constexpr int NCHAIN = 8;

__global__ void __launch_bounds__(256) k_probe_ffma(int iters, float seed, float *sink) {
  float a[NCHAIN];
  const float b = 0.999999f, c = 1e-7f;
#pragma unroll
  for (int k = 0; k < NCHAIN; ++k) a[k] = seed + k + threadIdx.x;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int j = 0; j < 16; ++j)
#pragma unroll
      for (int k = 0; k < NCHAIN; ++k) a[k] = fmaf(a[k], b, c);
  }
  float s = 0.f;
#pragma unroll
  for (int k = 0; k < NCHAIN; ++k) s += a[k];
  if (s == -1.2345f) sink[threadIdx.x] = s;
}

__global__ void __launch_bounds__(256) k_probe_dfma(int iters, double seed, double *sink) {
  double a[NCHAIN];
  const double b = 0.999999999, c = 1e-9;
#pragma unroll
  for (int k = 0; k < NCHAIN; ++k) a[k] = seed + k + threadIdx.x;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int j = 0; j < 16; ++j)
#pragma unroll
      for (int k = 0; k < NCHAIN; ++k) a[k] = fma(a[k], b, c);
  }
  double s = 0.0;
#pragma unroll
  for (int k = 0; k < NCHAIN; ++k) s += a[k];
  if (s == -1.2345) sink[threadIdx.x] = s;
}

// one __sincosf (a sine and a cosine on the special-function unit) per chain and round
__global__ void __launch_bounds__(256) k_probe_sincosf(int iters, float seed, float *sink) {
  float a[NCHAIN];
#pragma unroll
  for (int k = 0; k < NCHAIN; ++k) a[k] = seed + 0.1f * k + 1e-3f * threadIdx.x;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
      for (int k = 0; k < NCHAIN; ++k) {
        float s, c;
        __sincosf(a[k], &s, &c);
        a[k] = s + c;
      }
  }
  float s = 0.f;
#pragma unroll
  for (int k = 0; k < NCHAIN; ++k) s += a[k];
  if (s == -1.2345f) sink[threadIdx.x] = s;
}

// one rsqrtf per chain and round
__global__ void __launch_bounds__(256) k_probe_rsqrtf(int iters, float seed, float *sink) {
  float a[NCHAIN];
#pragma unroll
  for (int k = 0; k < NCHAIN; ++k) a[k] = seed + k + threadIdx.x;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
      for (int k = 0; k < NCHAIN; ++k) a[k] = rsqrtf(a[k]) + 1.0f;
  }
  float s = 0.f;
#pragma unroll
  for (int k = 0; k < NCHAIN; ++k) s += a[k];
  if (s == -1.2345f) sink[threadIdx.x] = s;
}

// one FP64 sincos (the CUDA math library routine, as the FP64 kernels call it) per chain and round
__global__ void __launch_bounds__(256) k_probe_dsincos(int iters, double seed, double *sink) {
  double a[NCHAIN];
#pragma unroll
  for (int k = 0; k < NCHAIN; ++k) a[k] = seed + 0.1 * k + 1e-3 * threadIdx.x;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < NCHAIN; ++k) {
      double s, c;
      sincos(a[k], &s, &c);
      a[k] = s + c;
    }
  }
  double s = 0.0;
#pragma unroll
  for (int k = 0; k < NCHAIN; ++k) s += a[k];
  if (s == -1.2345) sink[threadIdx.x] = s;
}

template <class K, class... Args>
double best_ms(K kernel, int blocks, cudaStream_t st, cudaEvent_t a, cudaEvent_t b, Args... args) {
  kernel<<<blocks, 256, 0, st>>>(args...);  // warm-up
  IGA_CUDA(cudaGetLastError());
  double best = 1e30;
  for (int rep = 0; rep < 5; ++rep) {
    IGA_CUDA(cudaEventRecord(a, st));
    kernel<<<blocks, 256, 0, st>>>(args...);
    IGA_CUDA(cudaEventRecord(b, st));
    IGA_CUDA(cudaEventSynchronize(b));
    float ms = 0.f;
    IGA_CUDA(cudaEventElapsedTime(&ms, a, b));
    best = std::min(best, (double)ms);
  }
  return best;
}

}  // namespace

}  // namespace igabem

extern "C" int igabem_measure_peaks(igabem_ctx *ctx, igabem_peaks *out) {
  using namespace igabem;
  return run_guarded([&] {
    if (!ctx || !out) fail(IGABEM_EINVAL, "NULL argument");
    IGA_CUDA(cudaSetDevice(ctx->device));
    int sms = 0, clk_khz = 0;
    IGA_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, ctx->device));
    cudaDeviceGetAttribute(&clk_khz, cudaDevAttrClockRate, ctx->device);
    cudaGetLastError();
    cudaStream_t st = ctx->stream;
    cudaEvent_t a, b;
    IGA_CUDA(cudaEventCreate(&a));
    IGA_CUDA(cudaEventCreate(&b));
    void *sink = nullptr;
    cudaError_t e = cudaMalloc(&sink, 256 * sizeof(double));
    if (e != cudaSuccess) {
      cudaEventDestroy(a);
      cudaEventDestroy(b);
      IGA_CUDA(e);
    }
    const int blocks = 8 * sms;
    const double threads = (double)blocks * 256;
    try {
      const int it32 = 4096, it64 = 256, itsf = 2048, itd = 64;
      double ms = best_ms(k_probe_ffma, blocks, st, a, b, it32, 1.0f, (float *)sink);
      out->fp32_tflops = threads * it32 * 16 * NCHAIN * 2.0 / (ms * 1e-3) / 1e12;
      ms = best_ms(k_probe_dfma, blocks, st, a, b, it64, 1.0, (double *)sink);
      out->fp64_tflops = threads * it64 * 16 * NCHAIN * 2.0 / (ms * 1e-3) / 1e12;
      ms = best_ms(k_probe_sincosf, blocks, st, a, b, itsf, 0.5f, (float *)sink);
      out->sincosf_gops = threads * itsf * 4 * NCHAIN / (ms * 1e-3) / 1e9;
      ms = best_ms(k_probe_rsqrtf, blocks, st, a, b, itsf, 2.0f, (float *)sink);
      out->rsqrtf_gops = threads * itsf * 4 * NCHAIN / (ms * 1e-3) / 1e9;
      ms = best_ms(k_probe_dsincos, blocks, st, a, b, itd, 0.5, (double *)sink);
      out->sincos_fp64_gops = threads * itd * NCHAIN / (ms * 1e-3) / 1e9;
      out->sm_count = sms;
      out->sm_clock_mhz_attr = clk_khz / 1000.0;
    } catch (...) {
      cudaFree(sink);
      cudaEventDestroy(a);
      cudaEventDestroy(b);
      throw;
    }
    cudaFree(sink);
    cudaEventDestroy(a);
    cudaEventDestroy(b);
  });
}
