// Measured instruction-throughput roofs of the composites' arithmetic.
//
// The blend loops of Alg. 1 and Alg. 2 are bound by arithmetic issue, not by
// memory: FP32 fused multiply-adds (the exponent, the erf polynomial, the
// blend), FP32 compares, min/max and selects (the gate, the clamp), and the
// multi-function unit for ex2 and rcp (one exponential and one reciprocal
// per erf evaluation, one exponential for the Gaussian).  Each kernel below
// keeps every SM busy with independent dependency chains of one instruction
// kind, so its rate is that kind's throughput on this GPU at the clock it
// runs at; sr_measure_alu_peaks times them with CUDA events.
#include <cuda_runtime.h>

#include "kernels.cuh"

namespace sr {
namespace {

constexpr int kPeakThreads = 256;
constexpr int kPeakChains = 8;   // independent chains per thread
constexpr int kPeakUnroll = 16;  // chain steps per loop iteration

__device__ __forceinline__ float ex2_op(float x) {
  float y;
  asm volatile("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

__device__ __forceinline__ float rcp_op(float x) {
  float y;
  asm volatile("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// the sum of the chains goes to sink only when it takes a value it never
// takes, so the chains stay live without memory traffic
__device__ __forceinline__ void keep(float* sink, const float* a) {
  float s = 0.0f;
#pragma unroll
  for (int c = 0; c < kPeakChains; ++c) s += a[c];
  if (s == -1.2345e30f) sink[threadIdx.x & 31] = s;
}

// one FP32 FMA per chain step
__global__ void __launch_bounds__(kPeakThreads) peak_ffma_kernel(float* sink, int iters, float seed) {
  float a[kPeakChains];
#pragma unroll
  for (int c = 0; c < kPeakChains; ++c) a[c] = seed + (float)(threadIdx.x + c);
  const float m = 0.9999999f, k = 1e-7f;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int u = 0; u < kPeakUnroll; ++u)
#pragma unroll
      for (int c = 0; c < kPeakChains; ++c) a[c] = __fmaf_rn(a[c], m, k);
  }
  keep(sink, a);
}

// one packed FP32x2 FMA (two lane results) per chain step
__global__ void __launch_bounds__(kPeakThreads) peak_ffma2_kernel(float* sink, int iters, float seed) {
  float2 a[kPeakChains];
#pragma unroll
  for (int c = 0; c < kPeakChains; ++c) a[c] = make_float2(seed + (float)(threadIdx.x + c), seed - (float)c);
  const float2 m = make_float2(0.9999999f, 0.9999998f), k = make_float2(1e-7f, 2e-7f);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int u = 0; u < kPeakUnroll; ++u)
#pragma unroll
      for (int c = 0; c < kPeakChains; ++c) a[c] = __ffma2_rn(a[c], m, k);
  }
  float s[kPeakChains];
#pragma unroll
  for (int c = 0; c < kPeakChains; ++c) s[c] = a[c].x + a[c].y;
  keep(sink, s);
}

// one FP32 min and one max per chain step (the gate and clamp kind of work)
__global__ void __launch_bounds__(kPeakThreads) peak_minmax_kernel(float* sink, int iters, float seed) {
  float a[kPeakChains];
#pragma unroll
  for (int c = 0; c < kPeakChains; ++c) a[c] = seed + (float)(threadIdx.x + c);
  const float lo = seed - 1.0f, hi = seed + 1e6f;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int u = 0; u < kPeakUnroll; ++u)
#pragma unroll
      for (int c = 0; c < kPeakChains; ++c) a[c] = fmaxf(fminf(a[c], hi), lo);
  }
  keep(sink, a);
}

// one ex2 (and one FP32 multiply that keeps the chain bounded) per step
__global__ void __launch_bounds__(kPeakThreads) peak_ex2_kernel(float* sink, int iters, float seed) {
  float a[kPeakChains];
#pragma unroll
  for (int c = 0; c < kPeakChains; ++c) a[c] = seed * 1e-3f + 1e-4f * (float)(threadIdx.x + c);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int u = 0; u < kPeakUnroll; ++u)
#pragma unroll
      for (int c = 0; c < kPeakChains; ++c) a[c] = ex2_op(__fmul_rn(a[c], -0.5f));
  }
  keep(sink, a);
}

// one rcp (and one FP32 add) per step
__global__ void __launch_bounds__(kPeakThreads) peak_rcp_kernel(float* sink, int iters, float seed) {
  float a[kPeakChains];
#pragma unroll
  for (int c = 0; c < kPeakChains; ++c) a[c] = seed * 1e-3f + 1e-4f * (float)(threadIdx.x + c);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int u = 0; u < kPeakUnroll; ++u)
#pragma unroll
      for (int c = 0; c < kPeakChains; ++c) a[c] = rcp_op(__fadd_rn(a[c], 1.0f));
  }
  keep(sink, a);
}

}  // namespace
}  // namespace sr

extern "C" sr_status sr_measure_alu_peaks(void* scratch, sr_alu_peaks* out, void* stream) {
  using namespace sr;
  if (!scratch || !out) return SR_ERR_INVALID;
  if (reinterpret_cast<uintptr_t>(scratch) % 16 != 0) return SR_ERR_INVALID;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) !=
                                                cudaSuccess)
    return SR_ERR_CUDA;
  float* sink = static_cast<float*>(scratch);
  const dim3 grid((unsigned)(sms * 8)), block(kPeakThreads);
  const double threads = (double)grid.x * kPeakThreads;
  const double per_iter = (double)kPeakUnroll * kPeakChains;  // chain steps per thread per iteration
  struct Probe {
    void (*fn)(float*, int, float);
    int iters;
    double ops_per_step;  // counted operations per chain step
    double* dst;
  };
  const Probe probes[5] = {{peak_ffma_kernel, 4096, 1.0, &out->fma_lane_ops_per_s},
                           {peak_ffma2_kernel, 2048, 2.0, &out->ffma2_lane_ops_per_s},
                           {peak_minmax_kernel, 2048, 2.0, &out->minmax_lane_ops_per_s},
                           {peak_ex2_kernel, 512, 1.0, &out->ex2_per_s},
                           {peak_rcp_kernel, 512, 1.0, &out->rcp_per_s}};
  cudaEvent_t ev[2];
  if (cudaEventCreate(&ev[0]) != cudaSuccess) return SR_ERR_CUDA;
  if (cudaEventCreate(&ev[1]) != cudaSuccess) {
    cudaEventDestroy(ev[0]);
    return SR_ERR_CUDA;
  }
  sr_status s = SR_OK;
  out->seconds = 0.0;
  for (const Probe& p : probes) {
    // one untimed launch, then the best of three
    float best = 1e30f;
    for (int rep = 0; rep < 4 && s == SR_OK; ++rep) {
      if (cudaEventRecord(ev[0], st) != cudaSuccess ||
          launch_plain(p.fn, grid, block, 0, st, sink, p.iters, 1.0f + rep) != cudaSuccess ||
          cudaEventRecord(ev[1], st) != cudaSuccess || cudaEventSynchronize(ev[1]) != cudaSuccess) {
        s = SR_ERR_CUDA;
        break;
      }
      count_launches(1);
      float ms = 0.0f;
      if (cudaEventElapsedTime(&ms, ev[0], ev[1]) != cudaSuccess) s = SR_ERR_CUDA;
      if (rep > 0) best = ms < best ? ms : best;
    }
    if (s != SR_OK) break;
    *p.dst = threads * p.iters * per_iter * p.ops_per_step / (best * 1e-3);
    out->seconds += best * 1e-3;
  }
  cudaEventDestroy(ev[0]);
  cudaEventDestroy(ev[1]);
  return s;
}
