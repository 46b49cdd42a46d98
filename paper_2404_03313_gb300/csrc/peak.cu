// The device's FP32 arithmetic rate, measured: the denominator of the ALU
// roofline that the eigen-solve-bound block-dual kernels (k >= 6, the stacked
// layout, SSST) are reported against.  Every thread runs kChains independent
// chains x <- x a + b (enough independent work per warp to cover the FMA
// latency at full occupancy), either as scalar FMAs or as packed FP32x2 FMAs
// (the form the Jacobi rotations use); rate = 2 flops per lane FMA / time.
#include <cuda_runtime.h>

#include "s3ttv.h"

namespace {

constexpr int kChains = 8;   // independent accumulators (packed: pairs) per thread
constexpr int kInner = 64;   // unrolled steps per loop iteration
constexpr int kThreads = 256;
constexpr int kCtasPerSm = 8;

typedef unsigned long long f32x2;
__device__ __forceinline__ f32x2 pack2(float lo, float hi) {
  f32x2 r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
  return r;
}
__device__ __forceinline__ float2 unpack2(f32x2 v) {
  float2 r;
  asm("mov.b64 {%0, %1}, %2;" : "=f"(r.x), "=f"(r.y) : "l"(v));
  return r;
}
__device__ __forceinline__ f32x2 ffma2(f32x2 a, f32x2 b, f32x2 c) {
  f32x2 r;
  asm volatile("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(a), "l"(b), "l"(c));
  return r;
}

// a in (0, 1), b > 0: every chain converges to b / (1 - a), no overflow or
// subnormals; the store never happens for such inputs but keeps the chains live
__global__ void __launch_bounds__(kThreads) fma_scalar_kernel(float *sink, int iters, float a, float b) {
  float x[kChains];
#pragma unroll
  for (int i = 0; i < kChains; ++i) x[i] = 1e-3f * (float)(threadIdx.x + i);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int r = 0; r < kInner; ++r)
#pragma unroll
      for (int i = 0; i < kChains; ++i) asm volatile("fma.rn.f32 %0, %0, %1, %2;" : "+f"(x[i]) : "f"(a), "f"(b));
  }
  float s = 0.f;
#pragma unroll
  for (int i = 0; i < kChains; ++i) s += x[i];
  if (s < 0.f) sink[blockIdx.x] = s;
}

__global__ void __launch_bounds__(kThreads) fma_packed_kernel(float *sink, int iters, float a, float b) {
  f32x2 x[kChains];
#pragma unroll
  for (int i = 0; i < kChains; ++i) x[i] = pack2(1e-3f * (float)(threadIdx.x + i), 2e-3f * (float)(threadIdx.x + i));
  const f32x2 a2 = pack2(a, a), b2 = pack2(b, b);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int r = 0; r < kInner; ++r)
#pragma unroll
      for (int i = 0; i < kChains; ++i) x[i] = ffma2(x[i], a2, b2);
  }
  float s = 0.f;
#pragma unroll
  for (int i = 0; i < kChains; ++i) {
    const float2 v = unpack2(x[i]);
    s += v.x + v.y;
  }
  if (s < 0.f) sink[blockIdx.x] = s;
}

struct Timer {
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  ~Timer() {
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
  }
};

}  // namespace

extern "C" int s3ttv_fp32_peak(int device, int packed, double *tflops) {
  if (!tflops || (packed != 0 && packed != 1)) return S3TTV_EINVAL;
  *tflops = 0.0;
  int prev = -1;
  if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
  if (cudaSetDevice(device) != cudaSuccess) {
    cudaGetLastError();
    return S3TTV_ECUDA;
  }
  int sms = 0;
  float *sink = nullptr;
  cudaStream_t st = nullptr;
  Timer t;
  int rc = S3TTV_OK;
  double flops_per_iter = 0.0;
  float ms = 0.f;
  int iters = 64;
  auto launch = [&](int n) {
    const dim3 grid(sms * kCtasPerSm);
    if (packed) fma_packed_kernel<<<grid, kThreads, 0, st>>>(sink, n, 0.999f, 1e-3f);
    else fma_scalar_kernel<<<grid, kThreads, 0, st>>>(sink, n, 0.999f, 1e-3f);
    return cudaGetLastError();
  };
  do {
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess || sms < 1 ||
        cudaMalloc(&sink, sizeof(float) * sms * kCtasPerSm) != cudaSuccess ||
        cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreate(&t.e0) != cudaSuccess || cudaEventCreate(&t.e1) != cudaSuccess) {
      rc = S3TTV_ECUDA;
      break;
    }
    flops_per_iter = 2.0 * (packed ? 2 : 1) * kChains * kInner * (double)sms * kCtasPerSm * kThreads;
    // warm-up and sizing: grow the loop count until one launch takes >= 20 ms
    bool ok = true;
    for (int round = 0; round < 12; ++round) {
      if (launch(iters) != cudaSuccess || cudaEventRecord(t.e0, st) != cudaSuccess || launch(iters) != cudaSuccess ||
          cudaEventRecord(t.e1, st) != cudaSuccess || cudaEventSynchronize(t.e1) != cudaSuccess ||
          cudaEventElapsedTime(&ms, t.e0, t.e1) != cudaSuccess) {
        ok = false;
        break;
      }
      if (ms >= 20.f || iters >= (1 << 20)) break;
      iters *= ms > 0.5f ? (int)(20.f / ms) + 1 : 16;
      if (iters > (1 << 20)) iters = 1 << 20;
    }
    if (!ok || !(ms > 0.f)) {
      rc = S3TTV_ECUDA;
      break;
    }
    *tflops = flops_per_iter * iters / (ms * 1e-3) / 1e12;
  } while (false);
  if (rc != S3TTV_OK) cudaGetLastError();
  if (st) cudaStreamDestroy(st);
  if (sink) cudaFree(sink);
  if (prev >= 0) cudaSetDevice(prev);
  return rc;
}
