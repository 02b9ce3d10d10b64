// fbs_peaks.cu -- throughput of the arithmetic pipes that the sweep kernels
// use, measured on the current device with CUDA events (fbs_measure_peaks in
// include/fbs.h): FP32 fused multiply-add, the MUFU base-2 exponential and
// logarithm approximations (ex2.approx, lg2.approx: what expf/__logf reduce
// to), 32-bit integer multiply-high (the Philox rounds) and FP64 fused
// multiply-add.  These are the denominators of the sweep's arithmetic
// roofline.  Nothing here changes a clock or any other device setting.
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "fbs.h"
#include "fbs_kernels.h"

namespace fbs {
namespace {

constexpr int kChains = 8;      // independent dependency chains per thread
constexpr int kThreads = 256;
constexpr int kBlocksPerSm = 8;

enum : int { kOpFfma = 0, kOpEx2 = 1, kOpLg2 = 2, kOpImulhi = 3, kOpDfma = 4, kNumOps = 5 };

__device__ __forceinline__ float ex2_approx(float x) {
  float y;
  asm volatile("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

__device__ __forceinline__ float lg2_approx(float x) {
  float y;
  asm volatile("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// Every thread runs kChains independent chains of `iters` operations of kind
// OP; the result is stored only under a condition the values never meet, so
// that the compiler keeps the work without adding memory traffic.
template <int OP>
__global__ void __launch_bounds__(kThreads) k_peak(int iters, float* sink) {
  const int tid = blockIdx.x * blockDim.x + threadIdx.x;
  if (OP == kOpDfma) {
    double x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = 1.0 + 1e-3 * (double)(tid + c);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
      for (int c = 0; c < kChains; ++c) x[c] = fma(x[c], 0.999999, 1e-7);
    }
    double s = 0.0;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += x[c];
    if (s == -1.0) sink[tid] = (float)s;
  } else if (OP == kOpImulhi) {
    uint32_t x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = 0x9E3779B9u * (uint32_t)(tid + c + 1);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
      for (int c = 0; c < kChains; ++c) x[c] = __umulhi(x[c], 0xD2511F53u) ^ (uint32_t)i;
    }
    uint32_t s = 0;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s ^= x[c];
    if (s == 0x12345678u) sink[tid] = (float)s;
  } else {
    float x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = 0.5f + 1e-3f * (float)((tid + c) & 255);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
      for (int c = 0; c < kChains; ++c) {
        if (OP == kOpFfma) x[c] = fmaf(x[c], 0.9999f, 1e-4f);
        else if (OP == kOpEx2) x[c] = ex2_approx(-x[c]);   // stays in (1/2, 1)
        else x[c] = lg2_approx(x[c] + 2.0f);              // stays in (1.58, 2)
      }
    }
    float s = 0.0f;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += x[c];
    if (s == -1.0f) sink[tid] = s;
  }
}

template <int OP>
cudaError_t time_op(int blocks, int iters, float* sink, cudaEvent_t a, cudaEvent_t b,
                    double* ops_per_s) {
  k_peak<OP><<<blocks, kThreads>>>(iters, sink);  // warm-up
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  float best = 1e30f;
  for (int r = 0; r < 3; ++r) {
    cudaEventRecord(a, 0);
    k_peak<OP><<<blocks, kThreads>>>(iters, sink);
    cudaEventRecord(b, 0);
    if ((e = cudaEventSynchronize(b)) != cudaSuccess) return e;
    float ms = 0.0f;
    if ((e = cudaEventElapsedTime(&ms, a, b)) != cudaSuccess) return e;
    if (ms < best) best = ms;
  }
  const double ops = (double)blocks * kThreads * kChains * (double)iters;
  *ops_per_s = ops / (best * 1e-3);
  return cudaSuccess;
}

}  // namespace
}  // namespace fbs

extern "C" int fbs_measure_peaks(double* out) {
  using namespace fbs;
  if (!out) {
    set_last_error("out is NULL");
    return FBS_E_ARG;
  }
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  float* sink = nullptr;
  const int blocks = sms * kBlocksPerSm;
  if (e == cudaSuccess) e = cudaMalloc((void**)&sink, sizeof(float) * (size_t)blocks * kThreads);
  cudaEvent_t a = nullptr, b = nullptr;
  if (e == cudaSuccess) e = cudaEventCreate(&a);
  if (e == cudaSuccess) e = cudaEventCreate(&b);
  // operations per launch: about 1e10 FP32 FMA, 2.5e9 MUFU or integer, 2.5e8 FP64
  if (e == cudaSuccess) e = time_op<kOpFfma>(blocks, 4096, sink, a, b, &out[0]);
  if (e == cudaSuccess) e = time_op<kOpEx2>(blocks, 1024, sink, a, b, &out[1]);
  if (e == cudaSuccess) e = time_op<kOpLg2>(blocks, 1024, sink, a, b, &out[2]);
  if (e == cudaSuccess) e = time_op<kOpImulhi>(blocks, 1024, sink, a, b, &out[3]);
  if (e == cudaSuccess) e = time_op<kOpDfma>(blocks, 128, sink, a, b, &out[4]);
  if (a) cudaEventDestroy(a);
  if (b) cudaEventDestroy(b);
  if (sink) cudaFree(sink);
  if (e != cudaSuccess) {
    set_last_error(std::string("fbs_measure_peaks: ") + cudaGetErrorString(e));
    return FBS_E_CUDA;
  }
  return FBS_OK;
}
