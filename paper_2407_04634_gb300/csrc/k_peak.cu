// ns_fma_peak: measured FMA throughput of the device's FP64 and FP32 pipes.  The
// FP64 path of the method is bound by the FP64 pipe (its dense products have more
// flops per byte than that pipe's ridge point), so its roofline needs this rate as
// a measured number rather than a datasheet one.
#include <algorithm>

#include "../../include/nullspace.h"
#include "ns_common.cuh"

namespace {

constexpr int kChains = 8;   // independent FMA chains per thread
constexpr int kUnroll = 16;  // FMAs of each chain per loop trip

// Every thread runs kChains independent dependency chains a <- a * b + c.  With
// 8 chains per thread and 8+ warps per scheduler the pipe, not the latency of one
// chain, sets the rate.  The final sum is written only for an impossible value so
// the chains stay live without a store per thread.
template <typename T>
__global__ void __launch_bounds__(256) k_fma_peak(T* out, T b, T c, int iters) {
  T a[kChains];
#pragma unroll
  for (int i = 0; i < kChains; ++i) a[i] = (T)(threadIdx.x + 1) * (T)1e-7 + (T)i;
  for (int k = 0; k < iters; ++k) {
#pragma unroll
    for (int u = 0; u < kUnroll; ++u)
#pragma unroll
      for (int i = 0; i < kChains; ++i) a[i] = fma(a[i], b, c);
  }
  T s = 0;
#pragma unroll
  for (int i = 0; i < kChains; ++i) s += a[i];
  if (s == (T)-1.25e30) out[blockIdx.x] = s;
}

template <typename T>
cudaError_t measure(double* tflops) {
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  const int grid = sms * 8, block = 256;  // 8 resident CTAs of 256 threads per SM
  // about 50 ms per launch at the expected rates (FP64 ~1.2 TFLOP/s, FP32 ~70 TFLOP/s)
  const int iters = sizeof(T) == 8 ? 1500 : 60000;
  T* out = nullptr;
  e = cudaMalloc(&out, sizeof(T) * grid);
  if (e != cudaSuccess) return e;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  float best = 1e30f;
  for (int rep = 0; rep < 4; ++rep) {  // the first launch is a warm-up
    cudaEventRecord(e0);
    k_fma_peak<T><<<grid, block>>>(out, (T)0.9999999, (T)1e-9, iters);
    cudaEventRecord(e1);
    e = cudaEventSynchronize(e1);
    if (e != cudaSuccess) break;
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (rep > 0) best = std::min(best, ms);
  }
  if (e == cudaSuccess) e = cudaGetLastError();
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(out);
  if (e != cudaSuccess) return e;
  const double fmas = (double)grid * block * iters * kUnroll * kChains;
  *tflops = 2.0 * fmas / (best * 1e-3) / 1e12;
  return cudaSuccess;
}

}  // namespace

extern "C" ns_status ns_fma_peak(int precision, double* tflops) {
  if (!tflops || (precision != NS_FP64 && precision != NS_MIXED)) return NS_ERR_INVALID_ARG;
  const cudaError_t e = precision == NS_FP64 ? measure<double>(tflops) : measure<float>(tflops);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return NS_ERR_CUDA;
  }
  return NS_OK;
}
