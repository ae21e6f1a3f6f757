// FMA-throughput probe (measurement only, not part of the method): the denominator of the
// ALU roofline of the FP64 kernels and of the double-word kernels (FP32 pipes).  Every thread runs
// kChains independent FMA chains, so the pipes see kChains independent instructions per thread
// between dependences; a full device of blocks hides the latency.
#include <cuda_runtime.h>

#include "../../include/xfft.h"

namespace {

constexpr int kChains = 8;

template <typename T>
__global__ void k_fma_probe(T* __restrict__ sink, int iters, T a, T b) {
  T x[kChains];
#pragma unroll
  for (int k = 0; k < kChains; ++k) x[k] = (T)(threadIdx.x + k) * (T)1e-3;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < kChains; ++k) x[k] = fma(x[k], a, b);
  }
  T s = 0;
#pragma unroll
  for (int k = 0; k < kChains; ++k) s += x[k];
  if (s == (T)-1.2345) sink[0] = s;  // never true for these inputs; keeps the chains alive
}

template <typename T>
cudaError_t probe(double* flops, cudaStream_t st) {
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  T* sink = nullptr;
  e = cudaMallocAsync((void**)&sink, sizeof(T), st);
  if (e != cudaSuccess) return e;
  cudaEvent_t t0 = nullptr, t1 = nullptr;
  cudaEventCreate(&t0);
  cudaEventCreate(&t1);
  const int blocks = sms * 8, threads = 256, iters = sizeof(T) == 8 ? 2048 : 16384;
  const T a = (T)0.999999, b = (T)1e-7;
  k_fma_probe<T><<<blocks, threads, 0, st>>>(sink, iters / 8, a, b);  // warm-up
  cudaEventRecord(t0, st);
  k_fma_probe<T><<<blocks, threads, 0, st>>>(sink, iters, a, b);
  cudaEventRecord(t1, st);
  e = cudaEventSynchronize(t1);
  float ms = 0.f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, t0, t1);
  cudaEventDestroy(t0);
  cudaEventDestroy(t1);
  cudaFreeAsync(sink, st);
  cudaStreamSynchronize(st);
  if (e == cudaSuccess) *flops = 2.0 * kChains * (double)iters * blocks * threads / (ms * 1e-3);
  return e;
}

}  // namespace

extern "C" xfft_status xfft_fma_rate(int precision, double* flops_per_s, void* stream) {
  if (!flops_per_s || (precision != XFFT_FP64 && precision != XFFT_FP32_REFINED)) return XFFT_EINVAL;
  const cudaError_t e = precision == XFFT_FP64 ? probe<double>(flops_per_s, (cudaStream_t)stream)
                                               : probe<float>(flops_per_s, (cudaStream_t)stream);
  return e == cudaSuccess ? XFFT_OK : XFFT_ECUDA;
}
