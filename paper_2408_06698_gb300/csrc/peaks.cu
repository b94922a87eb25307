// Measured fused multiply-add throughput of the current device, FP32 and FP64: the
// denominators of the arithmetic roofline of the kernels (which are bound by the FMA
// pipes, not by HBM).  Every thread runs 8 independent chains x <- x b + c (b, c passed at
// run time, |b| < 1 keeps x bounded); a full-occupancy grid of 8 CTAs of 256 threads per
// SM keeps every scheduler issuing.  flop = 2 x chains x 16 x iters x threads.
#include <cuda_runtime.h>

#include "../../include/hopu.h"

namespace {

constexpr int kChains = 8, kInner = 16, kThreads = 256, kBlocksPerSm = 8;

template <typename T>
__global__ void __launch_bounds__(kThreads) k_fma_chains(int iters, T b, T c, T* sink) {
  T x[kChains];
#pragma unroll
  for (int j = 0; j < kChains; ++j) x[j] = T(threadIdx.x + j) * T(1e-3);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int r = 0; r < kInner; ++r)
#pragma unroll
      for (int j = 0; j < kChains; ++j) x[j] = fma(x[j], b, c);
  }
  T s = T(0);
#pragma unroll
  for (int j = 0; j < kChains; ++j) s += x[j];
  if (s == T(-1234.5)) sink[0] = s;  // never true; keeps the chains live
}

template <typename T>
cudaError_t run(int iters, double* tflops) {
  int dev = 0, nsm = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  T* sink = nullptr;
  cudaStream_t st = nullptr;
  cudaEvent_t a = nullptr, b = nullptr;
  float ms = 0.f;
  const int grid = nsm * kBlocksPerSm;
  if ((e = cudaMalloc(&sink, sizeof(T))) != cudaSuccess) return e;
  if ((e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking)) == cudaSuccess &&
      (e = cudaEventCreate(&a)) == cudaSuccess && (e = cudaEventCreate(&b)) == cudaSuccess) {
    k_fma_chains<T><<<grid, kThreads, 0, st>>>(iters, T(0.999), T(1e-3), sink);  // warm-up
    cudaEventRecord(a, st);
    k_fma_chains<T><<<grid, kThreads, 0, st>>>(iters, T(0.999), T(1e-3), sink);
    cudaEventRecord(b, st);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaEventSynchronize(b);
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, a, b);
  }
  if (a) cudaEventDestroy(a);
  if (b) cudaEventDestroy(b);
  if (st) cudaStreamDestroy(st);
  cudaFree(sink);
  if (e != cudaSuccess) return e;
  const double flop = 2.0 * kChains * kInner * double(iters) * double(grid) * kThreads;
  *tflops = ms > 0.f ? flop / (double(ms) * 1e-3) / 1e12 : 0.0;
  return cudaSuccess;
}

}  // namespace

extern "C" hopu_status hopu_measure_alu_peak(int fp64, int iters, double* tflops) {
  if (!tflops || iters <= 0) return HOPU_EINVAL;
  const cudaError_t e = fp64 ? run<double>(iters, tflops) : run<float>(iters, tflops);
  return e == cudaSuccess ? HOPU_OK : HOPU_ECUDA;
}
