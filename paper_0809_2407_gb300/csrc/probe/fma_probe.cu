// Measured issue rate of the FP64 and FP32 fused multiply-add pipes of the current GPU: the
// denominators of the rooflines of the kernels bound by those pipes (the TSQR factorization and
// the FP32-storage and double-float forms).  Measurement tooling; the paper has no counterpart.
//
// Every thread runs 8 independent FMA chains x <- x a + b (a just below 1, so the values stay
// bounded) for `iters` iterations; the grid fills every SM with 8 blocks of 256 threads.  The rate
// is 2 flops x 8 chains x iters x threads over the CUDA-event time of the second of two launches.
#include <cuda_runtime.h>
#include <stdint.h>

namespace {

template <class T>
__global__ void __launch_bounds__(256) fma_chains(T* sink, int64_t iters, T a, T b) {
  T x[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) x[i] = (T)(threadIdx.x + 1) * (T)1e-3 + (T)i;
  for (int64_t it = 0; it < iters; ++it) {
#pragma unroll
    for (int i = 0; i < 8; ++i) x[i] = fma(x[i], a, b);
  }
  T s = 0;
#pragma unroll
  for (int i = 0; i < 8; ++i) s += x[i];
  if (s == (T)-1.5) sink[blockIdx.x] = s;  // never true; keeps the chains live
}

template <class T>
int run(int64_t iters, double* tflops, int blocks_per_sm = 8, int threads = 256) {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 1;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 1;
  const int blocks = sms * blocks_per_sm;
  T* sink = nullptr;
  if (cudaMalloc(&sink, sizeof(T) * blocks) != cudaSuccess) return 1;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  float ms = 0.f;
  for (int rep = 0; rep < 2; ++rep) {
    cudaEventRecord(e0);
    fma_chains<T><<<blocks, threads>>>(sink, iters, (T)0.9999999, (T)1e-7);
    cudaEventRecord(e1);
    cudaEventSynchronize(e1);
    cudaEventElapsedTime(&ms, e0, e1);
  }
  const cudaError_t err = cudaGetLastError();
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(sink);
  if (err != cudaSuccess || ms <= 0.f) return 1;
  *tflops = 2.0 * 8.0 * (double)iters * (double)blocks * (double)threads / (ms * 1e-3) / 1e12;
  return 0;
}

}  // namespace

// FMA rate in TFLOP/s of FP64 (fp32 == 0) or FP32 (fp32 != 0) on the current device; 0 on success.
extern "C" int tsqr_probe_fma_tflops(int fp32, long long iters, double* tflops) {
  if (!tflops || iters < 1) return 1;
  return fp32 ? run<float>(iters, tflops) : run<double>(iters, tflops);
}

// The same with `warps` warps on each SM (one block of 32 * warps threads per SM): how the rate
// grows with the number of warps issuing, i.e. what one warp alone can issue.  0 on success.
extern "C" int tsqr_probe_fma_tflops_warps(int fp32, int warps, long long iters, double* tflops) {
  if (!tflops || iters < 1 || warps < 1 || warps > 32) return 1;
  return fp32 ? run<float>(iters, tflops, 1, 32 * warps) : run<double>(iters, tflops, 1, 32 * warps);
}
