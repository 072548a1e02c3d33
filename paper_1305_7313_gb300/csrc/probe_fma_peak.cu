// probe_fma_peak.cu — a stand-alone program (not part of libfockx.so) that
// measures the FP64 and FP32 fused multiply-add throughput of the current GPU:
// the denominators of the FP64 and double-float forms' rooflines, which are
// bound by arithmetic, not by memory.
//
// Every thread runs K independent FMA chains for `iters` iterations and makes
// one store (out has exactly grid * block elements); no waits, no shared
// memory.  Flops = 2 * threads * iters * K per launch, timed with CUDA events
// over 5 launches after 3 warm-up launches.
//
//   nvcc -gencode arch=compute_103a,code=sm_103a -O3 -o /tmp/probe_fma_peak \
//       paper_1305_7313_gb300/csrc/probe_fma_peak.cu && /tmp/probe_fma_peak
#include <cstdio>
#include <cuda_runtime.h>

template <class T, int K>
__global__ void fma_loop(T* out, int iters, T a, T b) {
  T acc[K];
#pragma unroll
  for (int k = 0; k < K; ++k) acc[k] = T(threadIdx.x + k);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < K; ++k) acc[k] = fma(acc[k], a, b);
  }
  T s = 0;
#pragma unroll
  for (int k = 0; k < K; ++k) s += acc[k];
  out[(size_t)blockIdx.x * blockDim.x + threadIdx.x] = s;
}

template <class T, int K>
double run(int blocks, int threads, int iters) {
  T* out;
  size_t n = (size_t)blocks * threads;
  if (cudaMalloc(&out, n * sizeof(T)) != cudaSuccess) return -1;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  for (int w = 0; w < 3; ++w) fma_loop<T, K><<<blocks, threads>>>(out, iters, T(0.999999), T(1e-7));
  cudaEventRecord(e0);
  const int reps = 5;
  for (int r = 0; r < reps; ++r) fma_loop<T, K><<<blocks, threads>>>(out, iters, T(0.999999), T(1e-7));
  cudaEventRecord(e1);
  cudaEventSynchronize(e1);
  float ms = 0;
  cudaEventElapsedTime(&ms, e0, e1);
  cudaError_t err = cudaGetLastError();
  cudaFree(out);
  if (err != cudaSuccess) {
    printf("error %s\n", cudaGetErrorString(err));
    return -1;
  }
  double flops = 2.0 * n * (double)iters * K * reps;
  return flops / (ms * 1e-3) / 1e12;
}

int main() {
  int dev = 0, sms = 0, clk = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaDeviceGetAttribute(&clk, cudaDevAttrClockRate, dev);
  printf("SMs %d, max clock %d kHz\n", sms, clk);
  for (int per_sm : {4, 8, 16}) {
    const double n = (double)sms * per_sm * 256;
    const int iters = (int)(1.2e11 / (n * 16));  // ~0.1 s per launch at 1.2 TFLOP/s
    double t = run<double, 8>(sms * per_sm, 256, iters);
    printf("fp64 dfma: blocks %d x 256 threads, 8 chains: %.4f TFLOP/s\n", sms * per_sm, t);
  }
  for (int per_sm : {4, 8}) {
    const double n = (double)sms * per_sm * 256;
    const int iters = (int)(8e12 / (n * 16));  // ~0.1 s per launch at 80 TFLOP/s
    double t = run<float, 8>(sms * per_sm, 256, iters);
    printf("fp32 ffma: blocks %d x 256 threads, 8 chains: %.3f TFLOP/s\n", sms * per_sm, t);
  }
  return 0;
}
