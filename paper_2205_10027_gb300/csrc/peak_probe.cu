// Throughput probe of the FP64 pipe (the roofline denominator of the FP64 form): every
// thread runs eight independent FMA chains in registers.
#include <cmath>
#include "engine.h"

namespace glasso {
namespace {
__global__ void k_fma_chains(double* out, int iters, double a, double b) {
  double acc[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) acc[i] = threadIdx.x * 1e-3 + i;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int i = 0; i < 8; ++i) acc[i] = fma(acc[i], a, b);
  }
  double s = 0.0;
#pragma unroll
  for (int i = 0; i < 8; ++i) s += acc[i];
  out[(int64_t)blockIdx.x * blockDim.x + threadIdx.x] = s;
}
}  // namespace

double probe_fp64_tflops(int device) {
  CUDA_CHECK(cudaSetDevice(device));
  cudaDeviceProp prop;
  CUDA_CHECK(cudaGetDeviceProperties(&prop, device));
  const int blocks = prop.multiProcessorCount * 8, threads = 256, iters = 4096;
  double* out = nullptr;
  CUDA_CHECK(cudaMalloc(&out, sizeof(double) * blocks * threads));
  cudaEvent_t e0, e1;
  CUDA_CHECK(cudaEventCreate(&e0));
  CUDA_CHECK(cudaEventCreate(&e1));
  float best = 1e30f;
  for (int rep = 0; rep < 4; ++rep) {
    CUDA_CHECK(cudaEventRecord(e0));
    k_fma_chains<<<blocks, threads>>>(out, iters, 0.9999, 1e-7);
    LAUNCH_CHECK();
    CUDA_CHECK(cudaEventRecord(e1));
    CUDA_CHECK(cudaEventSynchronize(e1));
    float ms = 0.f;
    CUDA_CHECK(cudaEventElapsedTime(&ms, e0, e1));
    if (rep > 0) best = std::fmin(best, ms);
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(out);
  const double flops = 2.0 * 8 * iters * (double)blocks * threads;
  return flops / (best * 1e-3) / 1e12;
}
}  // namespace glasso
