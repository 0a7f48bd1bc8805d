// FP64 fused multiply-add throughput of this device: the denominator of the
// narrow phase's roofline fraction.  Each thread runs 8 independent DFMA
// chains so that issue, not latency, bounds the kernel.

#include <cstdio>

#include "ccd_kernels.cuh"

namespace {

constexpr int kChains = 8;
constexpr int kIters = 4096;

__global__ void k_dfma_chains(double *out, double a, double b) {
  double x[kChains];
#pragma unroll
  for (int i = 0; i < kChains; ++i) x[i] = threadIdx.x * 1e-3 + i;
  for (int it = 0; it < kIters; ++it) {
#pragma unroll
    for (int i = 0; i < kChains; ++i) x[i] = fma(x[i], a, b);
  }
  double s = 0;
#pragma unroll
  for (int i = 0; i < kChains; ++i) s += x[i];
  if (s == 12345.678) out[0] = s;   // keeps the chains live
}

}  // namespace

extern "C" int ccd_measure_fp64_peak(int device, double *gflops) {
  if (!gflops) return CCD_EINVAL;
  if (cudaSetDevice(device) != cudaSuccess) return CCD_ECUDA;
  cudaDeviceProp p;
  if (cudaGetDeviceProperties(&p, device) != cudaSuccess) return CCD_ECUDA;
  double *out = nullptr;
  if (cudaMalloc(&out, sizeof(double)) != cudaSuccess) return CCD_ENOMEM;
  const int threads = 256, blocks = p.multiProcessorCount * 8;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  k_dfma_chains<<<blocks, threads>>>(out, 0.999999, 1e-7);   // warm-up
  float best = 1e30f;
  for (int r = 0; r < 5; ++r) {
    cudaEventRecord(e0);
    k_dfma_chains<<<blocks, threads>>>(out, 0.999999, 1e-7);
    cudaEventRecord(e1);
    cudaEventSynchronize(e1);
    float ms = 0;
    cudaEventElapsedTime(&ms, e0, e1);
    best = ms < best ? ms : best;
  }
  cudaError_t err = cudaGetLastError();
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(out);
  if (err != cudaSuccess) return CCD_ECUDA;
  double flops = 2.0 * kChains * (double)kIters * threads * (double)blocks;
  *gflops = flops / (best * 1e-3) / 1e9;
  return CCD_OK;
}
