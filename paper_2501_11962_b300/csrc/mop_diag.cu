// Measured FP32 FMA throughput of the device, the denominator the pair kernels are compared
// with beside the nominal lanes x clock figure.  Every thread runs kChains independent FMA
// chains (x <- a x + b), enough to hide the FMA latency at full occupancy; the grid is a
// multiple of the SM count.
#include <cuda_runtime.h>

#include <cmath>

#include "../../include/mop.h"

namespace {

constexpr int kChains = 8;
constexpr int kUnroll = 16;
constexpr int kThreads = 256;

__global__ void __launch_bounds__(kThreads) k_fma_peak(float* out, int iters, float a, float b) {
  float x[kChains];
#pragma unroll
  for (int k = 0; k < kChains; ++k) x[k] = 1e-3f * (float)(threadIdx.x + k);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int r = 0; r < kUnroll; ++r)
#pragma unroll
      for (int k = 0; k < kChains; ++k) x[k] = fmaf(x[k], a, b);
  }
  float s = 0.f;
#pragma unroll
  for (int k = 0; k < kChains; ++k) s += x[k];
  if (s == -1.f) out[blockIdx.x * kThreads + threadIdx.x] = s;   // keeps the chains live
}

}  // namespace

extern "C" mop_status mop_measure_fp32_peak(int32_t device, double* tflops) {
  if (!tflops) return MOP_ERR_ARG;
  int prev = 0;
  if (cudaGetDevice(&prev) != cudaSuccess || cudaSetDevice(device) != cudaSuccess) {
    cudaGetLastError();
    return MOP_ERR_CUDA;
  }
  int sms = 0, per_sm = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_fma_peak, kThreads, 0);
  if (sms <= 0 || per_sm <= 0) {
    cudaSetDevice(prev);
    return MOP_ERR_CUDA;
  }
  const int blocks = sms * per_sm;
  const int iters = 20000;
  float* out = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  mop_status st = MOP_OK;
  float best = 0.f;
  if (cudaMalloc(&out, sizeof(float) * (size_t)blocks * kThreads) != cudaSuccess) {
    st = MOP_ERR_OOM;
  } else if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    st = MOP_ERR_CUDA;
  } else {
    k_fma_peak<<<blocks, kThreads>>>(out, iters / 10, 0.999999f, 1e-7f);   // warm-up
    for (int rep = 0; rep < 3 && st == MOP_OK; ++rep) {
      cudaEventRecord(e0);
      k_fma_peak<<<blocks, kThreads>>>(out, iters, 0.999999f, 1e-7f);
      cudaEventRecord(e1);
      float ms = 0.f;
      if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess || !(ms > 0.f))
        st = MOP_ERR_CUDA;
      else if (best == 0.f || ms < best)
        best = ms;
    }
  }
  if (st == MOP_OK) {
    const double flops = 2.0 * kChains * kUnroll * (double)iters * blocks * kThreads;
    *tflops = flops / (best * 1e-3) / 1e12;
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (out) cudaFree(out);
  cudaGetLastError();
  cudaSetDevice(prev);
  return st;
}
