// hosc_fp64_peak: the FP64 arithmetic rate of the GPU, measured (the denominator of the roofline of
// the all-FP64 sweep kernels, whose bound is the FP64 pipe, not memory). Every thread of a grid of
// 8 blocks of 256 threads per SM runs eight independent chains of fused multiply-adds on
// registers; 2 flops per FMA. The chains feed back into themselves, so the compiler keeps every
// FMA, and one store per thread keeps the result live.

#include <cuda_runtime.h>

#include "hosc.h"
#include "hosc_internal.h"

namespace {

constexpr int kChains = 8;
constexpr int kPeakThreads = 256;

__global__ void __launch_bounds__(kPeakThreads) k_fp64_fma(double* out, int iters, double a,
                                                           double b) {
  double x[kChains];
#pragma unroll
  for (int q = 0; q < kChains; ++q) x[q] = (double)(threadIdx.x + q) * 1e-3;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int q = 0; q < kChains; ++q) x[q] = fma(x[q], a, b);
  }
  double s = 0.0;
#pragma unroll
  for (int q = 0; q < kChains; ++q) s += x[q];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace

extern "C" hosc_status hosc_fp64_peak(int reps, double* tflops_out) {
  if (reps < 1 || !tflops_out) return HOSC_EINVAL;
  const int sms = hosc::device_sms();
  if (sms < 1) return HOSC_ECUDA;
  const int blocks = 8 * sms, iters = 1 << 14;
  double* out = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  hosc_status st = HOSC_ECUDA;
  if (cudaMalloc(&out, (size_t)blocks * kPeakThreads * sizeof(double)) == cudaSuccess &&
      cudaEventCreate(&e0) == cudaSuccess && cudaEventCreate(&e1) == cudaSuccess) {
    // a = 1 - 2^-30, b = 2^-40: the chains stay finite and non-trivial for any iteration count
    const double a = 1.0 - 0x1p-30, b = 0x1p-40;
    k_fp64_fma<<<blocks, kPeakThreads>>>(out, iters, a, b);   // warm-up
    cudaEventRecord(e0);
    for (int r = 0; r < reps; ++r) k_fp64_fma<<<blocks, kPeakThreads>>>(out, iters, a, b);
    cudaEventRecord(e1);
    float ms = 0.f;
    if (cudaEventSynchronize(e1) == cudaSuccess && cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess &&
        ms > 0.f) {
      const double flops = 2.0 * kChains * (double)iters * blocks * kPeakThreads * reps;
      *tflops_out = flops / (ms * 1e-3) / 1e12;
      st = HOSC_OK;
    }
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (out) cudaFree(out);
  cudaGetLastError();
  return st;
}
