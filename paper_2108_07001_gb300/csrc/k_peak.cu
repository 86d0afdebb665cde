// FP32 arithmetic peak of this GPU, measured: every SM filled with warps
// that run independent FMA chains, in the scalar form (fma.rn.f32) and the
// packed-pair form (fma.rn.f32x2).  The ALU-bound kernels of the chain are
// reported against the larger of the two.
#include <cuda_runtime.h>

#include "../../include/rx.h"
#include "rx_internal.cuh"

namespace rx {

constexpr int kPeakChains = 8;      // independent chains per thread
constexpr int kPeakThreads = 256;

__global__ void __launch_bounds__(kPeakThreads) fma_peak_kernel(float* out, int iters, float a, float b) {
  float x[kPeakChains];
#pragma unroll
  for (int j = 0; j < kPeakChains; ++j) x[j] = (float)(threadIdx.x + j);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int j = 0; j < kPeakChains; ++j) x[j] = fmaf(x[j], a, b);
  }
  float s = 0.f;
#pragma unroll
  for (int j = 0; j < kPeakChains; ++j) s += x[j];
  if (s == 1.2345f) out[blockIdx.x] = s;  // keeps the chains live; never true for these inputs
}

__global__ void __launch_bounds__(kPeakThreads) fma2_peak_kernel(float* out, int iters, float a, float b) {
  unsigned long long x[kPeakChains];
#pragma unroll
  for (int j = 0; j < kPeakChains; ++j) x[j] = f2pk((float)(threadIdx.x + j), (float)(threadIdx.x - j));
  const unsigned long long A = f2pk(a, a), B = f2pk(b, b);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int j = 0; j < kPeakChains; ++j) x[j] = f2fma(x[j], A, B);
  }
  float s = 0.f;
#pragma unroll
  for (int j = 0; j < kPeakChains; ++j) {
    float lo, hi;
    f2up(x[j], lo, hi);
    s += lo + hi;
  }
  if (s == 1.2345f) out[blockIdx.x] = s;
}

}  // namespace rx

extern "C" int rx_fp32_peak(int device, double* tflops_fma, double* tflops_fma2) {
  if (!tflops_fma || !tflops_fma2) return RX_EINVAL;
  cudaDeviceProp prop;
  if (cudaSetDevice(device) != cudaSuccess || cudaGetDeviceProperties(&prop, device) != cudaSuccess) {
    cudaGetLastError();
    return RX_EDEVICE;
  }
  const int blocks = prop.multiProcessorCount * 8;  // 2048 threads per SM
  const int iters = 4096;
  float* out = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e = cudaMalloc(&out, blocks * sizeof(float));
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  // a, b keep every value finite: x -> 0.5 x + 0.25 converges to 0.5
  double best[2] = {0.0, 0.0};
  for (int form = 0; form < 2 && e == cudaSuccess; ++form) {
    for (int rep = 0; rep < 8 && e == cudaSuccess; ++rep) {
      e = cudaEventRecord(e0, 0);
      if (form == 0) rx::fma_peak_kernel<<<blocks, rx::kPeakThreads>>>(out, iters, 0.5f, 0.25f);
      else rx::fma2_peak_kernel<<<blocks, rx::kPeakThreads>>>(out, iters, 0.5f, 0.25f);
      if (e == cudaSuccess) e = cudaGetLastError();
      if (e == cudaSuccess) e = cudaEventRecord(e1, 0);
      if (e == cudaSuccess) e = cudaEventSynchronize(e1);
      float ms = 0.f;
      if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
      if (e == cudaSuccess && rep >= 2 && ms > 0.f) {
        const double flops = (double)blocks * rx::kPeakThreads * iters * rx::kPeakChains * 2.0 * (form ? 2.0 : 1.0);
        const double tf = flops / (ms * 1e-3) / 1e12;
        if (tf > best[form]) best[form] = tf;
      }
    }
  }
  if (out) cudaFree(out);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (e != cudaSuccess) return RX_EDEVICE;
  *tflops_fma = best[0];
  *tflops_fma2 = best[1];
  return RX_OK;
}
