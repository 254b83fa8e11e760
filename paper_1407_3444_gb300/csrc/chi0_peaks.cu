// chi0_peaks.cu -- arithmetic peaks of the GPU the library runs on, measured with CUDA events:
// FP32 and FP64 fused multiply-add on the CUDA cores (independent dependency chains per thread,
// every SM busy) and the 5th-generation tensor cores (chi0_overlap_tc.cu: tcgen05.mma from
// shared memory into tensor memory).  The weight kernels' rooflines are reported against these
// numbers; nothing here changes a GPU setting.
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/chi0.h"
#include "chi0_internal.h"

namespace chi0int {
namespace {

constexpr int kPeakThreads = 256;
constexpr int kChains = 8;  // independent FMA chains per thread (latency x issue width)

template <typename T>
__global__ void __launch_bounds__(kPeakThreads) k_fma_peak(int iters, T a, T b, T *__restrict__ sink) {
  T x[kChains];
#pragma unroll
  for (int i = 0; i < kChains; ++i) x[i] = (T)(threadIdx.x + i) * a;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int u = 0; u < 16; ++u) {
#pragma unroll
      for (int i = 0; i < kChains; ++i) x[i] = fma(x[i], a, b);
    }
  }
  T s = T(0);
#pragma unroll
  for (int i = 0; i < kChains; ++i) s += x[i];
  if (s == T(-12345.678)) sink[blockIdx.x * blockDim.x + threadIdx.x] = s;  // keeps the chains alive
}

template <typename T>
int fma_peak(int iters, int blocks_per_sm, double *tflops, double *ms_out) {
  const int sms = device_sms();
  const int blocks = sms * blocks_per_sm;
  T *sink = nullptr;
  if (cudaMalloc(&sink, sizeof(T) * (size_t)blocks * kPeakThreads) != cudaSuccess) return CHI0_ENOMEM;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  const T a = (T)0.999999, b = (T)1e-7;
  k_fma_peak<T><<<blocks, kPeakThreads>>>(iters / 8 + 1, a, b, sink);  // warm-up
  cudaEventRecord(e0);
  k_fma_peak<T><<<blocks, kPeakThreads>>>(iters, a, b, sink);
  cudaEventRecord(e1);
  const cudaError_t e = cudaEventSynchronize(e1);
  float ms = 0.f;
  cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(sink);
  if (e != cudaSuccess || cudaGetLastError() != cudaSuccess) return CHI0_ECUDA;
  const double flops = 2.0 * 16.0 * kChains * (double)iters * blocks * kPeakThreads;
  *tflops = flops / (ms * 1e-3) / 1e12;
  *ms_out = ms;
  return CHI0_OK;
}

}  // namespace
}  // namespace chi0int

using namespace chi0int;

extern "C" int chi0_peak(int kind, int iters, double *tflops, double *ms) {
  if (!tflops || !ms || iters < 1) return CHI0_EINVAL;
  *tflops = 0.0;
  *ms = 0.0;
  switch (kind) {
    case CHI0_PEAK_FP32_FMA: return fma_peak<float>(iters, 8, tflops, ms);
    case CHI0_PEAK_FP64_FMA: return fma_peak<double>(iters, 8, tflops, ms);
    case CHI0_PEAK_TF32_MMA: return tc_peak(TC_TF32, iters, tflops, ms) == cudaSuccess ? CHI0_OK : CHI0_ECUDA;
    case CHI0_PEAK_BF16_MMA: return tc_peak(TC_BF16X3, iters, tflops, ms) == cudaSuccess ? CHI0_OK : CHI0_ECUDA;
    default: return CHI0_EINVAL;
  }
}
