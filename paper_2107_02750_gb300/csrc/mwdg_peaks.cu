// Measured arithmetic ceilings of the device (mwdg_fma_rate in
// include/mwdg.h): the rate of fused multiply-adds that the FP64 and FP32
// pipes sustain, so that a kernel bound by arithmetic rather than memory can
// be reported against a number taken on the same GPU.
#include <cmath>
#include <cstdint>

#include <cuda_runtime.h>

#include "mwdg.h"

namespace {

constexpr int FMA_TPB = 256;
constexpr int FMA_CHAINS = 8;  // independent accumulators a thread keeps in flight

// FMA_CHAINS independent chains x <- x * a + b per thread, iters times; the
// sum is stored only under a condition that the inputs never meet, so the
// chains are not removed and nothing is written
template <typename T>
__global__ void __launch_bounds__(FMA_TPB) k_fma_chains(T *sink, int iters, T a, T b) {
  T x[FMA_CHAINS];
#pragma unroll
  for (int c = 0; c < FMA_CHAINS; c++) x[c] = (T)(threadIdx.x + c) * (T)1e-3;
  for (int it = 0; it < iters; it++) {
#pragma unroll
    for (int c = 0; c < FMA_CHAINS; c++) x[c] = fma(x[c], a, b);
  }
  T s = T(0);
#pragma unroll
  for (int c = 0; c < FMA_CHAINS; c++) s += x[c];
  if (s == (T)-12345.0) sink[blockIdx.x] = s;
}

template <typename T>
mwdg_status rate(cudaStream_t st, double *out) {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0)
    return MWDG_ERR_CUDA;
  const int blocks = sms * 8;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return MWDG_ERR_CUDA;
  // a<1 and b keep every chain finite
  const T a = (T)0.999, b = (T)1e-3;
  int iters = 256;
  float ms = 0.0f;
  mwdg_status s = MWDG_OK;
  k_fma_chains<T><<<blocks, FMA_TPB, 0, st>>>(nullptr, iters, a, b);  // warm-up
  for (int round = 0; round < 16; round++) {
    cudaEventRecord(e0, st);
    k_fma_chains<T><<<blocks, FMA_TPB, 0, st>>>(nullptr, iters, a, b);
    cudaEventRecord(e1, st);
    if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
      s = MWDG_ERR_CUDA;
      break;
    }
    if (ms >= 20.0f || iters >= (1 << 24)) break;  // long enough that launch overhead is negligible
    iters *= 4;
  }
  if (s == MWDG_OK && cudaGetLastError() != cudaSuccess) s = MWDG_ERR_CUDA;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (s != MWDG_OK) return s;
  const double flops = 2.0 * FMA_CHAINS * (double)iters * (double)blocks * FMA_TPB;
  *out = flops / ((double)ms * 1e-3);
  return MWDG_OK;
}

}  // namespace

extern "C" mwdg_status mwdg_fma_rate(int32_t precision, void *cuda_stream, double *flops_per_s) {
  if (!flops_per_s || (precision != MWDG_F64 && precision != MWDG_F32)) return MWDG_ERR_ARG;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  return precision == MWDG_F64 ? rate<double>(st, flops_per_s) : rate<float>(st, flops_per_s);
}
