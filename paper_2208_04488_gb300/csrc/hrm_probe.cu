// FMA-pipe throughput probe: the denominator of the ALU roofline of the
// per-midpoint kernels. Independent FMA chains per thread, enough warps to
// fill every SM; flops = 2 x FMAs.
#include <cuda_runtime.h>

#include "../../include/hrm.h"

namespace {

constexpr int kChains = 8;

template <typename T>
__global__ void __launch_bounds__(256) k_fma(T* out, int iters, T a, T b) {
  T x[kChains];
#pragma unroll
  for (int i = 0; i < kChains; ++i) x[i] = T(threadIdx.x + i) * T(1e-3);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int i = 0; i < kChains; ++i) x[i] = fma(x[i], a, b);
  }
  T s = T(0);
#pragma unroll
  for (int i = 0; i < kChains; ++i) s += x[i];
  if (s == T(-1234.5)) out[0] = s;  // keeps the chains live; never true for these inputs
}

template <typename T>
hrm_status run(int iters, cudaStream_t s, double* flops_per_s) {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return HRM_E_CUDA;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int blocks = sms * 8, threads = 256;
  T* out = nullptr;
  if (cudaMallocAsync(&out, sizeof(T), s) != cudaSuccess) return HRM_E_NOMEM;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  k_fma<T><<<blocks, threads, 0, s>>>(out, iters / 4 + 1, T(0.999999), T(1e-7));
  cudaEventRecord(e0, s);
  k_fma<T><<<blocks, threads, 0, s>>>(out, iters, T(0.999999), T(1e-7));
  cudaEventRecord(e1, s);
  cudaEventSynchronize(e1);
  float ms = 0.f;
  cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFreeAsync(out, s);
  const cudaError_t err = cudaStreamSynchronize(s);
  if (err != cudaSuccess || ms <= 0.f) return HRM_E_CUDA;
  *flops_per_s = 2.0 * kChains * (double)iters * blocks * threads / (ms * 1e-3);
  return HRM_OK;
}

}  // namespace

extern "C" hrm_status hrm_probe_fma_peak(int32_t precision, int32_t iters, void* stream, double* flops_per_s) {
  if (!flops_per_s || iters <= 0) return HRM_E_INVAL;
  cudaStream_t s = (cudaStream_t)stream;
  return precision == HRM_FP32 ? run<float>(iters, s, flops_per_s) : run<double>(iters, s, flops_per_s);
}
