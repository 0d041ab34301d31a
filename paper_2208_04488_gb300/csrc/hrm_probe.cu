// Diagnostics, not steps of the method. The FMA-pipe throughput probe: the
// denominator of the ALU roofline of the per-midpoint kernels (independent FMA
// chains per thread, enough warps to fill every SM; flops = 2 x FMAs). The
// wait probe: the bounded mbarrier wait of the tensor-core kernels, made to run
// out on a phase that nothing completes.
#include <cuda_runtime.h>

#include "../../include/hrm.h"
#include "hrm_device.cuh"
#include "hrm_sync.cuh"
#include "hrm_tc.cuh"

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

// One CTA of 128 threads waits on phase 0 of a fresh mbarrier (count 1) that
// nothing arrives at, with the library's bounded wait; each wait that runs out
// is counted.
__global__ void __launch_bounds__(128) k_wait_probe(unsigned long long* expired) {
  __shared__ unsigned long long bar;
  if (threadIdx.x == 0) hrm::tc::bar_init(hrm::tc::smem_u32(&bar));
  __syncthreads();
  if (!hrm::tc::bar_wait(hrm::tc::smem_u32(&bar), 0u)) atomicAdd(expired, 1ull);
}

// The integer-pipe conversions of the precision form, element by element.
__global__ void k_convert(const double* in_d, const float* in_f, int64_t n, float* narrowed, double* widened) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  narrowed[i] = hrm::narrow_f64(in_d[i]);
  widened[i] = hrm::widen_f32(in_f[i]);
}

// Blocks waiting at a grid barrier that counts one block more than launched.
__global__ void __launch_bounds__(128) k_barrier_probe(hrm::GridSync* s, uint64_t limit_ns) {
  hrm::grid_barrier(s, gridDim.x + 1u, limit_ns);
}

}  // namespace

extern "C" hrm_status hrm_probe_barrier_timeout(void* stream, double limit_ms, int64_t* expired) {
  if (!expired || !(limit_ms > 0.0) || limit_ms > 10000.0) return HRM_E_INVAL;
  *expired = 0;
  cudaStream_t s = (cudaStream_t)stream;
  hrm::GridSync* d = nullptr;
  if (cudaMallocAsync(&d, sizeof *d, s) != cudaSuccess) return HRM_E_NOMEM;
  cudaMemsetAsync(d, 0, sizeof *d, s);
  k_barrier_probe<<<4, 128, 0, s>>>(d, (uint64_t)(limit_ms * 1e6));
  unsigned int h = 0;
  cudaMemcpyAsync(&h, &d->expired, sizeof h, cudaMemcpyDeviceToHost, s);
  cudaFreeAsync(d, s);
  if (cudaStreamSynchronize(s) != cudaSuccess) return HRM_E_CUDA;
  *expired = (int64_t)h;
  return h ? HRM_E_TIMEOUT : HRM_OK;
}

extern "C" hrm_status hrm_probe_convert(const double* in_d, const float* in_f, int64_t n, float* narrowed,
                                        double* widened, void* stream) {
  if (n < 0 || (n > 0 && (!in_d || !in_f || !narrowed || !widened))) return HRM_E_INVAL;
  if (n == 0) return HRM_OK;
  cudaStream_t s = (cudaStream_t)stream;
  k_convert<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(in_d, in_f, n, narrowed, widened);
  return cudaGetLastError() == cudaSuccess ? HRM_OK : HRM_E_CUDA;
}

extern "C" hrm_status hrm_probe_wait_timeout(void* stream, int64_t* expired) {
  if (!expired) return HRM_E_INVAL;
  *expired = 0;
  cudaStream_t s = (cudaStream_t)stream;
  unsigned long long* d = nullptr;
  if (cudaMallocAsync(&d, sizeof *d, s) != cudaSuccess) return HRM_E_NOMEM;
  cudaMemsetAsync(d, 0, sizeof *d, s);
  k_wait_probe<<<1, 128, 0, s>>>(d);
  unsigned long long h = 0;
  cudaMemcpyAsync(&h, d, sizeof h, cudaMemcpyDeviceToHost, s);
  cudaFreeAsync(d, s);
  if (cudaStreamSynchronize(s) != cudaSuccess) return HRM_E_CUDA;
  *expired = (int64_t)h;
  return h ? HRM_E_TIMEOUT : HRM_OK;
}

extern "C" hrm_status hrm_probe_fma_peak(int32_t precision, int32_t iters, void* stream, double* flops_per_s) {
  if (!flops_per_s || iters <= 0) return HRM_E_INVAL;
  cudaStream_t s = (cudaStream_t)stream;
  return precision == HRM_FP32 ? run<float>(iters, s, flops_per_s) : run<double>(iters, s, flops_per_s);
}
