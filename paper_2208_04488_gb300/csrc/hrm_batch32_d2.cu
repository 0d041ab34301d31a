// Batched-form persistent stage kernel for D = 2 of the precision form: FP32
// planes, FP32-bulk midpoints (FP64 limiters where a screen fails, out of
// line), the fast update; six blocks per SM as the single-context sweep.
#include "hrm_batch.cuh"

namespace hrm {

__global__ void __launch_bounds__(kBatchFace32Threads, 6) k_batch_stage32(StageArgs A) { batch_stage<2, true>(A); }

int batch_stage32_fit() {
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_batch_stage32, kBatchFace32Threads, 0) != cudaSuccess)
    return 0;
  return n;
}

cudaError_t batch_stage32_launch(int grid, const StageArgs& A, cudaStream_t s) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)grid);
  cfg.blockDim = dim3(kBatchFace32Threads);
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeCooperative;
  at[0].val.cooperative = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k_batch_stage32, A);
}

}  // namespace hrm
