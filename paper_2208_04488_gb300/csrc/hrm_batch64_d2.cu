// Batched-form persistent stage kernel for D = 2 in FP64: built without FMA
// contraction, like the single-instance FP64 units, so that every instance
// follows the FP64 path's rounding bit for bit.
#include "hrm_batch.cuh"

namespace hrm {

__global__ void __launch_bounds__(kBatchFace32Threads) k_batch_stage64(StageArgs A) { batch_stage<2, false>(A); }

int batch_stage64_fit() {
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_batch_stage64, kBatchFace32Threads, 0) != cudaSuccess)
    return 0;
  return n;
}

cudaError_t batch_stage64_launch(int grid, const StageArgs& A, cudaStream_t s) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)grid);
  cfg.blockDim = dim3(kBatchFace32Threads);
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeCooperative;
  at[0].val.cooperative = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k_batch_stage64, A);
}

}  // namespace hrm
