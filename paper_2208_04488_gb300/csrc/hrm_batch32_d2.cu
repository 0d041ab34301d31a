// Batched-form kernels for D = 2 of the precision form: FP32 planes, FP32-bulk
// midpoints and the fast update (built with FMA contraction).
#include "hrm_batch.cuh"

namespace hrm {

void batch_face32_d2(int dir, const BatchLaunch& L, const BatchInst* insts, const WorkItem* items, int nitems, int src,
                     const DevParams& p, cudaStream_t s) {
  if (dir == 0)
    k_batch_face<2, 0, true><<<L.grid, L.threads, 0, s>>>(insts, items, nitems, src, p);
  else
    k_batch_face<2, 1, true><<<L.grid, L.threads, 0, s>>>(insts, items, nitems, src, p);
}

void batch_prim32_d2(const BatchLaunch& L, const BatchInst* insts, const WorkItem* items, int nitems, int src, int tau,
                     cudaStream_t s) {
  k_batch_prim32<2><<<L.grid, L.threads, 0, s>>>(insts, items, nitems, src, tau);
}

void batch_update32_d2(const BatchLaunch& L, const BatchInst* insts, const WorkItem* items, int nitems, int src,
                       int dst, double a, double b, int relax, int count, cudaStream_t s) {
  k_batch_update<2, true><<<L.grid, L.threads, 0, s>>>(insts, items, nitems, src, dst, a, b, relax, count);
}

}  // namespace hrm
