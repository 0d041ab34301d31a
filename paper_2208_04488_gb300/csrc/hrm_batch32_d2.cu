// Batched-form kernels for D = 2 of the precision form: FP32 planes, FP32-bulk
// midpoints and the fast update (built with FMA contraction).
#include "hrm_batch.cuh"
#include "hrm_launch.h"

namespace hrm {

void batch_face32_d2(int N, int dir, const BatchLaunch& L, const BatchInst* insts, const WorkItem* items, int nitems,
                     int src, const DevParams& p, cudaStream_t s) {
  if (N == 2) {
    if (dir == 0)
      k_batch_face32<2, 0, 2><<<L.grid, L.threads, 0, s>>>(insts, items, nitems, src, p);
    else
      k_batch_face32<2, 1, 2><<<L.grid, L.threads, 0, s>>>(insts, items, nitems, src, p);
  } else {
    if (dir == 0)
      k_batch_face32<2, 0, 3><<<L.grid, L.threads, 0, s>>>(insts, items, nitems, src, p);
    else
      k_batch_face32<2, 1, 3><<<L.grid, L.threads, 0, s>>>(insts, items, nitems, src, p);
  }
}

namespace {
template <int DIR, int N>
void tiles_l(const BatchInst* insts, const WorkItem* tiles, int ntiles, int src, const DevParams& p,
             unsigned long long* list, uint32_t* count, cudaStream_t s) {
  cudaMemsetAsync(count, 0, sizeof(uint32_t), s);
  k_batch_face32_tiles<2, DIR, N><<<ntiles, kBatchFace32Threads, 0, s>>>(insts, tiles, src, p, list, count);
  k_batch_face32_fix<2, DIR, N><<<kFixBlocks, kFixThreads, 0, s>>>(insts, src, p, list, count);
}
}  // namespace

void batch_face32_tiles_d2(int N, int dir, const BatchInst* insts, const WorkItem* tiles, int ntiles, int src,
                           const DevParams& p, unsigned long long* list, uint32_t* count, cudaStream_t s) {
  if (N == 2) {
    if (dir == 0)
      tiles_l<0, 2>(insts, tiles, ntiles, src, p, list, count, s);
    else
      tiles_l<1, 2>(insts, tiles, ntiles, src, p, list, count, s);
  } else {
    if (dir == 0)
      tiles_l<0, 3>(insts, tiles, ntiles, src, p, list, count, s);
    else
      tiles_l<1, 3>(insts, tiles, ntiles, src, p, list, count, s);
  }
}

void batch_prim32_d2(int N, const BatchLaunch& L, const BatchInst* insts, const WorkItem* items, int nitems, int src,
                     int tau, cudaStream_t s) {
  if (N == 2)
    k_batch_prim32<2, 2><<<L.grid, L.threads, 0, s>>>(insts, items, nitems, src, tau);
  else
    k_batch_prim32<2, 3><<<L.grid, L.threads, 0, s>>>(insts, items, nitems, src, tau);
}

void batch_update32_d2(int N, const BatchLaunch& L, const BatchInst* insts, const WorkItem* items, int nitems,
                       int src, int dst, double a, double b, int relax, int count, cudaStream_t s) {
  if (N == 2)
    k_batch_update<2, true, 2><<<L.grid, L.threads, 0, s>>>(insts, items, nitems, src, dst, a, b, relax, count);
  else
    k_batch_update<2, true, 3><<<L.grid, L.threads, 0, s>>>(insts, items, nitems, src, dst, a, b, relax, count);
}

}  // namespace hrm
