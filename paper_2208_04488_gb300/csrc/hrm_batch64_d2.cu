// Batched-form kernels for D = 2 that must follow the FP64 path's rounding:
// primitives and CFL maxima, step scalars, FP64 midpoints, exact update.
// Built without FMA contraction, like the single-instance FP64 units.
#include "hrm_batch.cuh"

namespace hrm {

// Step scalars of every instance (thread per instance), as k_finalize.
__global__ void k_batch_finalize(const BatchInst* __restrict__ insts, int ninst, int D, double cfl) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < ninst; i += gridDim.x * blockDim.x) {
    const BatchInst& I = insts[i];
    StepState* st = I.st;
    double tau[3] = {0.0, 0.0, 0.0}, sum = 0.0;
    for (int d = 0; d < D; ++d) {
      tau[d] = __longlong_as_double((long long)st->tau_bits[d]);
      sum = sum + tau[d];
      st->tau_bits[d] = 0ull;
    }
    const double dt = cfl / sum;
    for (int d = 0; d < D; ++d) {
      const double sigma = tau[d] / sum;
      st->lam[d] = dt / (sigma * I.g.dx[d]);
      st->tau[d] = tau[d];
    }
    st->dt = dt;
    st->t = st->t + dt;
    st->steps = st->steps + 1;
  }
}


void batch_prim_d2(int N, const BatchLaunch& L, const BatchInst* insts, const WorkItem* items, int nitems, int src,
                   int tau, cudaStream_t s) {
  if (N == 2)
    k_batch_prim<2, 2><<<L.grid, L.threads, 0, s>>>(insts, items, nitems, src, 0, tau);
  else
    k_batch_prim<2, 3><<<L.grid, L.threads, 0, s>>>(insts, items, nitems, src, 0, tau);
}

void batch_finalize(const BatchInst* insts, int ninst, int D, double cfl, cudaStream_t s) {
  k_batch_finalize<<<(ninst + 127) / 128, 128, 0, s>>>(insts, ninst, D, cfl);
}

void batch_face64_tiles_d2(int N, int dir, const BatchInst* insts, const WorkItem* tiles, int ntiles, int src,
                           const DevParams& p, cudaStream_t s) {
  if (N == 2) {
    if (dir == 0)
      k_batch_face64_tiles<2, 0, 2><<<ntiles, kBatchFace32Threads, 0, s>>>(insts, tiles, src, p);
    else
      k_batch_face64_tiles<2, 1, 2><<<ntiles, kBatchFace32Threads, 0, s>>>(insts, tiles, src, p);
  } else {
    if (dir == 0)
      k_batch_face64_tiles<2, 0, 3><<<ntiles, kBatchFace32Threads, 0, s>>>(insts, tiles, src, p);
    else
      k_batch_face64_tiles<2, 1, 3><<<ntiles, kBatchFace32Threads, 0, s>>>(insts, tiles, src, p);
  }
}

void batch_face64_d2(int N, int dir, const BatchLaunch& L, const BatchInst* insts, const WorkItem* items, int nitems,
                     int src, const DevParams& p, cudaStream_t s) {
  if (N == 2) {
    if (dir == 0)
      k_batch_face64<2, 0, 2><<<L.grid, L.threads, 0, s>>>(insts, items, nitems, src, p);
    else
      k_batch_face64<2, 1, 2><<<L.grid, L.threads, 0, s>>>(insts, items, nitems, src, p);
  } else {
    if (dir == 0)
      k_batch_face64<2, 0, 3><<<L.grid, L.threads, 0, s>>>(insts, items, nitems, src, p);
    else
      k_batch_face64<2, 1, 3><<<L.grid, L.threads, 0, s>>>(insts, items, nitems, src, p);
  }
}

void batch_update64_d2(int N, const BatchLaunch& L, const BatchInst* insts, const WorkItem* items, int nitems,
                       int src, int dst, double a, double b, int relax, int count, cudaStream_t s) {
  if (N == 2)
    k_batch_update<2, false, 2><<<L.grid, L.threads, 0, s>>>(insts, items, nitems, src, dst, a, b, relax, count);
  else
    k_batch_update<2, false, 3><<<L.grid, L.threads, 0, s>>>(insts, items, nitems, src, dst, a, b, relax, count);
}

}  // namespace hrm
