// Host-side glue of the learned smoothness detector: what the context layer
// and the detector layer need from each other, and the launchers of the
// detector's kernels.
#pragma once

#include <cuda_runtime.h>

#include "../../include/hrm.h"
#include "hrm_launch.h"
#include "hrm_learned.cuh"

namespace hrm {

// What the detector reads from a context.
struct CtxView {
  int N, D, M;
  int64_t nc;
  DevGrid dg;
  DevFluid fl;
  DevParams dp;
  double* Wn;
  double* V;
  double* AUX;
  float* P32;
  float* R32;
  StepState* st;
  const CellKernels* ck;
  cudaStream_t stream;
};
hrm_status ctx_view(hrm_ctx* c, CtxView* out);
void ctx_add_launches(hrm_ctx* c, int64_t n);

const mlp::GateBlob* detector_blob(const hrm_detector* d);

// Midpoint count of direction dir.
__host__ __device__ inline int64_t face_total(const DevGrid& g, int dir) {
  return (g.n[0] + (dir == 0)) * (g.n[1] + (dir == 1)) * (g.n[2] + (dir == 2));
}

// Gate bytes of every midpoint of direction dir from the FP32 planes.
// waits: device counter of tensor-core waits that ran out.
void launch_gate(int N, int D, int dir, const float* P32, const float* R32, const DevGrid& g,
                 const mlp::GateBlob* blob, float zthr, uint8_t* gate, unsigned long long* waits, int max_blocks,
                 cudaStream_t s);

// Training-sample collection (hrm_learned_data.cu): pass 0 counts the kept
// midpoints per block of kCollectThreads, pass 1 writes them at the offsets
// the scan produced.
constexpr int kCollectThreads = 256;
struct CollectArgs {
  const double* V;
  const double* AUX;
  const float* P32;
  const float* R32;
  DevGrid g;
  double eps, delta;
  double keep_rough, keep_smooth, keep_flat;
  uint64_t salt;
  int32_t* counts;
  const int64_t* offsets;
  float* X;  // [cap][32]
  float* y;
  float* dev;
  int64_t cap;
};
void launch_collect(int N, int D, int dir, int pass, const CollectArgs& a, cudaStream_t s);
// offsets[b] = base + sum_{b' < b} counts[b'];  *total = sum of all counts
void launch_scan(const int32_t* counts, int64_t nb, int64_t base, int64_t* offsets, int64_t* total, cudaStream_t s);

}  // namespace hrm
