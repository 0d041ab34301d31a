// Precision-form screened sweep with the learned smoothness detector evaluated
// inside it: the step path of the precision form with the learned gate.
//
// A warp first tests its 32 stencils for uniformity (uniform_stencil). A
// uniform stencil takes the node's physical flux, which no interpolation
// choice affects, so a warp of uniform stencils never evaluates the network
// (at the start of the benchmark workloads about nine warps in ten). Any other
// warp forms the 30 features of each stencil (stencil_features, the gate
// kernel's function) and runs the network on its 32 rows with warp-level MMA
// (mlp::warp_logit); a non-uniform stencil whose logit exceeds the threshold
// then uses the linear weights. Compared with a gate kernel before the sweep,
// this removes one launch per direction and the second read of the stencil
// planes, and the network runs only where a stencil is not uniform.
//
// Gate bytes (one per midpoint, in `gate`): 1 linear weights, 0 full WENO-IS,
// 2 uniform stencil (exact node flux). The deferred-midpoint kernel reads them.
#pragma once

#include "hrm_learned.cuh"

namespace hrm {

template <int N, int D, int DIR>
__global__ void __launch_bounds__(kFaceThreads, 6)
    k_face32_net(const double* __restrict__ W, const float* __restrict__ P32, const float* __restrict__ R32,
                 double* __restrict__ out, DevGrid g, DevFluid f, DevParams pr, const StepState* __restrict__ st,
                 const mlp::GateBlob* __restrict__ blob, float zthr, uint8_t* __restrict__ gate,
                 uint32_t* __restrict__ list, uint32_t* __restrict__ count) {
  __shared__ __align__(16) __nv_bfloat16 X[kFaceThreads / 32][32][mlp::kWarpRow];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t t = patch_midpoint<DIR>(g);
  Nodes6 nd;
  const bool valid = face_nodes<DIR>(g, t, nd);
  const bool uni = !valid || uniform_stencil<N, D>(P32, g.ncells, nd);
  if (valid && uni) {
    uniform_flux<N, D, DIR>(t, nd, P32, out, g);
    gate[t] = 2;
  }
  if (__all_sync(0xffffffffu, uni)) return;  // the whole warp
  float x[mlp::kIn];
  if (uni) {
#pragma unroll
    for (int k = 0; k < mlp::kIn; ++k) x[k] = 0.f;
  } else {
    mlp::stencil_features<N, D, DIR>(nd, P32, R32, g.ncells, x);
  }
  mlp::warp_store_row(X[warp], lane, x);
  __syncwarp();
  const float z = mlp::warp_logit(*blob, X[warp], lane);
  bool need = false;
  if (!uni) {
    const bool lin = z > zthr;
    gate[t] = lin ? 1 : 0;
    need = !face32_body<N, D, DIR, true>(t, nd, W, nullptr, nullptr, P32, out, g, f, pr, st->lam[DIR], lin,
                                         nullptr, true);
  }
  defer_push(need, t, list, count);
}

}  // namespace hrm
