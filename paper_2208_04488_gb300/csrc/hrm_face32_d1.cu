// FP32-bulk per-midpoint kernels for D = 1, N = 2..3 species (the precision
// form: interpolation, Riemann fluxes and HCS in FP32; limiter theta in FP64).
#include "hrm_face32.cuh"
#include "hrm_face32_net.cuh"
#include "hrm_launch.h"

namespace hrm {
namespace {

constexpr int kD = 1;

template <int N, int DIR>
void launch(const double* W, const double* V, const double* AUX, const float* P32, double* out, const DevGrid& g,
            const DevFluid& f, const DevParams& p, const StepState* st, const GateArgs& gate, cudaStream_t s) {
  if constexpr (DIR < kD) {
    if (gate.defer_list) {
      cudaMemsetAsync(gate.defer_count, 0, sizeof(uint32_t), s);
      if (gate.net)
        k_face32_net<N, kD, DIR><<<patch_grid(g, DIR), kFaceThreads, 0, s>>>(
            W, P32, gate.R32, out, g, f, p, st, static_cast<const mlp::GateBlob*>(gate.net), gate.zthr,
            gate.out_gate, gate.defer_list, gate.defer_count);
      else
        k_face32_fast<N, kD, DIR><<<patch_grid(g, DIR), kFaceThreads, 0, s>>>(
            W, P32, out, g, f, p, st, gate.fixed, gate.defer_list, gate.defer_count);
      const cudaStream_t sf = fix_stream(gate, s);
      k_face32_fix<N, kD, DIR><<<kFixBlocks, kFixThreads, 0, sf>>>(W, P32, out, g, f, p, st, gate.fixed,
                                                                    gate.defer_list, gate.defer_count);
      fix_done(gate);
    } else {
      k_face32<N, kD, DIR><<<patch_grid(g, DIR), kFaceThreads, 0, s>>>(W, V, AUX, P32, out, g, f, p, st,
                                                                                gate.fixed);
    }
  }
}

}  // namespace

void update32_d1(int N, const double* Wn, const double* Wsrc, double* Wout, const double* F0, const double* F1,
                 const double* F2, const DevGrid& g, const DevFluid& f, StepState* st, double a, double b, int relax,
                 int count, cudaStream_t s) {
  const unsigned gr = grid_for(g.nint, kCellThreads);
  if (N == 2)
    k_update<2, kD, 0, true><<<gr, kCellThreads, 0, s>>>(Wn, Wsrc, Wout, F0, F1, F2, g, f, st, a, b, relax, count);
  else if (N == 3)
    k_update<3, kD, 0, true><<<gr, kCellThreads, 0, s>>>(Wn, Wsrc, Wout, F0, F1, F2, g, f, st, a, b, relax, count);
}

void update32p_d1(int N, const double* Wn, const double* Wsrc, double* Wout, const double* F0, const double* F1,
                  const double* F2, const DevGrid& g, const DevFluid& f, StepState* st, double a, double b, int relax,
                  int count, float* P32, float* R32, int tau, cudaStream_t s) {
  const unsigned gr = grid_for(g.nint, kCellThreads);
  if (N == 2)
    k_update32p<2, kD><<<gr, kCellThreads, 0, s>>>(Wn, Wsrc, Wout, F0, F1, F2, g, f, st, a, b, relax, count, P32, R32,
                                                    tau);
  else if (N == 3)
    k_update32p<3, kD><<<gr, kCellThreads, 0, s>>>(Wn, Wsrc, Wout, F0, F1, F2, g, f, st, a, b, relax, count, P32, R32,
                                                    tau);
}

void face32_d1(int N, int dir, const double* W, const double* V, const double* AUX, const float* P32, double* out,
               const DevGrid& g, const DevFluid& f, const DevParams& p, const StepState* st, const GateArgs& gate,
               cudaStream_t s) {
  if (N == 2) {
    if (dir == 0) launch<2, 0>(W, V, AUX, P32, out, g, f, p, st, gate, s);
    if (dir == 1) launch<2, 1>(W, V, AUX, P32, out, g, f, p, st, gate, s);
    if (dir == 2) launch<2, 2>(W, V, AUX, P32, out, g, f, p, st, gate, s);
  } else if (N == 3) {
    if (dir == 0) launch<3, 0>(W, V, AUX, P32, out, g, f, p, st, gate, s);
    if (dir == 1) launch<3, 1>(W, V, AUX, P32, out, g, f, p, st, gate, s);
    if (dir == 2) launch<3, 2>(W, V, AUX, P32, out, g, f, p, st, gate, s);
  }
}

void prim32_d1(int N, const double* W, float* P32, float* R32, const DevGrid& g, const DevFluid& f, StepState* st,
               int tau, cudaStream_t s) {
  const unsigned gr = grid_for(g.ncells, kCellThreads);
  if (N == 2)
    k_prim32<2, kD><<<gr, kCellThreads, 0, s>>>(W, P32, R32, g, f, st, tau);
  else if (N == 3)
    k_prim32<3, kD><<<gr, kCellThreads, 0, s>>>(W, P32, R32, g, f, st, tau);
}

}  // namespace hrm
