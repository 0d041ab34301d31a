// FP64 per-midpoint and per-cell-update kernels for D = 3, N = 2..3 species.
// Built without FMA contraction: the FP64 path evaluates the method's
// expressions in the same order and rounding as written, operation by operation.
#include "hrm_kernels.cuh"
#include "hrm_launch.h"

namespace hrm {
namespace {

constexpr int kD = 3;

template <int N, int DIR>
void face_l(int precision, const double* W, const double* V, const double* AUX, const float* P32, double* out,
            const DevGrid& g, const DevFluid& f, const DevParams& p, const StepState* st, const GateArgs& gate,
            cudaStream_t s) {
  if constexpr (DIR < kD) {
    if (precision == 1) {
      face32_d3(N, DIR, W, V, AUX, P32, out, g, f, p, st, gate, s);
      return;
    }
    k_face<double, N, kD, DIR><<<lane_patch_grid(g, DIR), kFaceThreads, 0, s>>>(W, V, AUX, out, g, f, p, st,
                                                                                gate.fixed);
  }
}

template <int N>
void update_l(int mode, int fast, const double* Wn, const double* Wsrc, double* Wout, const double* F0,
              const double* F1, const double* F2, const DevGrid& g, const DevFluid& f, StepState* st, double a,
              double b, int relax, int count, uint8_t* same, cudaStream_t s) {
  if (fast && mode == 0) {
    update32_d3(N, Wn, Wsrc, Wout, F0, F1, F2, g, f, st, a, b, relax, count, s);
    return;
  }
  const unsigned gr = grid_for(g.nint, kCellThreads);
  if (mode == 1)
    k_update<N, kD, 1><<<gr, kCellThreads, 0, s>>>(Wn, Wsrc, Wout, F0, F1, F2, g, f, st, a, b, relax, count);
  else
    k_update<N, kD, 0><<<gr, kCellThreads, 0, s>>>(Wn, Wsrc, Wout, F0, F1, F2, g, f, st, a, b, relax, count,
                                                   same);
}

template <int N>
const FaceKernels* table() {
  static const FaceKernels t = {{face_l<N, 0>, face_l<N, 1>, face_l<N, 2>}, update_l<N>};
  return &t;
}

}  // namespace

const FaceKernels* face_kernels_d3(int N) {
  if (N == 2) return table<2>();
  if (N == 3) return table<3>();
  return nullptr;
}

}  // namespace hrm
