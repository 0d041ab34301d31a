// Host-side launchers of the kernel templates, one table per (N, D), so that
// the C-ABI layer dispatches at run time and the heavy instantiations compile
// in separate translation units.
#pragma once

#include <cuda_runtime.h>

#include <cmath>

#include "hrm_device.cuh"

namespace hrm {

struct CellKernels {
  // P32 (nullable): FP32 planes for the precision form; R32 (nullable): FP32
  // rounding residues of rho, u_d, p for the learned gate
  // same (nullable; ignored with tau): per interior cell, nonzero where W is bit
  // for bit the state V, AUX, P32, R32 were computed from -- those cells are kept
  void (*prim)(const double* W, double* V, double* AUX, float* P32, float* R32, const DevGrid&, const DevFluid&,
               StepState*, int tau, const uint8_t* same, cudaStream_t);
  void (*ic)(const double* prim, double* W, const DevGrid&, const DevFluid&, int64_t c0, int64_t c1, cudaStream_t);
  void (*relax)(double* W, const DevGrid&, const DevFluid&, cudaStream_t);
  void (*fields)(const double* W, double* out, int field, const DevGrid&, const DevFluid&, cudaStream_t);
  void (*admiss)(const double* W, const DevGrid&, const DevFluid&, StepState*, cudaStream_t);
};

// Smoothness gate of a midpoint sweep: `fixed` (nullable) one byte per
// midpoint, nonzero = linear WENO weights there (a caller's fixed gate, or the
// bytes the learned detector's gate kernel wrote before the sweep).
struct GateArgs {
  const uint8_t* fixed = nullptr;
  // precision form with screens: the sweep defers midpoints whose screens fail
  // to a second kernel through this worklist (one entry per midpoint of the
  // direction) and counter; nullptr: one kernel with the fallbacks inline
  uint32_t* defer_list = nullptr;
  uint32_t* defer_count = nullptr;
  // optional: run the deferred midpoints on `side` (after ev_fast, recorded on
  // the sweep's stream) and record ev_fix there, so that they overlap the next
  // sweep; the caller joins ev_fix before the update
  cudaStream_t side = nullptr;
  cudaEvent_t ev_fast = nullptr, ev_fix = nullptr;
  // precision form with the learned detector (with a worklist): the sweep
  // evaluates the network itself (k_face32_net) from the FP32 planes and their
  // residues R32, with the detector's inference blob (an mlp::GateBlob) and the
  // logit threshold, and writes its gate bytes to `out_gate` (which the
  // deferred-midpoint kernel then reads as `fixed`)
  const void* net = nullptr;
  const float* R32 = nullptr;
  float zthr = 0.f;
  uint8_t* out_gate = nullptr;
};

// Stream of the deferred-midpoint kernel: gate.side (forked from s after the
// sweep) or s itself.
inline cudaStream_t fix_stream(const GateArgs& gate, cudaStream_t s) {
  if (!gate.side) return s;
  cudaEventRecord(gate.ev_fast, s);
  cudaStreamWaitEvent(gate.side, gate.ev_fast, 0);
  return gate.side;
}
inline void fix_done(const GateArgs& gate) {
  if (gate.side) cudaEventRecord(gate.ev_fix, gate.side);
}

// Launch shape of the deferred-midpoint kernel: one-warp blocks, 16 per SM.
constexpr int kFixBlocks = 2432;
constexpr int kFixThreads = 32;

struct FaceKernels {
  // precision: 0 FP64, 1 FP32 bulk
  void (*face[3])(int precision, const double* W, const double* V, const double* AUX, const float* P32,
                  double* out, const DevGrid&, const DevFluid&, const DevParams&, const StepState*,
                  const GateArgs& gate, cudaStream_t);
  // mode 0: RK combination, mode 1: write the RHS; fast: precision-form variant;
  // same (nullable; FP64 RK combination): per interior cell, set to 1 where
  // W_out equals W_src bit for bit, else 0
  void (*update)(int mode, int fast, const double* Wn, const double* Wsrc, double* Wout, const double* F0,
                 const double* F1, const double* F2, const DevGrid&, const DevFluid&, StepState*, double a,
                 double b, int relax, int count, uint8_t* same, cudaStream_t);
};

const CellKernels* cell_kernels(int N, int D);
const FaceKernels* face_kernels(int N, int D);
const FaceKernels* face_kernels_d1(int N);
const FaceKernels* face_kernels_d2(int N);
const FaceKernels* face_kernels_d3(int N);

// FP32-bulk midpoint kernels, compiled in their own units (with FMA contraction).
void update32_d1(int N, const double* Wn, const double* Wsrc, double* Wout, const double* F0, const double* F1,
                 const double* F2, const DevGrid&, const DevFluid&, StepState*, double a, double b, int relax,
                 int count, cudaStream_t);
void face32_d1(int N, int dir, const double* W, const double* V, const double* AUX, const float* P32, double* out,
               const DevGrid&, const DevFluid&, const DevParams&, const StepState*, const GateArgs& gate,
               cudaStream_t);
void update32_d2(int N, const double* Wn, const double* Wsrc, double* Wout, const double* F0, const double* F1,
                 const double* F2, const DevGrid&, const DevFluid&, StepState*, double a, double b, int relax,
                 int count, cudaStream_t);
void face32_d2(int N, int dir, const double* W, const double* V, const double* AUX, const float* P32, double* out,
               const DevGrid&, const DevFluid&, const DevParams&, const StepState*, const GateArgs& gate,
               cudaStream_t);
void update32_d3(int N, const double* Wn, const double* Wsrc, double* Wout, const double* F0, const double* F1,
                 const double* F2, const DevGrid&, const DevFluid&, StepState*, double a, double b, int relax,
                 int count, cudaStream_t);
void face32_d3(int N, int dir, const double* W, const double* V, const double* AUX, const float* P32, double* out,
               const DevGrid&, const DevFluid&, const DevParams&, const StepState*, const GateArgs& gate,
               cudaStream_t);

// Precision-form update fused with the next stage's FP32 planes (k_update32p;
// hrm_face32_dD.cu).
void update32p_d1(int N, const double* Wn, const double* Wsrc, double* Wout, const double* F0, const double* F1,
                  const double* F2, const DevGrid&, const DevFluid&, StepState*, double a, double b, int relax,
                  int count, float* P32, float* R32, int tau, cudaStream_t);
void update32p_d2(int N, const double* Wn, const double* Wsrc, double* Wout, const double* F0, const double* F1,
                  const double* F2, const DevGrid&, const DevFluid&, StepState*, double a, double b, int relax,
                  int count, float* P32, float* R32, int tau, cudaStream_t);
void update32p_d3(int N, const double* Wn, const double* Wsrc, double* Wout, const double* F0, const double* F1,
                  const double* F2, const DevGrid&, const DevFluid&, StepState*, double a, double b, int relax,
                  int count, float* P32, float* R32, int tau, cudaStream_t);
// tau: also accumulate the CFL maxima of W_out into st->tau_bits (a step's last
// stage; grids without Dirichlet slices, five-equation sound speed).
inline void launch_update32p(int N, int D, const double* Wn, const double* Wsrc, double* Wout, const double* F0,
                             const double* F1, const double* F2, const DevGrid& g, const DevFluid& f, StepState* st,
                             double a, double b, int relax, int count, float* P32, float* R32, cudaStream_t s,
                             int tau = 0) {
  if (D == 1) update32p_d1(N, Wn, Wsrc, Wout, F0, F1, F2, g, f, st, a, b, relax, count, P32, R32, tau, s);
  if (D == 2) update32p_d2(N, Wn, Wsrc, Wout, F0, F1, F2, g, f, st, a, b, relax, count, P32, R32, tau, s);
  if (D == 3) update32p_d3(N, Wn, Wsrc, Wout, F0, F1, F2, g, f, st, a, b, relax, count, P32, R32, tau, s);
}

// Primitive kernel of the precision form (FP32 planes only; hrm_face32_dD.cu).
void prim32_d1(int N, const double* W, float* P32, float* R32, const DevGrid&, const DevFluid&, StepState*, int tau,
               cudaStream_t);
void prim32_d2(int N, const double* W, float* P32, float* R32, const DevGrid&, const DevFluid&, StepState*, int tau,
               cudaStream_t);
void prim32_d3(int N, const double* W, float* P32, float* R32, const DevGrid&, const DevFluid&, StepState*, int tau,
               cudaStream_t);
inline void launch_prim32(int N, int D, const double* W, float* P32, float* R32, const DevGrid& g, const DevFluid& f,
                          StepState* st, int tau, cudaStream_t s) {
  if (D == 1) prim32_d1(N, W, P32, R32, g, f, st, tau, s);
  if (D == 2) prim32_d2(N, W, P32, R32, g, f, st, tau, s);
  if (D == 3) prim32_d3(N, W, P32, R32, g, f, st, tau, s);
}

void launch_finalize(StepState* st, const DevGrid& g, int D, double cfl, int mode, cudaStream_t s);
void launch_set_dt(StepState* st, double dt, cudaStream_t s);

inline unsigned grid_for(long long n, int threads) { return (unsigned)((n + threads - 1) / threads); }

// Blocks of kFaceThreads covering the midpoints of direction dir in the layout
// of patch_midpoint (linear, or patches of 32 x 4 where patched(g, dir)).
inline unsigned patch_grid(const DevGrid& g, int dir) {
  const long long f0 = g.n[0] + (dir == 0), f1 = g.n[1] + (dir == 1), f2 = g.n[2] + (dir == 2);
  if (!patched(g, dir)) return grid_for(f0 * f1 * f2, 128);
  const long long nbx = (f0 + 31) / 32;
  return (unsigned)(dir == 1 ? nbx * ((f1 + 3) / 4) * f2 : nbx * f1 * ((f2 + 3) / 4));
}

// Blocks of kFaceThreads covering the midpoints of direction dir of a 2D or 3D
// grid in the layout of lane_patch_midpoint (32 x 4 midpoints per block).
inline unsigned lane_patch_grid(const DevGrid& g, int dir) {
  const long long f0 = g.n[0] + (dir == 0), f1 = g.n[1] + (dir == 1), f2 = g.n[2] + (dir == 2);
  return (unsigned)(((f0 + 31) / 32) * ((f1 + 3) / 4) * f2);
}

// Smallest float not below x (thresholds of the FP32 screens).
inline float float_up(double x) {
  float f = (float)x;
  if ((double)f < x) f = std::nextafter(f, INFINITY);
  return f;
}

// The screens certify "theta = 1 and no hard switch" from "every checked
// quantity >= its limiter threshold", which implies the hard-switch tests only
// when each hard-switch threshold is at most the limiter threshold.
inline void fill_screen(DevParams& d, int requested) {
  d.screen = requested && d.hs_ar <= d.eps_ar && d.hs_a <= d.eps_a && d.hs_rhoe <= d.eps_rhoe;
  d.eps_ar_f = float_up(d.eps_ar);
  d.eps_rhoe_f = float_up(d.eps_rhoe);
  d.hs_rc2_f = float_up(d.hs_rc2);
  d.eps_a_mf = float_up(d.eps_a + 1e-13);
  d.weno_eps_f = (float)d.weno_eps;
  d.Cs_f = (float)d.Cs;
  d.pad_ = 0;
}

}  // namespace hrm
