// Per-cell kernels, instantiated for N = 2..3 species and D = 1..3 dimensions.
// Built without FMA contraction (see hrm_cell.cuh).
#include "hrm_cell.cuh"
#include "hrm_launch.h"

namespace hrm {

// Step scalars from the reduced tau_d (Sec. 4.1.2): dt = cfl / sum tau, or the
// requested dt; sigma_d = tau_d / sum tau, lambda_d = dt / (sigma_d dx_d).
// mode 0 advances the step time and count, mode 1 only answers a dt query.
__global__ void k_finalize(StepState* st, DevGrid g, int D, double cfl, int mode) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double tau[3] = {0.0, 0.0, 0.0}, sum = 0.0;
  for (int d = 0; d < D; ++d) {
    tau[d] = __longlong_as_double((long long)st->tau_bits[d]);
    sum = sum + tau[d];
    st->tau_bits[d] = 0ull;
  }
  const double dt = (mode == 0 && st->dt_req > 0.0) ? st->dt_req : cfl / sum;
  for (int d = 0; d < D; ++d) {
    const double sigma = tau[d] / sum;
    st->lam[d] = dt / (sigma * g.dx[d]);
    st->tau[d] = tau[d];
  }
  st->dt = dt;
  if (mode == 0) {
    st->t = st->t + dt;
    st->steps = st->steps + 1;
  }
}

__global__ void k_set_dt(StepState* st, double dt_req) {
  if (threadIdx.x == 0 && blockIdx.x == 0) st->dt_req = dt_req;
}

namespace {

template <int N, int D>
void prim_l(const double* W, double* V, double* AUX, float* P32, float* R32, const DevGrid& g, const DevFluid& f,
            StepState* st, int tau, const uint8_t* same, cudaStream_t s) {
  k_prim<N, D><<<grid_for(g.ncells, kCellThreads), kCellThreads, 0, s>>>(W, V, AUX, P32, R32, g, f, st, tau,
                                                                          tau ? nullptr : same);
}
template <int N, int D>
void ic_l(const double* prim, double* W, const DevGrid& g, const DevFluid& f, int64_t c0, int64_t c1,
          cudaStream_t s) {
  if (c1 <= c0) return;
  k_ic<N, D><<<grid_for(c1 - c0, kCellThreads), kCellThreads, 0, s>>>(prim, W, g, f, c0, c1);
}
template <int N, int D>
void relax_l(double* W, const DevGrid& g, const DevFluid& f, cudaStream_t s) {
  k_relax<N, D><<<grid_for(g.nint, kCellThreads), kCellThreads, 0, s>>>(W, g, f);
}
template <int N, int D>
void fields_l(const double* W, double* out, int field, const DevGrid& g, const DevFluid& f, cudaStream_t s) {
  k_fields<N, D><<<grid_for(g.nint, kCellThreads), kCellThreads, 0, s>>>(W, out, field, g, f);
}
template <int N, int D>
void admiss_l(const double* W, const DevGrid& g, const DevFluid& f, StepState* st, cudaStream_t s) {
  k_admiss<N, D><<<grid_for(g.nint, kCellThreads), kCellThreads, 0, s>>>(W, g, f, st);
}

template <int N, int D>
const CellKernels* table() {
  static const CellKernels t = {prim_l<N, D>, ic_l<N, D>, relax_l<N, D>, fields_l<N, D>, admiss_l<N, D>};
  return &t;
}

}  // namespace

const CellKernels* cell_kernels(int N, int D) {
  if (N == 2 && D == 1) return table<2, 1>();
  if (N == 2 && D == 2) return table<2, 2>();
  if (N == 2 && D == 3) return table<2, 3>();
  if (N == 3 && D == 1) return table<3, 1>();
  if (N == 3 && D == 2) return table<3, 2>();
  if (N == 3 && D == 3) return table<3, 3>();
  return nullptr;
}

void launch_finalize(StepState* st, const DevGrid& g, int D, double cfl, int mode, cudaStream_t s) {
  k_finalize<<<1, 32, 0, s>>>(st, g, D, cfl, mode);
}

void launch_set_dt(StepState* st, double dt, cudaStream_t s) { k_set_dt<<<1, 32, 0, s>>>(st, dt); }

}  // namespace hrm
