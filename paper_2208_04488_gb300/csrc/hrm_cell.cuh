// Per-cell kernels: primitive variables and the CFL reduction, the step-scalar
// finalisation, the initial state in p-T equilibrium, standalone relaxation,
// output fields and admissibility counters. Compiled without FMA contraction
// (these are cheap), so their results are the IEEE-rounded evaluation of the
// expressions as written.
#pragma once

#include "hrm_kernels.cuh"

namespace hrm {

// Primitive variables of a conservative vector (Sec. 2): rho = sum alpha_k rho_k,
// u_d = rho u_d / rho, p from the mixture EOS p/(gbar-1) + gbar pbar_inf/(gbar-1) =
// rho (e - qbar), rho c^2 = gbar (p + pbar_inf), c = sqrt(rho c^2 / rho).
template <int N, int D>
__device__ __forceinline__ void cell_prim(const double* W, const DevFluid& f, double* V, double& rho,
                                          double& c, double& rc2) {
  using L = Lay<N, D>;
  rho = 0.0;
#pragma unroll
  for (int k = 0; k < N; ++k) rho += W[k];
  double S, P;
  mix_SP<double, N>(f, &W[L::AL], S, P);
  const double re = rhoe_tilde<N, D>(W, f);
  const double p = (re - P) / S;
#pragma unroll
  for (int k = 0; k < N; ++k) V[k] = W[k];
#pragma unroll
  for (int d = 0; d < D; ++d) V[L::MOM + d] = W[L::MOM + d] / rho;
  V[L::EN] = p;
#pragma unroll
  for (int k = 0; k < N - 1; ++k) V[L::AL + k] = W[L::AL + k];
  rc2 = rho_c2(S, P, p);
  c = sqrt(rc2 / rho);
}

// Order-preserving bits of a non-negative double (IEEE order equals unsigned order).
__device__ __forceinline__ unsigned long long dbits(double x) {
  return (unsigned long long)__double_as_longlong(x);
}

// Four-equation HRM sound speed (Eq. 4_eqn_sos): Psi_k and Gamma by implicit
// differentiation of A_p p^2 + B_p p + C_p = 0 at the relaxed pressure p.
// Optionally also returns Psi_k (N values) and Gamma.
template <int N, int D>
__device__ __forceinline__ double c4eq(const double* W, const DevFluid& f, double p, double* Psi = nullptr,
                                       double* Gam_out = nullptr) {
  const int l = f.liq;
  double rho = 0.0;
#pragma unroll
  for (int k = 0; k < N; ++k) rho += W[k];
  double Y[N];
#pragma unroll
  for (int k = 0; k < N; ++k) Y[k] = W[k] / rho;
  const double re = rhoe_tilde<N, D>(W, f);
  double cvb = 0.0, cpb = 0.0, qb = 0.0;
#pragma unroll
  for (int k = 0; k < N; ++k) {
    cvb += Y[k] * f.cv[k];
    cpb += Y[k] * f.cp[k];
    qb += Y[k] * f.q[k];
  }
  const double pinf1 = f.pinf[l], R1 = f.Rg[l], Rb = cpb - cvb;
  const double Bp = -(re * Rb - pinf1 * cvb - pinf1 * Y[l] * R1);
  const double den = 2.0 * cvb * p + Bp;
  const double Gam = (-(-(rho * Rb) * p - pinf1 * rho * (Rb - Y[l] * R1)) / den) / rho;
  if (Gam_out) *Gam_out = Gam;
  double c2 = Gam * p / rho;
  const double e = re / rho + qb;
#pragma unroll
  for (int k = 0; k < N; ++k) {
    const double dre = e - f.q[k];
    const double dcv = (f.cv[k] - cvb) / rho;
    const double dRb = (f.Rg[k] - Rb) / rho;
    const double dY1 = ((k == l ? 1.0 : 0.0) - Y[l]) / rho;
    const double dB = -(dre * Rb + re * dRb - pinf1 * dcv - pinf1 * R1 * dY1);
    const double dC = -(pinf1 * (dre * (Rb - Y[l] * R1) + re * (dRb - R1 * dY1)));
    const double psi = -(dcv * p * p + dB * p + dC) / den;
    if (Psi) Psi[k] = psi;
    c2 += Y[k] * psi;
  }
  return sqrt(c2);
}

// Four-equation HRM sound speed of a conservative vector: relaxed p, then Eq.
// 4_eqn_sos (the CFL speed option params.cfl_sound = 1).
template <int N, int D>
__device__ __forceinline__ double c4_of_cell(const double* w, const DevFluid& f) {
  double wr[Lay<N, D>::M], pT[2];
#pragma unroll
  for (int m = 0; m < Lay<N, D>::M; ++m) wr[m] = w[m];
  relax_cell<N, D>(wr, f, pT);
  return c4eq<N, D>(w, f, pT[0]);
}

// Per cell: V (M planes), AUX = (c, rho, rho c^2). With `tau`, also the running
// maxima tau_d = max(|u_d| + c)/dx_d (Sec. 4.1.2): warp shuffles, then one
// atomicMax per block and direction on the order-preserving bits. tau = 1 takes
// the five-equation c, tau = 2 the four-equation HRM c (Eq. 4_eqn_sos).
// One cell c < ncells: primitives, AUX, optional FP32 planes and, for the
// learned gate, the FP32 rounding residues of rho, u_d and p (R32, D + 2
// planes: rho, u_0 .. u_{D-1}, p); s[d] = (|u_d| + c)/dx_d, with the
// four-equation c when c4.
template <int N, int D>
__device__ __forceinline__ void prim_body(int64_t c, const double* __restrict__ W, double* __restrict__ V,
                                          double* __restrict__ AUX, float* __restrict__ P32,
                                          float* __restrict__ R32, const DevGrid& g, const DevFluid& f, double* s,
                                          bool c4 = false) {
  using L = Lay<N, D>;
  constexpr int M = L::M;
  const int64_t nc = g.ncells;
  {
    double w[M], v[M], rho, cs, rc2;
#pragma unroll
    for (int m = 0; m < M; ++m) w[m] = W[m * nc + c];
    cell_prim<N, D>(w, f, v, rho, cs, rc2);
#pragma unroll
    for (int m = 0; m < M; ++m) V[m * nc + c] = v[m];
    AUX[c] = cs;
    AUX[nc + c] = rho;
    AUX[2 * nc + c] = rc2;
    if (P32) {
      // FP32 copies for the precision form: V, c, rho, rho c^2, rho u_d, E
#pragma unroll
      for (int m = 0; m < M; ++m) P32[m * nc + c] = (float)v[m];
      P32[M * nc + c] = (float)cs;
      P32[(M + 1) * nc + c] = (float)rho;
      P32[(M + 2) * nc + c] = (float)rc2;
#pragma unroll
      for (int d = 0; d < D; ++d) P32[(M + 3 + d) * nc + c] = (float)w[L::MOM + d];
      P32[(M + 3 + D) * nc + c] = (float)w[L::EN];
#pragma unroll
      for (int k = 0; k < N - 1; ++k) {
        const double a = w[L::AL + k];
        P32[(M + 4 + D + k) * nc + c] = (float)(a - (double)(float)a);  // rounding residue
      }
    }
    if (R32) {
      R32[c] = (float)(rho - (double)(float)rho);
#pragma unroll
      for (int d = 0; d < D; ++d) {
        const double u = v[L::MOM + d];
        R32[(1 + d) * nc + c] = (float)(u - (double)(float)u);
      }
      R32[(1 + D) * nc + c] = (float)(v[L::EN] - (double)(float)v[L::EN]);
    }
    const double cw = c4 ? c4_of_cell<N, D>(w, f) : cs;  // wave speed of the CFL maxima
#pragma unroll
    for (int d = 0; d < D; ++d) s[d] = (fabs(v[L::MOM + d]) + cw) / g.dx[d];
  }
}

// Block-level max of s[d] over the threads of the block, then one atomicMax per
// direction on the order-preserving bits (NaN reduces as the largest value).
template <int D>
__device__ __forceinline__ void block_tau_max(const double* s, unsigned long long* tau_bits) {
  __shared__ unsigned long long red[D][kCellThreads / 32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int d = 0; d < D; ++d) {
    unsigned long long b = dbits(s[d]);
    // NaN wave speeds (non-admissible states) reduce as the largest value
    if (s[d] != s[d]) b = 0x7ff8000000000000ull;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const unsigned long long x = __shfl_xor_sync(0xffffffffu, b, o);
      b = x > b ? x : b;
    }
    if (lane == 0) red[d][wid] = b;
  }
  __syncthreads();
  if (threadIdx.x < D) {
    unsigned long long b = 0;
    for (int w = 0; w < (int)(blockDim.x / 32); ++w) b = red[threadIdx.x][w] > b ? red[threadIdx.x][w] : b;
    atomicMax(&tau_bits[threadIdx.x], b);
  }
  __syncthreads();  // red is reused by the next call in a persistent loop
}

// same (nullable, only without the CFL maxima): one byte per interior cell, set
// where the last update left the cell's state bit for bit as it was in the
// source whose primitives V, AUX (and P32, R32) already hold -- those are kept.
template <int N, int D>
__global__ void __launch_bounds__(kCellThreads)
    k_prim(const double* __restrict__ W, double* __restrict__ V, double* __restrict__ AUX,
           float* __restrict__ P32, float* __restrict__ R32, DevGrid g, DevFluid f, StepState* st, int tau,
           const uint8_t* __restrict__ same) {
  const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  double s[D];
#pragma unroll
  for (int d = 0; d < D; ++d) s[d] = 0.0;
  const bool kept = same != nullptr && c < g.nint && same[c] != 0;
  if (c < g.ncells && !kept) prim_body<N, D>(c, W, V, AUX, P32, R32, g, f, s, tau == 2);
  if (!tau) return;
  block_tau_max<D>(s, st->tau_bits);
}

// Initial state from primitive planes (alpha_1..alpha_{N-1}, u_d, p, T) in p-T
// equilibrium: rho_k = (p + p_inf_k) / ((gamma_k - 1) c_v,k T) and the mixture EOS;
// cells c0 <= c < c1.
template <int N, int D>
__global__ void __launch_bounds__(kCellThreads)
    k_ic(const double* __restrict__ prim, double* __restrict__ W, DevGrid g, DevFluid f, int64_t c0, int64_t c1) {
  using L = Lay<N, D>;
  const int64_t c = c0 + (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t nc = g.ncells;
  if (c >= c1) return;
  double al[N], s = 0.0;
#pragma unroll
  for (int k = 0; k < N - 1; ++k) {
    al[k] = prim[k * nc + c];
    s += al[k];
  }
  al[N - 1] = 1.0 - s;
  const double p = prim[(N + D - 1) * nc + c], T = prim[(N + D) * nc + c];
  double rho = 0.0, E = 0.0, ar[N];
#pragma unroll
  for (int k = 0; k < N; ++k) {
    const double rhok = (p + f.pinf[k]) / (f.Rg[k] * T);
    ar[k] = al[k] * rhok;
    rho = rho + ar[k];
    E = E + al[k] * (p + f.gamma[k] * f.pinf[k]) * f.inv_gm1[k] + ar[k] * f.q[k];
  }
  double kin = 0.0;
#pragma unroll
  for (int d = 0; d < D; ++d) {
    const double u = prim[(N - 1 + d) * nc + c];
    kin = kin + u * u;
    W[(L::MOM + d) * nc + c] = rho * u;
  }
  E = E + 0.5 * rho * kin;
#pragma unroll
  for (int k = 0; k < N; ++k) W[k * nc + c] = ar[k];
  W[L::EN * nc + c] = E;
#pragma unroll
  for (int k = 0; k < N - 1; ++k) W[(L::AL + k) * nc + c] = al[k];
}

template <int N, int D>
__global__ void __launch_bounds__(kCellThreads) k_relax(double* W, DevGrid g, DevFluid f) {
  using L = Lay<N, D>;
  const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t nc = g.ncells;
  if (c >= g.nint) return;
  double w[L::M];
#pragma unroll
  for (int m = 0; m < L::M; ++m) w[m] = W[m * nc + c];
  relax_cell<N, D>(w, f);
#pragma unroll
  for (int k = 0; k < N - 1; ++k) W[(L::AL + k) * nc + c] = w[L::AL + k];
}

// Output fields of the current state (HRM_FIELD_*).
template <int N, int D>
__global__ void __launch_bounds__(kCellThreads)
    k_fields(const double* __restrict__ W, double* __restrict__ out, int field, DevGrid g, DevFluid f) {
  using L = Lay<N, D>;
  constexpr int M = L::M;
  const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t nc = g.ncells;
  if (c >= g.nint) return;
  double w[M], v[M], rho, cs, rc2;
#pragma unroll
  for (int m = 0; m < M; ++m) w[m] = W[m * nc + c];
  if (field == 8) {
    // numerical schlieren |grad rho| / rho: central differences, neighbours
    // through the boundary conditions (copy, wrap, or the prescribed state)
    const int64_t ijk[3] = {c % g.n[0], (c / g.n[0]) % g.n[1], c / (g.n[0] * g.n[1])};
    auto rho_at = [&](int64_t cell) {
      double r = 0.0;
#pragma unroll
      for (int k = 0; k < N; ++k) r += W[k * nc + cell];
      return r;
    };
    double r0 = 0.0;
#pragma unroll
    for (int k = 0; k < N; ++k) r0 += w[k];
    double g2 = 0.0;
#pragma unroll
    for (int d = 0; d < D; ++d) {
      int64_t nb[2];
#pragma unroll
      for (int side = 0; side < 2; ++side) {
        const int64_t j = ijk[d] + (side ? 1 : -1);
        int64_t q[3] = {ijk[0], ijk[1], ijk[2]};
        if ((j < 0 || j >= g.n[d]) && g.bc[2 * d + side] == 2) {
          int64_t tr = 0, stride = 1;
          for (int e = 0; e < 3; ++e)
            if (e != d) {
              tr += q[e] * stride;
              stride *= g.n[e];
            }
          nb[side] = g.goff[2 * d + side] + tr;
        } else {
          q[d] = bc_map(g, d, j);
          nb[side] = (q[2] * g.n[1] + q[1]) * g.n[0] + q[0];
        }
      }
      const double gd = (rho_at(nb[1]) - rho_at(nb[0])) * (0.5 * g.inv_dx[d]);
      g2 += gd * gd;
    }
    out[c] = sqrt(g2) / r0;
    return;
  }
  if (field == 6 || field == 7) {
    // all N volume fractions (alpha_N = 1 - the others) or mass fractions Y_k
    double r = 0.0, sa = 0.0;
#pragma unroll
    for (int k = 0; k < N; ++k) r += w[k];
#pragma unroll
    for (int k = 0; k < N - 1; ++k) sa += w[L::AL + k];
#pragma unroll
    for (int k = 0; k < N; ++k)
      out[k * nc + c] = field == 7 ? w[k] / r : (k < N - 1 ? w[L::AL + k] : 1.0 - sa);
    return;
  }
  if (field == 1 || field == 2) {
    cell_prim<N, D>(w, f, v, rho, cs, rc2);
    if (field == 1) {
#pragma unroll
      for (int m = 0; m < M; ++m) out[m * nc + c] = v[m];
    } else {
      out[c] = cs;
    }
    return;
  }
  double pT[2];
  double wr[M];
#pragma unroll
  for (int m = 0; m < M; ++m) wr[m] = w[m];
  relax_cell<N, D>(wr, f, pT);
  if (field == 3) {
    out[c] = pT[0];
    out[nc + c] = pT[1];
  } else if (field == 5) {
    double Psi[N], Gam;
    c4eq<N, D>(w, f, pT[0], Psi, &Gam);
#pragma unroll
    for (int k = 0; k < N; ++k) out[k * nc + c] = Psi[k];
    out[N * nc + c] = Gam;
  } else {
    out[c] = c4eq<N, D>(w, f, pT[0]);
  }
}

template <int N, int D>
__global__ void __launch_bounds__(kCellThreads)
    k_admiss(const double* __restrict__ W, DevGrid g, DevFluid f, StepState* st) {
  using L = Lay<N, D>;
  const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t nc = g.ncells;
  if (c >= g.nint) return;
  double w[L::M];
#pragma unroll
  for (int m = 0; m < L::M; ++m) w[m] = W[m * nc + c];
  count_bits(st, admissibility_bits<N, D>(w, f));
}

}  // namespace hrm
