// Device-side building blocks of the PP-WCNS-IS fractional algorithm
// (Wong, Angel & Kiris, arXiv 2208.04488) for sm_103a.
//
// Everything here is register-resident, templated on the number of species N,
// the number of dimensions D and the bulk compute type R (double for the FP64
// path, float for the precision form). The state itself always lives in FP64.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#define HRM_MAXN 4

namespace hrm {

// ---------------------------------------------------------------- launch-time descriptions

// Species constants, derived once on the host from gamma, p_inf, c_v, q (Sec. 2).
struct DevFluid {
  int32_t liq;  // index of the stiffened gas (Sec. 4.2 calls it species 1)
  int32_t has_q;  // 1 when some q_k != 0 (the precision form skips sum alpha_k rho_k q_k otherwise)
  double inv_gm1[HRM_MAXN];    // 1/(gamma_k - 1)
  double gpinf_gm1[HRM_MAXN];  // gamma_k p_inf_k / (gamma_k - 1)
  double cv[HRM_MAXN], cp[HRM_MAXN], Rg[HRM_MAXN];  // c_v, c_p, c_p - c_v
  double q[HRM_MAXN], pinf[HRM_MAXN], gamma[HRM_MAXN];
  // FP32 roundings of inv_gm1, gpinf_gm1 and q for the precision form
  float inv_gm1_f[HRM_MAXN], gpinf_gm1_f[HRM_MAXN], q_f[HRM_MAXN];
};

// Fill the FP32 copies of the species constants (host).
inline void fill_fluid_f(DevFluid& f) {
  f.has_q = 0;
  for (int k = 0; k < HRM_MAXN; ++k) {
    if (f.q[k] != 0.0) f.has_q = 1;
    f.inv_gm1_f[k] = (float)f.inv_gm1[k];
    f.gpinf_gm1_f[k] = (float)f.gpinf_gm1[k];
    f.q_f[k] = (float)f.q[k];
  }
}

// Species constants in the arithmetic type R.
__device__ __forceinline__ double inv_gm1_of(const DevFluid& f, int k, double) { return f.inv_gm1[k]; }
__device__ __forceinline__ float inv_gm1_of(const DevFluid& f, int k, float) { return f.inv_gm1_f[k]; }
__device__ __forceinline__ double gpinf_gm1_of(const DevFluid& f, int k, double) { return f.gpinf_gm1[k]; }
__device__ __forceinline__ float gpinf_gm1_of(const DevFluid& f, int k, float) { return f.gpinf_gm1_f[k]; }
__device__ __forceinline__ double q_of(const DevFluid& f, int k, double) { return f.q[k]; }
__device__ __forceinline__ float q_of(const DevFluid& f, int k, float) { return f.q_f[k]; }

// Cells are stored plane by plane (x fastest). A Dirichlet side keeps its
// boundary state as one slice of ghost cells stored after the nint interior
// cells of every plane (slice cells: the other directions' indices, lowest
// fastest), so ncells = nint + the slices and every per-plane stride is ncells.
struct DevGrid {
  int64_t n[3];
  int64_t ncells;   // stored cells per plane (interior + Dirichlet slices)
  int64_t nint;     // interior cells
  int64_t goff[6];  // first cell of side b's slice (bc[b] == 2), else 0
  double dx[3], inv_dx[3];
  int32_t bc[6];  // 0 transmissive, 1 periodic, 2 Dirichlet
  unsigned long long* oob;  // bounds-check builds: count of out-of-range indices (else unused)
};

// Bounds-check builds (-DHRM_BOUNDS_CHECK): an index outside [0, n) is counted
// in g.oob and replaced by 0 instead of being used; release builds use it as is.
#ifdef HRM_BOUNDS_CHECK
__device__ __forceinline__ int64_t hrm_checked_index(const DevGrid& g, int64_t i, int64_t n) {
  if (i >= 0 && i < n) return i;
  if (g.oob) atomicAdd(g.oob, 1ull);
  return 0;
}
#define HRM_IDX(g, i, n) hrm_checked_index((g), (i), (n))
#else
#define HRM_IDX(g, i, n) (i)
#endif

struct DevParams {
  int32_t limiters, blend, scheme, qexp;
  double eps_ar, eps_a, eps_rhoe, hs_ar, hs_a, hs_rc2, hs_rhoe, weno_eps, Cs;
  // precision form: certify the limiters' no-op in FP32 first (screen), with
  // the thresholds rounded up to FP32
  int32_t screen, pad_;
  float eps_ar_f, eps_rhoe_f, hs_rc2_f, eps_a_mf;  // eps_a_mf: eps_a + 1e-13 (float-float margin)
  float weno_eps_f, Cs_f;                          // FP32 roundings of weno_eps and Cs
};

// ---------------------------------------------------------------- FP32 <-> FP64 on the integer pipes
// GB300 executes FP64 instructions, the FP32 <-> FP64 conversions included, at
// 1/64 of the FP32 rate. The precision form converts tens of values per cell and
// per midpoint, so these two build the converted encodings from the IEEE-754
// formats with integer operations instead; each gives exactly the hardware
// conversion's result (the GPU tests compare them bit for bit).

// float -> double, exact: sign kept, exponent rebiased by 1023 - 127 = 896,
// mantissa moved up by 52 - 23 = 29 bits. Zeros are built here; subnormal,
// infinite and NaN inputs use the hardware conversion.
__device__ __forceinline__ double widen_f32(float x) {
  const uint32_t u = __float_as_uint(x);
  const uint32_t mag = u & 0x7fffffffu;
  if (mag - 0x00800000u >= 0x7f000000u) {  // not a normal number
    if (mag == 0u) return __hiloint2double((int)(u & 0x80000000u), 0);
    return (double)x;
  }
  const uint32_t hi = (u & 0x80000000u) | ((mag >> 3) + (896u << 20));
  return __hiloint2double((int)hi, (int)(u << 29));
}

// double -> float, rounded to nearest with ties to even: the 52-bit mantissa
// keeps its top 23 bits and the 29 dropped bits decide the rounding (a carry
// may move into the exponent, up to infinity past the largest float). Done
// here for results with a normal float exponent (1..254) and for zeros; other
// inputs (subnormal or overflowing results, infinities, NaN) use the hardware
// conversion.
__device__ __forceinline__ float narrow_f64(double x) {
  const uint32_t hi = (uint32_t)__double2hiint(x), lo = (uint32_t)__double2loint(x);
  const uint32_t e = (hi >> 20) & 0x7ffu;
  if (e - 897u >= 254u) {
    if (((hi & 0x7fffffffu) | lo) == 0u) return __uint_as_float(hi & 0x80000000u);
    return (float)x;
  }
  const uint32_t m = ((hi & 0xfffffu) << 3) | (lo >> 29);
  const uint32_t r = lo & 0x1fffffffu;
  const uint32_t f = (hi & 0x80000000u) | ((e - 896u) << 23) | m;
  return __uint_as_float(f + ((r > 0x10000000u || (r == 0x10000000u && (m & 1u))) ? 1u : 0u));
}

// Per-step scalars kept on the device so that a captured graph needs no host input.
struct StepState {
  double dt;        // step size in use
  double dt_req;    // > 0: requested step; <= 0: CFL step
  double cfl;
  double lam[3];    // flux-limiter lambda_d = dt / (sigma_d dx_d)
  double tau[3];    // tau_d of the step-start state
  double t;         // simulated time
  long long steps;
  unsigned long long tau_bits[3];  // running maxima (bit patterns of non-negative doubles)
  unsigned long long counts[4];    // admissibility counters
  unsigned long long waits;        // bounded tensor-core waits that ran out (learned gate)
  int wn_relaxed;  // nonzero: every interior cell of W^n came out of the form's relaxation (set by the host)
  int planes_tau;  // nonzero: the FP32 planes and tau_bits already hold W^n's (set by the host)
};

// Whether the midpoints of direction dir go to blocks in patches of 32 along x
// by 4 along dir (one warp per row), so that a block's four warps read 9 rows
// of nodes instead of 24 and share them in L1: always for z (z neighbours lie a
// whole plane apart); for y on rows of at most 1024 cells (measured: the FP32
// step 1.2 % faster at 1024 x 512, 1.6 % slower at 2048 x 1024, where the
// linear layout's concurrently running blocks already share the rows in L2).
__host__ __device__ inline bool patched(const DevGrid& g, int dir) {
  return dir == 2 || (dir == 1 && g.n[0] <= 1024);
}

// ---------------------------------------------------------------- small helpers

template <typename T> __device__ __forceinline__ T dmin(T a, T b) { return (b < a) ? b : a; }
template <typename T> __device__ __forceinline__ T dmax(T a, T b) { return (a < b) ? b : a; }

__device__ __forceinline__ double rsqrt_r(double x) { return sqrt(x); }
__device__ __forceinline__ float rsqrt_r(float x) { return sqrtf(x); }
// tanh|x| = m / (m + 2), m = expm1(2|x|): Taylor series of expm1 below 0.5, else
// exp(y) = 2^k exp(r) with Cody-Waite reduction (y = k ln2 + r, ln2 split into
// a 32-bit head and its tail) and the Taylor series of exp(r); 1 above 22.
// Built without contraction, every rounding is fixed by the expression order.
__device__ __forceinline__ double tanh_r(double x) {
  constexpr double kLn2 = 0.6931471805599453;
  constexpr double kLn2Hi = 0.6931471803691238;
  constexpr double kLn2Lo = 1.9082149292705877e-10;
  const double ax = fabs(x);
  double t;
  if (ax > 22.0) {
    t = 1.0;
  } else {
    const double y = 2.0 * ax;
    double m;
    if (y < 0.5) {
      double s = 1.0;
#pragma unroll
      for (int k = 18; k >= 2; --k) s = 1.0 + (y * (1.0 / (double)k)) * s;
      m = y * s;
    } else {
      const double k = rint(y / kLn2);
      const double r = (y - k * kLn2Hi) - k * kLn2Lo;
      double s = 1.0;
#pragma unroll
      for (int j = 17; j >= 1; --j) s = 1.0 + (r * (1.0 / (double)j)) * s;
      m = ldexp(s, (int)k) - 1.0;
    }
    t = m / (m + 2.0);
  }
  return x < 0.0 ? -t : t;
}
__device__ __forceinline__ float tanh_r(float x) { return tanhf(x); }

// Index of cell j (may lie in the 3 ghost layers) along direction d under the
// boundary condition of that side: transmissive copies the first interior cell
// (zeroth-order extrapolation), periodic wraps. (Dirichlet sides are resolved
// by the caller, which knows the transverse index.)
__device__ __forceinline__ int64_t bc_map(const DevGrid& g, int d, int64_t j) {
  const int64_t n = g.n[d];
  if (j < 0) return g.bc[2 * d] == 1 ? j + n : 0;
  if (j >= n) return g.bc[2 * d + 1] == 1 ? j - n : n - 1;
  return j;
}

template <int N, int D>
struct Lay {
  static constexpr int M = 2 * N + D;
  static constexpr int MOM = N;          // first momentum / velocity slot
  static constexpr int EN = N + D;       // E in W, p in V
  static constexpr int AL = N + D + 1;   // first stored volume fraction
  static constexpr int NC = N + D + 1;   // number of conservative (non-alpha) slots
};

// ---------------------------------------------------------------- mixture rules (Sec. 2)

// S = 1/(gbar - 1), P = gbar pbar_inf / (gbar - 1) from the N-1 stored alphas.
template <typename R, int N>
__device__ __forceinline__ void mix_SP(const DevFluid& f, const R* al_stored, R& S, R& P) {
  R sum = R(0);
  S = R(0);
  P = R(0);
#pragma unroll
  for (int k = 0; k < N - 1; ++k) sum = sum + al_stored[k];
  const R last = R(1) - sum;  // alpha_N = 1 - sum of the others (Sec. 2)
#pragma unroll
  for (int k = 0; k < N; ++k) {
    R a = (k < N - 1) ? al_stored[k] : last;
    S = S + a * inv_gm1_of(f, k, R());
    P = P + a * gpinf_gm1_of(f, k, R());
  }
}

// rho c^2 = gbar (p + pbar_inf) = (1 + 1/S) p + P/S
template <typename R>
__device__ __forceinline__ R rho_c2(R S, R P, R p) {
  R gb = R(1) + R(1) / S;
  return gb * p + P / S;
}

// ---------------------------------------------------------------- WENO-IS (App. C)

// Left-biased incremental-stencil WENO value at x_{i+1/2} from
// (u_{i-2}, u_{i-1}, u_i, u_{i+1}, u_{i+2}).
// The incremental-stencil weights eta_k (App. C) scaled by the common positive
// factor (beta_0 + eps)(beta_1 + eps)(beta_01 + eps)(beta_2 + eps)(beta_3 + eps):
// omega_k = eta_k / sum_s eta_s is unchanged, and no division is left, e.g.
// eta_0 (...) = d_0 [(beta_0 + eps)(beta_01 + eps) + tau_5^2] (beta_1 + eps)(beta_2 + eps)(beta_3 + eps).
// The operation order is the oracle's (bit-identical FP64 path).
template <typename R>
__device__ __forceinline__ void weno_eta(R b0, R b1, R b01, R b2, R b3, R tau5, R eps, R& e0, R& e1, R& e2,
                                         R& e3) {
  const R a = b0 + eps, b = b1 + eps, c = b01 + eps, g2 = b2 + eps, g3 = b3 + eps;
  const R t2 = tau5 * tau5;
  const R g23 = g2 * g3;
  const R abc = (a * b) * c;
  e0 = R(15.0 / 32.0) * ((a * c + t2) * (b * g23));
  e1 = R(5.0 / 32.0) * ((b * c + t2) * (a * g23));
  e2 = R(5.0 / 16.0) * ((g2 + tau5) * (abc * g3));
  e3 = R(1.0 / 16.0) * ((g3 + tau5) * (abc * g2));
}

template <typename R>
__device__ __forceinline__ R weno_is(R um2, R um1, R u0, R up1, R up2, R eps) {
  // A constant stencil (five bit-identical values): every sub-stencil
  // interpolant reproduces the constant and the weights sum to one (App. C),
  // so the value is that constant, returned as it is -- as the oracle does.
  // Integer compares only.
  static_assert(sizeof(R) == 8, "FP64 interpolation");
  {
    const long long c = __double_as_longlong(u0);
    if ((__double_as_longlong(um2) == c) & (__double_as_longlong(um1) == c) & (__double_as_longlong(up1) == c) &
        (__double_as_longlong(up2) == c))
      return u0;
  }
  const R s0 = R(0.5) * (u0 + up1);
  const R s1 = R(0.5) * (R(3) * u0 - um1);
  const R s2 = R(0.125) * (R(3) * u0 + R(6) * up1 - up2);
  const R s3 = R(0.125) * (R(3) * um2 - R(10) * um1 + R(15) * u0);
  const R c13_12 = R(13.0 / 12.0);
  R t;
  const R b0 = (u0 - up1) * (u0 - up1);
  const R b1 = (um1 - u0) * (um1 - u0);
  t = um1 - R(2) * u0 + up1;
  const R t01 = um1 - up1;
  const R b01 = c13_12 * t * t + R(0.25) * t01 * t01;
  t = u0 - R(2) * up1 + up2;
  R tt = R(3) * u0 - R(4) * up1 + up2;
  const R b2 = c13_12 * t * t + R(0.25) * tt * tt;
  t = um2 - R(2) * um1 + u0;
  tt = um2 - R(4) * um1 + R(3) * u0;
  const R b3 = c13_12 * t * t + R(0.25) * tt * tt;
  t = up2 - R(4) * up1 + R(6) * u0 - R(4) * um1 + um2;
  tt = up2 - R(2) * up1 + R(2) * um1 - um2;
  const R tau5 = c13_12 * t * t + R(0.25) * tt * tt;
  R e0, e1, e2, e3;
  weno_eta<R>(b0, b1, b01, b2, b3, tau5, eps, e0, e1, e2, e3);
  const R es = e0 + e1 + e2 + e3;
  // sum_k omega_k S_k with omega_k = e_k / es: the normalisation applied once
  return (e0 * s0 + e1 * s1 + e2 * s2 + e3 * s3) / es;
}

// The same interpolation with every nonlinear weight replaced by its linear
// weight d_k (the value a smoothness gate selects): sum_k d_k S_k, evaluated
// in the order written so that the FP64 units reproduce it bit for bit.
template <typename R>
__device__ __forceinline__ R weno_lin(R um2, R um1, R u0, R up1, R up2) {
  // a constant stencil: the linear weights sum to one as well (App. C)
  static_assert(sizeof(R) == 8, "FP64 interpolation");
  {
    const long long c = __double_as_longlong(u0);
    if ((__double_as_longlong(um2) == c) & (__double_as_longlong(um1) == c) & (__double_as_longlong(up1) == c) &
        (__double_as_longlong(up2) == c))
      return u0;
  }
  const R s0 = R(0.5) * (u0 + up1);
  const R s1 = R(0.5) * (R(3) * u0 - um1);
  const R s2 = R(0.125) * (R(3) * u0 + R(6) * up1 - up2);
  const R s3 = R(0.125) * (R(3) * um2 - R(10) * um1 + R(15) * u0);
  return R(15.0 / 32.0) * s0 + R(5.0 / 32.0) * s1 + R(5.0 / 16.0) * s2 + R(1.0 / 16.0) * s3;
}

template <typename R>
__device__ __forceinline__ R weno_sel(bool lin, R um2, R um1, R u0, R up1, R up2, R eps) {
  return lin ? weno_lin<R>(um2, um1, u0, up1, up2) : weno_is<R>(um2, um1, u0, up1, up2, eps);
}

// Largest |omega_k - d_k| of the WENO-IS weights of one stencil (App. C): the
// smoothness label of the learned gate. NaN propagates.
template <typename R>
__device__ __forceinline__ R weno_dev(R um2, R um1, R u0, R up1, R up2, R eps) {
  const R c13_12 = R(13.0 / 12.0);
  R t;
  const R b0 = (u0 - up1) * (u0 - up1);
  const R b1 = (um1 - u0) * (um1 - u0);
  t = um1 - R(2) * u0 + up1;
  const R t01 = um1 - up1;
  const R b01 = c13_12 * t * t + R(0.25) * t01 * t01;
  t = u0 - R(2) * up1 + up2;
  R tt = R(3) * u0 - R(4) * up1 + up2;
  const R b2 = c13_12 * t * t + R(0.25) * tt * tt;
  t = um2 - R(2) * um1 + u0;
  tt = um2 - R(4) * um1 + R(3) * u0;
  const R b3 = c13_12 * t * t + R(0.25) * tt * tt;
  t = up2 - R(4) * up1 + R(6) * u0 - R(4) * um1 + um2;
  tt = up2 - R(2) * up1 + R(2) * um1 - um2;
  const R tau5 = c13_12 * t * t + R(0.25) * tt * tt;
  R e0, e1, e2, e3;
  weno_eta<R>(b0, b1, b01, b2, b3, tau5, eps, e0, e1, e2, e3);
  const R es = e0 + e1 + e2 + e3;
  const R dv[4] = {e0 / es - R(15.0 / 32.0), e1 / es - R(5.0 / 32.0), e2 / es - R(5.0 / 16.0),
                   e3 / es - R(1.0 / 16.0)};
  R mx = R(0);
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const R d = dv[k] < R(0) ? -dv[k] : dv[k];
    if (!(d <= mx)) mx = d;
  }
  return mx;
}

// ---------------------------------------------------------------- HLLC (Sec. 4.1.1)

// Conservative vector, total energy and sound speed of a primitive state.
template <typename R, int N, int D>
struct PrimState {
  R V[Lay<N, D>::M];
  R rho, E, c;
};

template <typename R, int N, int D>
__device__ __forceinline__ void prim_state(const DevFluid& f, PrimState<R, N, D>& s) {
  using L = Lay<N, D>;
  R rho = R(0), rq = R(0), kin = R(0);
#pragma unroll
  for (int k = 0; k < N; ++k) {
    rho = rho + s.V[k];
    rq = rq + s.V[k] * q_of(f, k, R());
  }
#pragma unroll
  for (int d = 0; d < D; ++d) kin = kin + s.V[L::MOM + d] * s.V[L::MOM + d];
  R S, P;
  mix_SP<R, N>(f, &s.V[L::AL], S, P);
  const R p = s.V[L::EN];
  s.rho = rho;
  s.E = (S * p + P) + R(0.5) * rho * kin + rq;
  s.c = rsqrt_r(rho_c2(S, P, p) / rho);
}

// HLLC flux of the flux-source form G (F^HLLC plus the upwind alpha s_* in the
// alpha slots) and s_*, from two primitive states. At s_* = 0 the two star
// fluxes are averaged ((1 +- sign)/2 with sign(0) = 0).
template <typename R, int N, int D, int DIR>
__device__ __forceinline__ R hllc(const DevFluid& f, PrimState<R, N, D>& Ls, PrimState<R, N, D>& Rs,
                                  R* G) {
  using L = Lay<N, D>;
  constexpr int M = L::M;
  prim_state<R, N, D>(f, Ls);
  prim_state<R, N, D>(f, Rs);
  const R uL = Ls.V[L::MOM + DIR], uR = Rs.V[L::MOM + DIR];
  const R pL = Ls.V[L::EN], pR = Rs.V[L::EN];
  const R ubar = R(0.5) * (uL + uR), cbar = R(0.5) * (Ls.c + Rs.c);
  const R sL = dmin(ubar - cbar, uL - Ls.c);
  const R sR = dmax(ubar + cbar, uR + Rs.c);
  const R ss = (pR - pL + Ls.rho * uL * (sL - uL) - Rs.rho * uR * (sR - uR)) /
               (Ls.rho * (sL - uL) - Rs.rho * (sR - uR));
  const int sg = (ss > R(0)) ? 1 : ((ss < R(0)) ? -1 : 0);
  const R wL = (sg > 0) ? R(1) : ((sg < 0) ? R(0) : R(0.5));
  const R wR = R(1) - wL;
#pragma unroll
  for (int m = 0; m < M; ++m) G[m] = R(0);
#pragma unroll
  for (int side = 0; side < 2; ++side) {
    if ((side == 0 && sg < 0) || (side == 1 && sg > 0)) continue;
    PrimState<R, N, D>& K = side == 0 ? Ls : Rs;
    const R w = side == 0 ? wL : wR;
    const R uK = side == 0 ? uL : uR;
    const R pK = side == 0 ? pL : pR;
    const R sK = side == 0 ? sL : sR;
    const R sfac = side == 0 ? dmin(R(0), sL) : dmax(R(0), sR);
    const R chi = (sK - uK) / (sK - ss);
    // F_K + s_{-/+} (W_{*,K} - W_K), conservative slots
#pragma unroll
    for (int k = 0; k < N; ++k) {
      const R wk = K.V[k];
      G[k] = G[k] + w * (wk * uK + sfac * (chi * wk - wk));
    }
#pragma unroll
    for (int d = 0; d < D; ++d) {
      const R mom = K.rho * K.V[L::MOM + d];
      R Fm = mom * uK;
      if (d == DIR) Fm = Fm + pK;
      const R ms = (d == DIR) ? chi * K.rho * ss : chi * K.rho * K.V[L::MOM + d];
      G[L::MOM + d] = G[L::MOM + d] + w * (Fm + sfac * (ms - mom));
    }
    const R Es = chi * (K.E + (ss - uK) * (K.rho * ss + pK / (sK - uK)));
    G[L::EN] = G[L::EN] + w * ((K.E + pK) * uK + sfac * (Es - K.E));
#pragma unroll
    for (int k = 0; k < N - 1; ++k) G[L::AL + k] = G[L::AL + k] + w * (K.V[L::AL + k] * ss);
  }
  return ss;
}

}  // namespace hrm
