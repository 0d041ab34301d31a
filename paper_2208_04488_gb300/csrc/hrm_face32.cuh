// Precision form of the per-midpoint kernel: characteristic projection,
// WENO-IS, both HLLC solves, HCS and the sensor blend in FP32; the
// interpolation-limiter and flux-limiter theta solves, the half-cell states and
// everything downstream (flux difference, RK combination, relaxation) in FP64.
#pragma once

#include "hrm_cell.cuh"

namespace hrm {

// FP32 planes written by k_prim for the precision form (per cell):
// V[0..M-1], c, rho, rho c^2, rho u_d (D planes), E, and the rounding residues
// alpha_k - (float)alpha_k of the N-1 stored volume fractions, so that
// differences of volume fractions near 1 keep their full precision.
template <int N, int D>
struct P32Lay {
  static constexpr int M = Lay<N, D>::M;
  static constexpr int C = M, RHO = M + 1, RC2 = M + 2, MOM = M + 3, E = M + 3 + D, ALO = M + 4 + D;
  static constexpr int PLANES = M + 4 + D + (N - 1);
};

// Incremental-stencil WENO (App. C) in FP32 on the stencil's differences from
// its central value, scaled so that the largest is 1; eps scales with them
// (floored at 1e-15 so that no ratio tau5 / (beta + eps) can overflow). The
// sub-stencil interpolants reproduce constants, so this equals the unscaled
// scheme up to rounding and to smoothness indicators below 1e-15 of the
// stencil's range.
// A stencil whose range is below 1e-30 is taken as constant: its reciprocal
// would leave the normal float range (1/s = inf for subnormal s).
constexpr float kTinyRange = 1e-30f;

// Linear-weight (gated) interpolation on the differences from the central value:
// sum_k d_k S_k = u_0 + (3 a - 20 b + 60 d - 5 e) / 128.
__device__ __forceinline__ float lin_increment(float a, float b, float d, float e) {
  return (3.f * a - 20.f * b + 60.f * d - 5.f * e) * (1.f / 128.f);
}

// WENO-IS (App. C) of the precision form on differences from the central node
// (a, b, d, e = u_{i-2}, u_{i-1}, u_{i+1}, u_{i+2} minus u_i, scaled to unit
// range): the same sub-stencil values, smoothness indicators, tau_5 and weights
// as weno_is, with the multiply-adds written as fmaf and the five weight
// divisions as approximate reciprocals (__fdividef, within 2 ulp; every
// denominator lies in [1e-15, 1e3]).
__device__ __forceinline__ float weno_is_f32(float a, float b, float d, float e, float eps) {
  const float s0 = 0.5f * d;
  const float s1 = -0.5f * b;
  const float s2 = 0.125f * fmaf(6.f, d, -e);
  const float s3 = 0.125f * fmaf(3.f, a, -10.f * b);
  const float c13_12 = 13.f / 12.f;
  const float b0 = d * d;
  const float b1 = b * b;
  float t = b + d, tt = b - d;
  const float b01 = fmaf(c13_12 * t, t, 0.25f * tt * tt);
  t = fmaf(-2.f, d, e);
  tt = fmaf(-4.f, d, e);
  const float b2 = fmaf(c13_12 * t, t, 0.25f * tt * tt);
  t = fmaf(-2.f, b, a);
  tt = fmaf(-4.f, b, a);
  const float b3 = fmaf(c13_12 * t, t, 0.25f * tt * tt);
  t = fmaf(-4.f, d + b, e + a);
  tt = fmaf(2.f, b - d, e - a);
  const float tau5 = fmaf(c13_12 * t, t, 0.25f * tt * tt);
  const float q01 = __fdividef(tau5, b01 + eps);
  const float e0 = (15.f / 32.f) * fmaf(__fdividef(tau5, b0 + eps), q01, 1.f);
  const float e1 = (5.f / 32.f) * fmaf(__fdividef(tau5, b1 + eps), q01, 1.f);
  const float e2 = (5.f / 16.f) * (1.f + __fdividef(tau5, b2 + eps));
  const float e3 = (1.f / 16.f) * (1.f + __fdividef(tau5, b3 + eps));
  const float es = (e0 + e1) + (e2 + e3);
  return __fdividef(fmaf(e0, s0, fmaf(e1, s1, fmaf(e2, s2, e3 * s3))), es);
}

__device__ __forceinline__ float weno_is_scaled(float um2, float um1, float u0, float up1, float up2, float eps,
                                                bool lin = false) {
  float a = um2 - u0, b = um1 - u0, d = up1 - u0, e = up2 - u0;
  if (lin) return u0 + lin_increment(a, b, d, e);
  const float s = fmaxf(fmaxf(fabsf(a), fabsf(b)), fmaxf(fabsf(d), fabsf(e)));
  if (!(s > kTinyRange)) return u0;
  const float inv = __frcp_rn(s);
  a *= inv;
  b *= inv;
  d *= inv;
  e *= inv;
  const float eps_s = fmaxf(eps * inv * inv, 1e-15f);
  return fmaf(s, weno_is_f32(a, b, d, e, eps_s), u0);
}

// WENO-IS increment from already-formed differences (u_j - u_0) of a stencil
// whose central value is the reference (left-biased order um2, um1, up1, up2).
__device__ __forceinline__ float weno_increment(float a, float b, float d, float e, float eps, bool lin = false) {
  if (lin) return lin_increment(a, b, d, e);
  const float s = fmaxf(fmaxf(fabsf(a), fabsf(b)), fmaxf(fabsf(d), fabsf(e)));
  if (!(s > kTinyRange)) return 0.f;
  const float inv = __frcp_rn(s);
  const float eps_s = fmaxf(eps * inv * inv, 1e-15f);
  return s * weno_is_f32(a * inv, b * inv, d * inv, e * inv, eps_s);
}

// Interpolation limiter of the precision form: partial densities from FP32,
// volume fractions carried in FP64 (at, the N-1 stored ones); theta in FP64.
template <int N, int D>
__device__ __forceinline__ void interp_limit32(float* Vt, double* at, const double* Vn, double rc2n,
                                               const DevFluid& f, const DevParams& pr) {
  using L = Lay<N, D>;
  constexpr int M = L::M;
#pragma unroll
  for (int k = 0; k < N; ++k) {
    const double lo = Vn[k], hi = (double)Vt[k];
    const double tgt = dmin(pr.eps_ar, lo);
    double th = 1.0;
    if (hi < tgt) th = (tgt - lo) / (hi - lo);
    Vt[k] = (float)((1.0 - th) * lo + th * hi);
  }
  double alt[N], aln[N];
  {
    double st = 0.0, sn = 0.0;
#pragma unroll
    for (int k = 0; k < N - 1; ++k) {
      alt[k] = at[k];
      aln[k] = Vn[L::AL + k];
      st += alt[k];
      sn += aln[k];
    }
    alt[N - 1] = 1.0 - st;
    aln[N - 1] = 1.0 - sn;
  }
  double th = 1.0;
#pragma unroll
  for (int k = 0; k < N; ++k) {
    const double tgt = dmin(pr.eps_a, aln[k]);
    if (alt[k] < tgt) th = dmin(th, (tgt - aln[k]) / (alt[k] - aln[k]));
  }
#pragma unroll
  for (int k = 0; k < N - 1; ++k) at[k] = (1.0 - th) * aln[k] + th * alt[k];
  bool hs = false;
  {
    double st = 0.0;
#pragma unroll
    for (int k = 0; k < N - 1; ++k) {
      alt[k] = at[k];
      st += alt[k];
    }
    alt[N - 1] = 1.0 - st;
  }
#pragma unroll
  for (int k = 0; k < N; ++k) {
    hs |= (double)Vt[k] < dmin(pr.hs_ar, Vn[k]);
    hs |= alt[k] < dmin(pr.hs_a, aln[k]);
  }
  double S, P;
  mix_SP<double, N>(f, alt, S, P);
  hs |= rho_c2(S, P, (double)Vt[L::EN]) < dmin(pr.hs_rc2, rc2n);
  if (hs) {
#pragma unroll
    for (int m = 0; m < M; ++m) Vt[m] = (float)Vn[m];
#pragma unroll
    for (int k = 0; k < N - 1; ++k) at[k] = Vn[L::AL + k];
  }
#pragma unroll
  for (int k = 0; k < N - 1; ++k) Vt[L::AL + k] = (float)at[k];
}

// Upwind alpha flux of HLLC (Sec. 4.1.1) in FP64: (1 + sign s*)/2 aL s* + (1 - sign s*)/2 aR s*.
__device__ __forceinline__ double alpha_flux(double aL, double aR, double ss) {
  if (ss > 0.0) return aL * ss;
  if (ss < 0.0) return aR * ss;
  return 0.5 * (aL * ss) + 0.5 * (aR * ss);
}

// ---------------------------------------------------------------- float-float
// Unevaluated sums hi + lo of two floats built with error-free
// transformations (Knuth's TwoSum, the FMA TwoProduct): about 2^-48 relative
// precision, on the FP32 pipe. The volume-fraction slots of the precision form
// use them: differences of volume fractions near 1 must keep the minor phase
// (1e-8) exact to far below its size.
struct ff {
  float hi, lo;
};
__device__ __forceinline__ ff ff_sum(float a, float b) {
  const float s = a + b, bb = s - a;
  return {s, (a - (s - bb)) + (b - bb)};
}
__device__ __forceinline__ ff ff_prod(float a, float b) {
  const float p = a * b;
  return {p, fmaf(a, b, -p)};
}
__device__ __forceinline__ ff ff_add(ff a, ff b) {
  const ff s = ff_sum(a.hi, b.hi);
  return ff_sum(s.hi, s.lo + (a.lo + b.lo));
}
__device__ __forceinline__ ff ff_sub(ff a, ff b) { return ff_add(a, ff{-b.hi, -b.lo}); }
__device__ __forceinline__ ff ff_mulf(ff a, float b) {
  const ff p = ff_prod(a.hi, b);
  return ff_sum(p.hi, fmaf(a.lo, b, p.lo));
}
__device__ __forceinline__ ff ff_mul(ff a, ff b) {
  const ff p = ff_prod(a.hi, b.hi);
  return ff_sum(p.hi, fmaf(a.hi, b.lo, fmaf(a.lo, b.hi, p.lo)));
}
__device__ __forceinline__ ff ff_of(double x) {
  const float h = narrow_f64(x);
  return {h, narrow_f64(x - widen_f32(h))};
}
__device__ __forceinline__ double ff_d(ff a) { return widen_f32(a.hi) + widen_f32(a.lo); }
__device__ __forceinline__ float ff_f(ff a) { return a.hi + a.lo; }
#define HRM_FF(c) ff{(float)(c), (float)((c) - (double)(float)(c))}

// ---------------------------------------------------------------- FP32 screens
// Each screen returns true only when the FP64 limiter is certain to leave its
// input unchanged: every quantity the limiter tests lies at or above the
// limiter threshold (which implies theta = 1 -- the target is min(eps, first-
// order value) -- and, with hard-switch thresholds not above the limiter
// thresholds, no hard switch). FP32 values are tested with a bound on their
// rounding error against the FP64 evaluation; float-float volume fractions
// with an absolute margin (pr.eps_a_mf = eps_a + 1e-13, rounded up). Where a
// screen fails, the FP64 limiter runs.

// u32 = 2^-24; the bounds below allow 16 u32 (partial densities, momenta,
// energy: inputs rounded once, a product, a difference and an FMA) and
// 32 u32 (rho c^2, rho e~).
constexpr float kScreenRel = 16.0f * 5.9604645e-8f;
constexpr float kScreenRel2 = 32.0f * 5.9604645e-8f;

// Interpolation limiter (Sec. 4.3.2) on one side: partial densities of the
// FP32 midpoint state, the volume fractions at (float-float, the N-1 stored
// ones), rho c^2 for the hard switch.
template <int N, int D>
__device__ __forceinline__ bool interp_screen32(const float* Vt, const ff* at, const DevFluid& f,
                                                const DevParams& pr) {
  using L = Lay<N, D>;
  bool ok = true;
#pragma unroll
  for (int k = 0; k < N; ++k) ok &= Vt[k] >= pr.eps_ar_f;  // float >= (eps rounded up) => double >= eps
  ff rest{1.f, 0.f};
  float a[N];
#pragma unroll
  for (int k = 0; k < N - 1; ++k) {
    a[k] = ff_f(at[k]);
    ok &= a[k] >= pr.eps_a_mf;
    rest = ff_sub(rest, at[k]);
  }
  a[N - 1] = ff_f(rest);
  ok &= a[N - 1] >= pr.eps_a_mf;
  float S = 0.f, P = 0.f;
#pragma unroll
  for (int k = 0; k < N; ++k) {
    S += a[k] * f.inv_gm1_f[k];
    P += a[k] * f.gpinf_gm1_f[k];
  }
  const float iS = 1.f / S;
  const float t1 = (1.f + iS) * Vt[L::EN], t2 = P * iS;
  ok &= (t1 + t2) - kScreenRel2 * (fabsf(t1) + fabsf(t2)) >= pr.hs_rc2_f;
  return ok;
}

// Flux limiter (Sec. 4.3.2): the high-order half-cell states W_i^+ and
// W_{i+1}^- from the FP32 node states and the FP32 midpoint flux g32 --
// partial densities and rho e~ in FP32 with error bounds -- and their volume
// fractions in float-float from the node values (ai, aj) and the alpha slots
// (gm, gp); lam2 = 2 lambda as float-float.
template <int N, int D, int DIR>
__device__ __forceinline__ bool flux_screen32(const float* __restrict__ P32, int64_t nc, const Nodes6& nd,
                                              const float* g32, const ff* gm, const ff* gp, const ff* ai,
                                              const ff* aj, ff lam2, const DevFluid& f, const DevParams& pr) {
  using L = Lay<N, D>;
  using Q = P32Lay<N, D>;
  bool ok = true;
#pragma unroll
  for (int side = 0; side < 2; ++side) {
    ff rest{1.f, 0.f};
#pragma unroll
    for (int k = 0; k < N - 1; ++k) {
      const ff a = side == 0 ? ff_sub(ai[k], ff_mul(lam2, gm[k])) : ff_add(aj[k], ff_mul(lam2, gp[k]));
      ok &= ff_f(a) >= pr.eps_a_mf;
      rest = ff_sub(rest, a);
    }
    ok &= ff_f(rest) >= pr.eps_a_mf;
  }
  const float s2 = lam2.hi;
  float qmax = 0.f;
#pragma unroll
  for (int k = 0; k < N; ++k) qmax = fmaxf(qmax, fabsf(f.q_f[k]));
#pragma unroll
  for (int side = 0; side < 2; ++side) {
    const int64_t c = nd.c[2 + side];
    const float sg = side == 0 ? -s2 : s2;
    const float un = P32[(int64_t)(L::MOM + DIR) * nc + c], p = P32[(int64_t)L::EN * nc + c];
    // partial densities
    float rho = 0.f, rq = 0.f, erho = 0.f;
#pragma unroll
    for (int k = 0; k < N; ++k) {
      const float w = P32[(int64_t)k * nc + c];
      const float F = w * un;
      const float h = w + sg * (g32[k] - F);
      const float e = kScreenRel * (fabsf(w) + s2 * (fabsf(g32[k]) + fabsf(F)));
      ok &= h - e >= pr.eps_ar_f;
      rho += h;
      rq += h * f.q_f[k];
      erho += e;
    }
    // momentum and energy, and rho e~ = E - |rho u|^2 / (2 rho) - sum alpha_k rho_k q_k
    float m2 = 0.f, emom = 0.f;
#pragma unroll
    for (int d = 0; d < D; ++d) {
      const float w = P32[(int64_t)(Q::MOM + d) * nc + c];
      const float F = w * un + (d == DIR ? p : 0.f);
      const float h = w + sg * (g32[L::MOM + d] - F);
      m2 += h * h;
      emom += kScreenRel * (fabsf(w) + s2 * (fabsf(g32[L::MOM + d]) + fabsf(w * un) + fabsf(p))) * fabsf(h);
    }
    const float wE = P32[(int64_t)Q::E * nc + c];
    const float FE = (wE + p) * un;
    const float E = wE + sg * (g32[L::EN] - FE);
    const float eE = kScreenRel * (fabsf(wE) + s2 * (fabsf(g32[L::EN]) + fabsf(wE * un) + fabsf(p * un)));
    const float irho = 1.f / rho;
    const float kin = 0.5f * m2 * irho;
    const float re = E - kin - rq;
    // error: E, |m| |dm| / rho, (|u|^2 / 2 + max|q|) drho, evaluation rounding
    const float err = eE + emom * irho + (kin * irho + qmax) * erho +
                      kScreenRel2 * (fabsf(E) + kin + fabsf(rq));
    ok &= re - err >= pr.eps_rhoe_f;
  }
  return ok;
}

// ---------------------------------------------------------------- per-cell planes
// Primitive kernel of the precision form: writes only the FP32 planes the
// midpoint kernel reads (P32Lay) -- the stored values, u_d, p, c, rho, rho c^2,
// the volume-fraction rounding residues -- and, for the learned gate, the
// residues of rho, u_d and p (R32); with `tau`, the CFL maxima. FP64 only where
// the EOS cancels: the mixture constants S, P, the energy sums and the pressure
// numerator rho e~ - P (E ~ P ~ 1e9 against p ~ 1e5 for a stiffened gas); the
// division by S, the velocities, rho c^2 and c in FP32 (their FP32 values are
// all the midpoint kernel uses). The node states the FP64 limiters need where a
// screen fails are evaluated from W there.
// FP32 planes of one cell from its FP64 state w (M values), its density rho
// and R_e = rho (rho e~) = rho (E - sum alpha_k rho_k q_k) - |rho u|^2 / 2. The
// pressure numerator rho (rho e~ - P) = R_e - rho P is formed in FP64 (it
// cancels where p_inf ~ 1e9 Pa meets the ambient pressure), then
// p = (R_e - rho P) / (rho S) in FP32; no FP64 division. S = 1/(gbar - 1) and
// the P of the FP32 sound speed come from the FP32 volume fractions (all their
// terms are positive). Returns u_d and c.
template <int N, int D>
__device__ __forceinline__ void prim32_store(int64_t c, const double* w, double rho, double Re,
                                             float* __restrict__ P32, float* __restrict__ R32, int64_t nc,
                                             const DevFluid& f, float* u, float& cs) {
  using L = Lay<N, D>;
  using Q = P32Lay<N, D>;
  double sa = 0.0;
#pragma unroll
  for (int k = 0; k < N - 1; ++k) sa += w[L::AL + k];
  const double aN = 1.0 - sa;
  double P = 0.0;
  float S32 = 0.f, Pf = 0.f;
#pragma unroll
  for (int k = 0; k < N; ++k) {
    const double a = k < N - 1 ? w[L::AL + k] : aN;
    const float a32 = narrow_f64(a);
    S32 += a32 * f.inv_gm1_f[k];
    if (f.pinf[k] != 0.0) {  // one stiffened gas at most: P has one term
      P = fma(a, f.gpinf_gm1[k], P);
      Pf += a32 * f.gpinf_gm1_f[k];
    }
  }
  const double num = fma(-rho, P, Re);  // rho (rho e~ - P)
  const float rho32 = narrow_f64(rho), irho32 = 1.f / rho32;
  const float iS = 1.f / S32;
  const float rS32 = rho32 * S32, irS = 1.f / rS32;
  const float p = narrow_f64(num) * irS;
  const float rc2 = (1.f + iS) * p + Pf * iS;
  cs = sqrtf(rc2 * irho32);
#pragma unroll
  for (int d = 0; d < D; ++d) u[d] = narrow_f64(w[L::MOM + d]) * irho32;
#pragma unroll
  for (int k = 0; k < N; ++k) P32[k * nc + c] = narrow_f64(w[k]);
#pragma unroll
  for (int d = 0; d < D; ++d) {
    P32[(L::MOM + d) * nc + c] = u[d];
    P32[(Q::MOM + d) * nc + c] = narrow_f64(w[L::MOM + d]);
  }
  P32[L::EN * nc + c] = p;
  P32[Q::C * nc + c] = cs;
  P32[Q::RHO * nc + c] = rho32;
  P32[Q::RC2 * nc + c] = rc2;
  P32[Q::E * nc + c] = narrow_f64(w[L::EN]);
#pragma unroll
  for (int k = 0; k < N - 1; ++k) {
    const double a = w[L::AL + k];
    const float ah = narrow_f64(a);
    P32[(L::AL + k) * nc + c] = ah;
    P32[(Q::ALO + k) * nc + c] = narrow_f64(a - widen_f32(ah));
  }
  if (R32) {
    // residues: rho exactly; u_d and p from the FP64 remainders of m - u rho and
    // (R_e - rho P) - p rho S (rho S in FP64 here)
    R32[c] = narrow_f64(rho - widen_f32(rho32));
#pragma unroll
    for (int d = 0; d < D; ++d) R32[(1 + d) * nc + c] = narrow_f64(w[L::MOM + d] - widen_f32(u[d]) * rho) * irho32;
    double S = 0.0;
#pragma unroll
    for (int k = 0; k < N; ++k) S = fma(k < N - 1 ? w[L::AL + k] : aN, f.inv_gm1[k], S);
    R32[(1 + D) * nc + c] = narrow_f64(num - widen_f32(p) * (rho * S)) * irS;
  }
}

// rho and R_e of a conservative state (the inputs of prim32_store).
template <int N, int D>
__device__ __forceinline__ void rho_Re(const double* w, const DevFluid& f, double& rho, double& Re) {
  using L = Lay<N, D>;
  double rq = 0.0, m2 = 0.0;
  rho = 0.0;
#pragma unroll
  for (int k = 0; k < N; ++k) rho += w[k];
  if (f.has_q) {
#pragma unroll
    for (int k = 0; k < N; ++k) rq = fma(w[k], f.q[k], rq);
  }
#pragma unroll
  for (int d = 0; d < D; ++d) m2 = fma(w[L::MOM + d], w[L::MOM + d], m2);
  Re = fma(rho, w[L::EN] - rq, -0.5 * m2);
}

template <int N, int D>
__device__ __forceinline__ void prim32_body(int64_t c, const double* __restrict__ W, float* __restrict__ P32,
                                            float* __restrict__ R32, const DevGrid& g, const DevFluid& f,
                                            double* s, bool c4 = false) {
  using L = Lay<N, D>;
  constexpr int M = L::M;
  const int64_t nc = g.ncells;
  double w[M];
#pragma unroll
  for (int m = 0; m < M; ++m) w[m] = W[m * nc + c];
  double rho, Re;
  rho_Re<N, D>(w, f, rho, Re);
  float u[D], cs;
  prim32_store<N, D>(c, w, rho, Re, P32, R32, nc, f, u, cs);
  if (c4) {
    const double cw = c4_of_cell<N, D>(w, f);  // four-equation HRM c (FP64)
#pragma unroll
    for (int d = 0; d < D; ++d) s[d] = ((double)fabsf(u[d]) + cw) * g.inv_dx[d];
    return;
  }
#pragma unroll
  for (int d = 0; d < D; ++d) s[d] = widen_f32((fabsf(u[d]) + cs) * narrow_f64(g.inv_dx[d]));
}

template <int N, int D>
__global__ void __launch_bounds__(kCellThreads)
    k_prim32(const double* __restrict__ W, float* __restrict__ P32, float* __restrict__ R32, DevGrid g, DevFluid f,
             StepState* st, int tau) {
  // a step's first primitive pass: the previous step's last update may have
  // written these planes and CFL maxima already (k_update32p with tau)
  if (tau && st->planes_tau) return;
  const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  double s[D];
#pragma unroll
  for (int d = 0; d < D; ++d) s[d] = 0.0;
  if (c < g.ncells) prim32_body<N, D>(c, W, P32, R32, g, f, s, tau == 2);
  if (!tau) return;
  block_tau_max<D>(s, st->tau_bits);
}

// True when every FP32 plane holds the same value at the six nodes of a
// midpoint (a NaN anywhere makes it false). One pass without branches, so
// that many loads are in flight at once: measured on the 1024x512
// shock-bubble, rounds of four planes with an exit after each, or
// short-circuit compares (each load waiting for the previous compare), made
// the check cost as much as the work it saves. PARTIAL: four planes per loop
// trip instead of all of them unrolled, for the batched stage kernel, whose
// register budget is shared with every phase (fully unrolled there, the
// check's loads spilled: 16.6 against 11.8 ms per batched step). The result
// is the same either way.
template <int N, int D, bool PARTIAL = false>
__device__ __forceinline__ bool uniform_stencil(const float* __restrict__ P32, int64_t nc, const Nodes6& nd) {
  bool same = true;
#pragma unroll(PARTIAL ? 4 : P32Lay<N, D>::PLANES)
  for (int q = 0; q < P32Lay<N, D>::PLANES; ++q) {
    const float* p = P32 + (int64_t)q * nc;
    float v[6];
#pragma unroll
    for (int j = 0; j < 6; ++j) v[j] = p[nd.c[j]];
    same = same & (v[0] == v[2]) & (v[1] == v[2]) & (v[3] == v[2]) & (v[4] == v[2]) & (v[5] == v[2]);
  }
  return same;
}

// Midpoint t of a uniform stencil: the node's physical flux from the
// conservative planes (the HCS node-flux expression at node i), zero alpha slots.
template <int N, int D, int DIR>
__device__ __forceinline__ void uniform_flux(int64_t t, const Nodes6& nd, const float* __restrict__ P32,
                                             double* __restrict__ out, const DevGrid& g) {
  using L = Lay<N, D>;
  using Q = P32Lay<N, D>;
  constexpr int M = L::M;
  const int64_t nc = g.ncells;
  const int64_t nf = face_count<DIR>(g);
  auto ld = [&](int plane) -> float { return P32[(int64_t)plane * nc + nd.c[2]]; };
  const float un = ld(L::MOM + DIR), pn = ld(L::EN);
#pragma unroll
  for (int m = 0; m < L::NC; ++m) {
    float v;
    if (m < L::MOM)
      v = ld(m) * un;
    else if (m < L::EN)
      v = ld(Q::MOM + (m - L::MOM)) * un + ((m - L::MOM) == DIR ? pn : 0.f);
    else
      v = (ld(Q::E) + pn) * un;
    out[m * nf + t] = widen_f32(v);
  }
#pragma unroll
  for (int k = 0; k < N - 1; ++k) {
    out[(L::AL + k) * nf + t] = 0.0;
    out[(M + k) * nf + t] = 0.0;
  }
}

// Appends index t to a worklist where `need` (all lanes of the warp call it;
// warp-aggregated: one atomic per warp; order not significant).
__device__ __forceinline__ void defer_push(bool need, int64_t t, uint32_t* __restrict__ list,
                                           uint32_t* __restrict__ count) {
  const unsigned m = __ballot_sync(0xffffffffu, need);
  if (m == 0u) return;
  const int lane = threadIdx.x & 31, leader = __ffs(m) - 1;
  uint32_t base = 0;
  if (lane == leader) base = atomicAdd(count, (uint32_t)__popc(m));
  base = __shfl_sync(0xffffffffu, base, leader);
  if (need) list[base + __popc(m & ((1u << lane) - 1u))] = (uint32_t)t;
}

// Precision-form update of one RK stage with the next stage's primitives fused
// in: the flux difference and SSP-RK combination (fast_combine), the
// relaxation (relax_fast), the admissibility count, the store of W_out, then
// the FP32 planes of W_out (prim32_store) that the next stage's sweeps read --
// in place of a separate k_prim32 pass over W_out. Interior cells only: the
// planes of Dirichlet slices keep what the stage's first primitive pass wrote
// (their states do not change).
template <int N, int D>
__device__ __forceinline__ void update32p_cell(int64_t c, const double* Wn, const double* Wsrc, double* Wout,
                                               const double* __restrict__ F0, const double* __restrict__ F1,
                                               const double* __restrict__ F2, const DevGrid& g, const DevFluid& f,
                                               StepState* st, double a, double b, int relax, int count,
                                               float* __restrict__ P32, float* __restrict__ R32,
                                               double* s = nullptr) {
  using L = Lay<N, D>;
  using Q = P32Lay<N, D>;
  constexpr int M = L::M;
  const int64_t nc = g.ncells;
  // the cell's five-equation CFL speeds (|u_d| + c) / dx_d, as k_prim32 forms them
  auto speeds = [&](const float* u, float cs) {
#pragma unroll
    for (int d = 0; d < D; ++d) s[d] = widen_f32((fabsf(u[d]) + cs) * narrow_f64(g.inv_dx[d]));
  };
  double Ws[M], Wo[M];
#pragma unroll
  for (int m = 0; m < M; ++m) Ws[m] = Wsrc[m * nc + c];
  const bool with_wn = a != 0.0;
  if ((!relax || st->wn_relaxed) && stage_keeps_cell<N, D>(c, Wn, Ws, F0, F1, F2, g, with_wn)) {
    // W_out = W_src exactly, and the planes already hold those of W_src
    if (Wout != Wsrc && !(with_wn && Wout == Wn)) {
#pragma unroll
      for (int m = 0; m < M; ++m) Wout[m * nc + c] = Ws[m];
    }
    if (count) count_bits(st, admissibility_bits<N, D>(Ws, f));
    if (s) {
      float u[D];
#pragma unroll
      for (int d = 0; d < D; ++d) u[d] = P32[(int64_t)(L::MOM + d) * nc + c];
      speeds(u, P32[(int64_t)Q::C * nc + c]);
    }
    return;
  }
  fast_combine<N, D>(c, Wn, Ws, F0, F1, F2, g, st->dt, a, b, Wo);
  double rho, Re;
  if (relax)
    relax_fast<N, D>(Wo, f, rho, Re);
  else
    rho_Re<N, D>(Wo, f, rho, Re);
  if (count) count_bits(st, admissibility_bits<N, D>(Wo, f));
#pragma unroll
  for (int m = 0; m < M; ++m) Wout[m * nc + c] = Wo[m];
  float u[D], cs;
  prim32_store<N, D>(c, Wo, rho, Re, P32, R32, nc, f, u, cs);
  if (s) speeds(u, cs);
}

template <int N, int D>
__global__ void __launch_bounds__(kCellThreads)
    k_update32p(const double* Wn, const double* Wsrc, double* Wout, const double* __restrict__ F0,
                const double* __restrict__ F1, const double* __restrict__ F2, DevGrid g, DevFluid f,
                StepState* st, double a, double b, int relax, int count, float* __restrict__ P32,
                float* __restrict__ R32, int tau = 0) {
  const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (!tau) {
    if (c >= g.nint) return;
    update32p_cell<N, D>(c, Wn, Wsrc, Wout, F0, F1, F2, g, f, st, a, b, relax, count, P32, R32);
    return;
  }
  // a step's last stage (tau): the next step's planes and CFL maxima as well,
  // which k_prim32 then leaves as they are (grids without Dirichlet slices,
  // whose cells this kernel does not cover)
  double s[D];
#pragma unroll
  for (int d = 0; d < D; ++d) s[d] = 0.0;
  if (c < g.nint) update32p_cell<N, D>(c, Wn, Wsrc, Wout, F0, F1, F2, g, f, st, a, b, relax, count, P32, R32, s);
  block_tau_max<D>(s, st->tau_bits);
}

// DEFER: where a screen fails (or for the first-order scheme) return false
// without writing the midpoint, so that the FP64 fallback code is not part of
// the kernel; the midpoint is then computed by the full body (k_face32_fix).
// Returns true when the midpoint's outputs were written.
// XSMEM: the per-thread column of biased values lives in `xs` (the caller's
// shared memory, 2 x M x kFaceThreads floats) instead of a static array of its own.
// nonuniform: the caller has found the stencil not uniform (uniform_stencil).
template <int N, int D, int DIR, bool DEFER = false, bool XSMEM = false>
__device__ __forceinline__ bool face32_body(int64_t t, const Nodes6& nd, const double* __restrict__ W,
                                            const double* __restrict__ V, const double* __restrict__ AUX,
                                            const float* __restrict__ P32, double* __restrict__ out,
                                            const DevGrid& g, const DevFluid& f, const DevParams& pr, double lam,
                                            bool lin = false, float* xs = nullptr, bool nonuniform = false) {
  using L = Lay<N, D>;
  using Q = P32Lay<N, D>;
  constexpr int M = L::M;
  const int64_t nc = g.ncells;
  const int64_t nf = face_count<DIR>(g);
  auto ld = [&](int plane, int j) -> float { return P32[(int64_t)plane * nc + nd.c[j]]; };
  // node state j in FP64 from W (the FP64 limiters' inputs where a screen fails);
  // returns rho c^2
  auto load_node = [&](int j, double* Vn, double* Wn) -> double {
    double w[M], rho, cs, rc2;
#pragma unroll
    for (int m = 0; m < M; ++m) {
      w[m] = W[m * nc + nd.c[j]];
      if (Wn) Wn[m] = w[m];
    }
    cell_prim<N, D>(w, f, Vn, rho, cs, rc2);
    return rc2;
  };
  // first-order HLLC in FP32 from the node states, alpha slots in FP64
  auto first_order = [&](const double* Vi, const double* Vj, FluxPack<N, D>& H) {
    PrimState<float, N, D> a, b;
#pragma unroll
    for (int m = 0; m < M; ++m) {
      a.V[m] = ld(m, 2);
      b.V[m] = ld(m, 3);
    }
    float GH[M];
    const double uH = (double)hllc<float, N, D, DIR>(f, a, b, GH);
#pragma unroll
    for (int m = 0; m < L::NC; ++m) H.Gc[m] = (double)GH[m];
#pragma unroll
    for (int k = 0; k < N - 1; ++k) {
      const double ga = alpha_flux(Vi[L::AL + k], Vj[L::AL + k], uH);
      H.gm[k] = ga - uH * Vi[L::AL + k];
      H.gp[k] = ga - uH * Vj[L::AL + k];
    }
  };

  FluxPack<N, D> G;
  if (pr.scheme == 1) {
    if constexpr (DEFER) return false;
    double Vi[M], Vj[M];
    load_node(2, Vi, nullptr);
    load_node(3, Vj, nullptr);
    first_order(Vi, Vj, G);
  } else {
    // Uniform stencil: the scheme's midpoint flux is then the node's physical
    // flux with zero alpha slots, in exact arithmetic. WENO-IS reproduces a
    // constant (App. C), so both interpolated states equal the node state; the
    // HLLC flux of two equal states is their physical flux (Sec. 4.1.1); the HCS
    // weights psi - 2 a1 + 2 a2 - 2 a3 sum to one, so any sensor blend returns
    // it; the node state is a limiter's first-order candidate as well, so both
    // positivity limiters, whatever their theta or hard switch, return it
    // (Sec. 4.3.2); and with no alpha differences the quasi-conservative alpha
    // slots vanish. Here that value is formed directly (the node flux of the
    // conservative planes, as the HCS term reads it) instead of through rounded
    // steps that would only cancel; every FP32 sweep takes the same exit, so
    // they stay bit-identical to one another.
    if (!nonuniform && uniform_stencil<N, D, XSMEM>(P32, nc, nd)) {
      // (uniform_flux, written out here: as a call the sweep spills more)
      const float un = ld(L::MOM + DIR, 2), pn = ld(L::EN, 2);
#pragma unroll
      for (int m = 0; m < L::NC; ++m) {
        float v;
        if (m < L::MOM)
          v = ld(m, 2) * un;
        else if (m < L::EN)
          v = ld(Q::MOM + (m - L::MOM), 2) * un + ((m - L::MOM) == DIR ? pn : 0.f);
        else
          v = (ld(Q::E, 2) + pn) * un;
        out[m * nf + t] = widen_f32(v);
      }
#pragma unroll
      for (int k = 0; k < N - 1; ++k) {
        out[(L::AL + k) * nf + t] = 0.0;
        out[(M + k) * nf + t] = 0.0;
      }
      return true;
    }
    float p6[6], u6[6];
#pragma unroll
    for (int j = 0; j < 6; ++j) {
      p6[j] = ld(L::EN, j);
      u6[j] = ld(L::MOM + DIR, j);
    }
    const float rhob = 0.5f * (ld(Q::RHO, 2) + ld(Q::RHO, 3));
    const float cb = 0.5f * (ld(Q::C, 2) + ld(Q::C, 3));
    const float inv_rc = 1.f / (rhob * cb);
    const float rc2b = rhob * cb * cb;
    const float eps = pr.weno_eps_f;
    // The N + D + 1 characteristic fields other than the volume fractions in one
    // loop, so that the WENO-IS code exists once (the sweep is bound by
    // instruction fetch when it is unrolled): field fi = 0 is u - p/(rho c)
    // (slot 0), 1..N the species alpha_k rho_k - (alpha_k rho_k)~ p/(rho c^2)
    // (slots 1..N), then the tangential velocities (slots N+1..N+D-1) and last
    // u + p/(rho c) (slot M-1). Each field is a node plane (or u_n) plus a
    // multiple of p; the biased values go through a per-thread shared column.
    float* sU;
    if constexpr (XSMEM) {
      sU = xs;
    } else {
      __shared__ float sU_own[2 * M * kFaceThreads];
      sU = sU_own;
    }
    const int tid = threadIdx.x;
    auto col = [&](int side, int slot) -> float& { return sU[(side * M + slot) * kFaceThreads + tid]; };
    // (a gated midpoint skips the projection: see below)
#pragma unroll 1
    for (int fi = 0; fi < (lin ? 0 : L::NC); ++fi) {
      int plane = -1;  // -1: the normal velocity
      float cp;        // coefficient of p
      if (fi == 0 || fi == N + D) {
        cp = fi == 0 ? -inv_rc : inv_rc;
      } else if (fi <= N) {
        plane = fi - 1;
        cp = -((0.5f * (ld(plane, 2) + ld(plane, 3))) / rc2b);
      } else {
        const int t_ = fi - N - 1;
        plane = L::MOM + (t_ < DIR ? t_ : t_ + 1);
        cp = 0.f;
      }
      // The projection is linear with the midpoint's frozen eigenvectors, so the
      // field is interpolated as increments: d6[j] is the projection of the
      // primitive differences V_j - V_i (exactly zero where they vanish), the
      // columns take the WENO-IS increments about node i (left) and node i+1
      // (right), and the back-projection below adds R times them to the node
      // values. In exact arithmetic the same as interpolating the projected
      // values and back-projecting them; in FP32 it keeps the projection's
      // rounding off a uniform or nearly uniform stencil.
      float d6[6];
      const float v2 = plane < 0 ? u6[2] : ld(plane, 2);
#pragma unroll
      for (int j = 0; j < 6; ++j) d6[j] = ((plane < 0 ? u6[j] : ld(plane, j)) - v2) + cp * (p6[j] - p6[2]);
      const int slot = fi == N + D ? M - 1 : fi;
      col(0, slot) = weno_increment(d6[0], d6[1], d6[3], d6[4], eps);
      col(1, slot) = weno_increment(d6[5] - d6[3], d6[4] - d6[3], -d6[3], d6[1] - d6[3], eps);
    }
    float UL[M], UR[M], arb[N];
    if (!lin) {
#pragma unroll
      for (int m = 0; m < M; ++m) {
        if (m >= N + D && m < M - 1) continue;  // volume fractions: below
        UL[m] = col(0, m);
        UR[m] = col(1, m);
      }
#pragma unroll
      for (int k = 0; k < N; ++k) arb[k] = 0.5f * (ld(k, 2) + ld(k, 3));
    }
    // volume fractions (float-float): node values ai, aj from the value and
    // residue planes, node differences dA[k][j] = alpha_j - alpha_i, and the
    // WENO-IS increments of the identity fields (on FP32 differences) that give
    // the midpoint values aL = ai + incL, aR = aj + incR
    constexpr int NA = N > 1 ? N - 1 : 1;
    ff ai[NA], aj[NA], dA[NA][6], at_L[NA], at_R[NA];
    float incL[NA], incR[NA];
#pragma unroll
    for (int k = 0; k < N - 1; ++k) {
      float hi6[6], lo6[6];
#pragma unroll
      for (int j = 0; j < 6; ++j) {
        hi6[j] = ld(L::AL + k, j);
        lo6[j] = ld(Q::ALO + k, j);
      }
      ai[k] = ff{hi6[2], lo6[2]};
      aj[k] = ff{hi6[3], lo6[3]};
#pragma unroll
      for (int j = 0; j < 6; ++j) {
        const ff dh = ff_sum(hi6[j], -hi6[2]);
        dA[k][j] = ff_sum(dh.hi, dh.lo + (lo6[j] - lo6[2]));
      }
      auto dl = [&](int j, int c) { return (hi6[j] - hi6[c]) + (lo6[j] - lo6[c]); };
      incL[k] = weno_increment(dl(0, 2), dl(1, 2), dl(3, 2), dl(4, 2), eps, lin);
      incR[k] = weno_increment(dl(5, 3), dl(4, 3), dl(2, 3), dl(1, 3), eps, lin);
      at_L[k] = ff_add(ai[k], ff{incL[k], 0.f});
      at_R[k] = ff_add(aj[k], ff{incR[k], 0.f});
      UL[N + D + k] = ff_f(at_L[k]);
      UR[N + D + k] = ff_f(at_R[k]);
    }
    PrimState<float, N, D> sl, sr;
    if (lin) {
      // Gated midpoint: with the linear weights the interpolation sum_k d_k S_k
      // is linear in the node values, so it commutes with the characteristic
      // projection (R sum_k d_k S_k(R^-1 v) = sum_k d_k S_k(v)) and the primitive
      // variables are interpolated directly; the volume fractions as above.
      auto lin5 = [](float um2, float um1, float u0, float up1, float up2) {
        return u0 + lin_increment(um2 - u0, um1 - u0, up1 - u0, up2 - u0);
      };
      float v6[6];
#pragma unroll
      for (int m = 0; m < L::NC; ++m) {
#pragma unroll
        for (int j = 0; j < 6; ++j) v6[j] = m == L::MOM + DIR ? u6[j] : (m == L::EN ? p6[j] : ld(m, j));
        sl.V[m] = lin5(v6[0], v6[1], v6[2], v6[3], v6[4]);
        sr.V[m] = lin5(v6[5], v6[4], v6[3], v6[2], v6[1]);
      }
#pragma unroll
      for (int k = 0; k < N - 1; ++k) {
        sl.V[L::AL + k] = UL[N + D + k];
        sr.V[L::AL + k] = UR[N + D + k];
      }
    } else {
      float h[N];
#pragma unroll
      for (int k = 0; k < N; ++k) h[k] = arb[k] / (2.f * cb);
      const float rc_2 = rhob * cb * 0.5f;
#pragma unroll
      for (int side = 0; side < 2; ++side) {
        const float* U = side == 0 ? UL : UR;  // increments (the volume fractions: values)
        float* Vt = side == 0 ? sl.V : sr.V;
        const int j = 2 + side;                // node i or i+1
#pragma unroll
        for (int k = 0; k < N; ++k) Vt[k] = ld(k, j) + (U[1 + k] + h[k] * (U[M - 1] - U[0]));
        Vt[L::MOM + DIR] = u6[j] + 0.5f * (U[0] + U[M - 1]);
        int t_ = 0;
#pragma unroll
        for (int d = 0; d < D; ++d) {
          if (d == DIR) continue;
          Vt[L::MOM + d] = ld(L::MOM + d, j) + U[N + 1 + t_];
          ++t_;
        }
        Vt[L::EN] = p6[j] + rc_2 * (U[M - 1] - U[0]);
#pragma unroll
        for (int k = 0; k < N - 1; ++k) Vt[L::AL + k] = U[N + D + k];
      }
    }
    // midpoint volume fractions relative to node i (the upwind candidates of
    // the alpha flux): dL = aL - alpha_i, dR = aR - alpha_i
    ff dL[NA], dR[NA];
#pragma unroll
    for (int k = 0; k < N - 1; ++k) {
      dL[k] = ff{incL[k], 0.f};
      dR[k] = ff_add(dA[k][3], ff{incR[k], 0.f});
    }
    if (pr.limiters) {
      // FP64 limiter where the screen cannot certify it; volume fractions it
      // leaves unchanged keep their float-float values (so that the result
      // does not depend on whether the screen ran)
      if (!(pr.screen && interp_screen32<N, D>(sl.V, at_L, f, pr))) {
        if constexpr (DEFER) return false;
        double Vn[M], a0[NA], a1[NA];
        const double rc2n = load_node(2, Vn, nullptr);
#pragma unroll
        for (int k = 0; k < N - 1; ++k) a0[k] = a1[k] = Vn[L::AL + k] + (double)incL[k];
        interp_limit32<N, D>(sl.V, a1, Vn, rc2n, f, pr);
#pragma unroll
        for (int k = 0; k < N - 1; ++k) {
          if (a1[k] != a0[k])
            dL[k] = ff_of(a1[k] - Vn[L::AL + k]);
          else
            sl.V[L::AL + k] = UL[N + D + k];
        }
      }
      if (!(pr.screen && interp_screen32<N, D>(sr.V, at_R, f, pr))) {
        if constexpr (DEFER) return false;
        double Vn[M], a0[NA], a1[NA];
        const double rc2n = load_node(3, Vn, nullptr);
#pragma unroll
        for (int k = 0; k < N - 1; ++k) a0[k] = a1[k] = Vn[L::AL + k] + (double)incR[k];
        interp_limit32<N, D>(sr.V, a1, Vn, rc2n, f, pr);
#pragma unroll
        for (int k = 0; k < N - 1; ++k) {
          if (a1[k] != a0[k])
            dR[k] = ff_of(a1[k] - W[(L::AL + k) * nc + nd.c[2]]);
          else
            sr.V[L::AL + k] = UR[N + D + k];
        }
      }
    }
    float Gt[M];
    const float ut = hllc<float, N, D, DIR>(f, sl, sr, Gt);
    constexpr float psi = 256.0f / 175.0f;
    constexpr float a1 = 101.0f / 420.0f, a2 = 1.0f / 105.0f, a3 = 1.0f / 2100.0f;
    float sig = 0.f;
    if (pr.blend) {
      float r6[6];
#pragma unroll
      for (int j = 0; j < 6; ++j) r6[j] = ld(Q::RHO, j);
      auto half = [](float a, float b, float c, float d, float e) -> float {
        const float num = fabsf(16.f * b - a - 30.f * c + 16.f * d - e);
        const float den = fabsf(a + 16.f * b + 30.f * c + 16.f * d + e);
        return den == 0.f ? 0.f : num / den;
      };
      const float sr_ = 0.5f * (half(r6[1], r6[2], r6[3], r6[4], r6[5]) + half(r6[0], r6[1], r6[2], r6[3], r6[4]));
      const float sp_ = 0.5f * (half(p6[1], p6[2], p6[3], p6[4], p6[5]) + half(p6[0], p6[1], p6[2], p6[3], p6[4]));
      const float prod = sr_ * sp_;
      float pw = prod;
      for (int e = 1; e < pr.qexp; ++e) pw = pw * prod;
      sig = tanhf(pr.Cs_f * pw);
    }
    // HCS and the sensor blend as deviations from r, the mean of the two
    // nodes' values: the HCS weights sum to one (psi - 2 a1 + 2 a2 - 2 a3 = 1),
    // so in exact arithmetic this is psi g~ - a1 (g_i + g_i+1) + a2 (...) -
    // a3 (...) blended as sig g~ + (1 - sig) g_HCS; in FP32 its rounding scales
    // with the deviations and vanishes where all inputs equal r.
    auto hcs_blend = [&](float gt, float g0, float g1, float g2, float g3, float g4, float g5) -> float {
      const float r = 0.5f * (g2 + g3);
      const float h = r + (psi * (gt - r) - a1 * ((g2 - r) + (g3 - r)) + a2 * ((g1 - r) + (g4 - r)) -
                           a3 * ((g0 - r) + (g5 - r)));
      return h + sig * (gt - h);
    };
    const float uhat = hcs_blend(ut, u6[0], u6[1], u6[2], u6[3], u6[4], u6[5]);
    float g32[L::NC];
#pragma unroll
    for (int m = 0; m < L::NC; ++m) {
      float Gn[6];
#pragma unroll
      for (int j = 0; j < 6; ++j) {
        const float un = u6[j];
        float v;
        if (m < L::MOM)
          v = ld(m, j) * un;
        else if (m < L::EN)
          v = ld(Q::MOM + (m - L::MOM), j) * un + ((m - L::MOM) == DIR ? p6[j] : 0.f);
        else
          v = (ld(Q::E, j) + p6[j]) * un;
        Gn[j] = v;
      }
      g32[m] = hcs_blend(Gt[m], Gn[0], Gn[1], Gn[2], Gn[3], Gn[4], Gn[5]);
      G.Gc[m] = widen_f32(g32[m]);
    }
    // alpha slots, quasi-conservative form (Eq. G_pm): with alpha_j = alpha_i +
    // dA_j, the blended HCS alpha flux is alpha_i u^ + Rh, where u^ is the blended
    // HCS velocity and Rh the same combination of dA_j u_j and of the upwind
    // midpoint difference times u~; so G^- = Rh and G^+ = Rh - u^ dA_{i+1}
    // exactly, and both are formed in float-float (a uniform alpha gives zero).
    ff gmf[NA], gpf[NA];
    {
      const ff PSI = HRM_FF(256.0 / 175.0), C1 = HRM_FF(101.0 / 420.0), C2 = HRM_FF(1.0 / 105.0),
               C3 = HRM_FF(1.0 / 2100.0);
      const ff om = ff_sum(1.f, -sig);
#pragma unroll
      for (int k = 0; k < N - 1; ++k) {
        const ff dup = ut > 0.f ? dL[k] : (ut < 0.f ? dR[k] : ff{0.f, 0.f});
        const ff A = ff_mulf(dup, ut);
        ff B = ff_mul(PSI, A);
        B = ff_sub(B, ff_mul(C1, ff_mulf(dA[k][3], u6[3])));
        B = ff_add(B, ff_mul(C2, ff_add(ff_mulf(dA[k][1], u6[1]), ff_mulf(dA[k][4], u6[4]))));
        B = ff_sub(B, ff_mul(C3, ff_add(ff_mulf(dA[k][0], u6[0]), ff_mulf(dA[k][5], u6[5]))));
        gmf[k] = ff_add(ff_mulf(A, sig), ff_mul(om, B));
        gpf[k] = ff_sub(gmf[k], ff_mulf(dA[k][3], uhat));
        G.gm[k] = ff_d(gmf[k]);
        G.gp[k] = ff_d(gpf[k]);
      }
    }
    if (pr.limiters &&
        !(pr.screen && flux_screen32<N, D, DIR>(P32, nc, nd, g32, gmf, gpf, ai, aj, ff_of(2.0 * lam), f, pr))) {
      if constexpr (DEFER) return false;
      double Vi[M], Vj[M], Wi[M], Wj[M];
      load_node(2, Vi, Wi);
      load_node(3, Vj, Wj);
      FluxPack<N, D> H;
      first_order(Vi, Vj, H);
      double Fi[L::NC], Fj[L::NC];
      node_flux<N, D, DIR>(Wi, Vi, Fi);
      node_flux<N, D, DIR>(Wj, Vj, Fj);
      flux_limit<N, D, DIR, true>(Wi, Wj, Fi, Fj, lam, G, H, f, pr, Vi, Vj);
    }
  }
#pragma unroll
  for (int m = 0; m < L::NC; ++m) out[m * nf + t] = G.Gc[m];
#pragma unroll
  for (int k = 0; k < N - 1; ++k) {
    out[(L::AL + k) * nf + t] = G.gm[k];
    out[(M + k) * nf + t] = G.gp[k];
  }
  return true;
}

// Screened sweep without the FP64 fallbacks (about a third of the full body's
// code and at most 80 registers, so six blocks per SM, with some values
// spilled; seven or more blocks changed the compiler's FP32 contraction):
// midpoints whose screens fail are appended to `list` (warp-aggregated; order
// not significant) for k_face32_fix. *count must be 0 at launch; list holds one
// entry per midpoint.
template <int N, int D, int DIR>
__global__ void __launch_bounds__(kFaceThreads, 6)
    k_face32_fast(const double* __restrict__ W, const float* __restrict__ P32, double* __restrict__ out, DevGrid g,
                  DevFluid f, DevParams pr, const StepState* __restrict__ st, const uint8_t* __restrict__ gate,
                  uint32_t* __restrict__ list, uint32_t* __restrict__ count) {
  const int64_t t = patch_midpoint<DIR>(g);
  Nodes6 nd;
  bool need = false;
  if (face_nodes<DIR>(g, t, nd)) {
    const bool lin = gate != nullptr && gate[t] != 0;
    need = !face32_body<N, D, DIR, true>(t, nd, W, nullptr, nullptr, P32, out, g, f, pr, st->lam[DIR], lin);
  }
  defer_push(need, t, list, count);
}

// The midpoints a k_face32_fast launch deferred, with the full body (FP64
// limiters where the screens fail). The list is short (tens to hundreds of
// midpoints) and each entry is a long chain of FP64 work, so entries go to
// one-warp blocks lane-major: entry i to block i mod gridDim, spreading a
// short list over every SM rather than packing it into a few warps.
template <int N, int D, int DIR>
__global__ void __launch_bounds__(kFaceThreads, 2)
    k_face32_fix(const double* __restrict__ W, const float* __restrict__ P32, double* __restrict__ out, DevGrid g,
                 DevFluid f, DevParams pr, const StepState* __restrict__ st, const uint8_t* __restrict__ gate,
                 const uint32_t* __restrict__ list, const uint32_t* __restrict__ count) {
  const int64_t n = *count;
  for (int64_t r = threadIdx.x;; r += blockDim.x) {
    const int64_t i = r * gridDim.x + blockIdx.x;
    if (i >= n) break;
    const int64_t t = list[i];
    Nodes6 nd;
    if (!face_nodes<DIR>(g, t, nd)) continue;
    const bool lin = gate != nullptr && gate[t] != 0;
    face32_body<N, D, DIR>(t, nd, W, nullptr, nullptr, P32, out, g, f, pr, st->lam[DIR], lin);
  }
}

template <int N, int D, int DIR>
__global__ void __launch_bounds__(kFaceThreads, 3)
    k_face32(const double* __restrict__ W, const double* __restrict__ V, const double* __restrict__ AUX,
             const float* __restrict__ P32, double* __restrict__ out, DevGrid g, DevFluid f, DevParams pr,
             const StepState* __restrict__ st, const uint8_t* __restrict__ gate) {
  const int64_t t = patch_midpoint<DIR>(g);
  Nodes6 nd;
  if (!face_nodes<DIR>(g, t, nd)) return;
  const bool lin = gate != nullptr && gate[t] != 0;
  face32_body<N, D, DIR>(t, nd, W, V, AUX, P32, out, g, f, pr, st->lam[DIR], lin);
}

}  // namespace hrm
