// Precision form of the per-midpoint kernel: characteristic projection,
// WENO-IS, both HLLC solves, HCS and the sensor blend in FP32; the
// interpolation-limiter and flux-limiter theta solves, the half-cell states and
// everything downstream (flux difference, RK combination, relaxation) in FP64.
#pragma once

#include "hrm_kernels.cuh"

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

__device__ __forceinline__ float weno_is_scaled(float um2, float um1, float u0, float up1, float up2, float eps,
                                                bool lin = false) {
  float a = um2 - u0, b = um1 - u0, d = up1 - u0, e = up2 - u0;
  if (lin) return u0 + lin_increment(a, b, d, e);
  const float s = fmaxf(fmaxf(fabsf(a), fabsf(b)), fmaxf(fabsf(d), fabsf(e)));
  if (!(s > kTinyRange)) return u0;
  const float inv = 1.f / s;
  a *= inv;
  b *= inv;
  d *= inv;
  e *= inv;
  const float eps_s = fmaxf(eps * inv * inv, 1e-15f);
  return u0 + s * weno_is<float>(a, b, 0.f, d, e, eps_s);
}

// WENO-IS increment from already-formed differences (u_j - u_0) of a stencil
// whose central value is the reference (left-biased order um2, um1, up1, up2).
__device__ __forceinline__ float weno_increment(float a, float b, float d, float e, float eps, bool lin = false) {
  if (lin) return lin_increment(a, b, d, e);
  const float s = fmaxf(fmaxf(fabsf(a), fabsf(b)), fmaxf(fabsf(d), fabsf(e)));
  if (!(s > kTinyRange)) return 0.f;
  const float inv = 1.f / s;
  const float eps_s = fmaxf(eps * inv * inv, 1e-15f);
  return s * weno_is<float>(a * inv, b * inv, 0.f, d * inv, e * inv, eps_s);
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

template <int N, int D, int DIR>
__device__ __forceinline__ void face32_body(int64_t t, const Nodes6& nd, const double* __restrict__ W,
                                            const double* __restrict__ V, const double* __restrict__ AUX,
                                            const float* __restrict__ P32, double* __restrict__ out,
                                            const DevGrid& g, const DevFluid& f, const DevParams& pr, double lam,
                                            bool lin = false) {
  using L = Lay<N, D>;
  using Q = P32Lay<N, D>;
  constexpr int M = L::M;
  const int64_t nc = g.ncells;
  const int64_t nf = face_count<DIR>(g);
  auto ld = [&](int plane, int j) -> float { return P32[(int64_t)plane * nc + nd.c[j]]; };

  // node states i, i+1 in FP64 for the limiters
  double Vi[M], Vj[M], Wi[M], Wj[M];
#pragma unroll
  for (int m = 0; m < M; ++m) {
    Vi[m] = V[m * nc + nd.c[2]];
    Vj[m] = V[m * nc + nd.c[3]];
    Wi[m] = W[m * nc + nd.c[2]];
    Wj[m] = W[m * nc + nd.c[3]];
  }

  // first-order HLLC in FP32 from the node states
  FluxPack<N, D> H;
  {
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
  }

  FluxPack<N, D> G;
  if (pr.scheme == 1) {
    G = H;
  } else {
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
    const float eps = (float)pr.weno_eps;
    float UL[M], UR[M], w6[6];
#pragma unroll
    for (int j = 0; j < 6; ++j) w6[j] = u6[j] - inv_rc * p6[j];
    UL[0] = weno_is_scaled(w6[0], w6[1], w6[2], w6[3], w6[4], eps, lin);
    UR[0] = weno_is_scaled(w6[5], w6[4], w6[3], w6[2], w6[1], eps, lin);
#pragma unroll
    for (int j = 0; j < 6; ++j) w6[j] = u6[j] + inv_rc * p6[j];
    UL[M - 1] = weno_is_scaled(w6[0], w6[1], w6[2], w6[3], w6[4], eps, lin);
    UR[M - 1] = weno_is_scaled(w6[5], w6[4], w6[3], w6[2], w6[1], eps, lin);
    float arb[N];
#pragma unroll
    for (int k = 0; k < N; ++k) {
#pragma unroll
      for (int j = 0; j < 6; ++j) w6[j] = ld(k, j);
      arb[k] = 0.5f * (w6[2] + w6[3]);
      const float coef = arb[k] / rc2b;
#pragma unroll
      for (int j = 0; j < 6; ++j) w6[j] = w6[j] - coef * p6[j];
      UL[1 + k] = weno_is_scaled(w6[0], w6[1], w6[2], w6[3], w6[4], eps, lin);
      UR[1 + k] = weno_is_scaled(w6[5], w6[4], w6[3], w6[2], w6[1], eps, lin);
    }
    {
      int t_ = 0;
#pragma unroll
      for (int d = 0; d < D; ++d) {
        if (d == DIR) continue;
#pragma unroll
        for (int j = 0; j < 6; ++j) w6[j] = ld(L::MOM + d, j);
        UL[N + 1 + t_] = weno_is_scaled(w6[0], w6[1], w6[2], w6[3], w6[4], eps, lin);
        UR[N + 1 + t_] = weno_is_scaled(w6[5], w6[4], w6[3], w6[2], w6[1], eps, lin);
        ++t_;
      }
    }
    // volume fractions: increments of the identity fields on exact differences
    // (FP32 value differences plus residue differences), added to the FP64 node values
    double aL[N > 1 ? N - 1 : 1], aR[N > 1 ? N - 1 : 1];
#pragma unroll
    for (int k = 0; k < N - 1; ++k) {
      float hi6[6], lo6[6];
#pragma unroll
      for (int j = 0; j < 6; ++j) {
        hi6[j] = ld(L::AL + k, j);
        lo6[j] = ld(Q::ALO + k, j);
      }
      auto dl = [&](int j, int c) { return (hi6[j] - hi6[c]) + (lo6[j] - lo6[c]); };
      aL[k] = Vi[L::AL + k] + (double)weno_increment(dl(0, 2), dl(1, 2), dl(3, 2), dl(4, 2), eps, lin);
      aR[k] = Vj[L::AL + k] + (double)weno_increment(dl(5, 3), dl(4, 3), dl(2, 3), dl(1, 3), eps, lin);
      UL[N + D + k] = (float)aL[k];
      UR[N + D + k] = (float)aR[k];
    }
    PrimState<float, N, D> sl, sr;
    {
      float h[N];
#pragma unroll
      for (int k = 0; k < N; ++k) h[k] = arb[k] / (2.f * cb);
      const float rc_2 = rhob * cb * 0.5f;
#pragma unroll
      for (int side = 0; side < 2; ++side) {
        const float* U = side == 0 ? UL : UR;
        float* Vt = side == 0 ? sl.V : sr.V;
#pragma unroll
        for (int k = 0; k < N; ++k) Vt[k] = U[1 + k] + h[k] * (U[M - 1] - U[0]);
        Vt[L::MOM + DIR] = 0.5f * (U[0] + U[M - 1]);
        int t_ = 0;
#pragma unroll
        for (int d = 0; d < D; ++d) {
          if (d == DIR) continue;
          Vt[L::MOM + d] = U[N + 1 + t_];
          ++t_;
        }
        Vt[L::EN] = rc_2 * (U[M - 1] - U[0]);
#pragma unroll
        for (int k = 0; k < N - 1; ++k) Vt[L::AL + k] = U[N + D + k];
      }
    }
    if (pr.limiters) {
      interp_limit32<N, D>(sl.V, aL, Vi, AUX[2 * nc + nd.c[2]], f, pr);
      interp_limit32<N, D>(sr.V, aR, Vj, AUX[2 * nc + nd.c[3]], f, pr);
    }
    float Gt[M];
    const float ut = hllc<float, N, D, DIR>(f, sl, sr, Gt);
    double Gt_a[N > 1 ? N - 1 : 1];
#pragma unroll
    for (int k = 0; k < N - 1; ++k) Gt_a[k] = alpha_flux(aL[k], aR[k], (double)ut);
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
      sig = tanhf((float)pr.Cs * pw);
    }
    const float one_m = 1.f - sig;
    const float uhcs = psi * ut - a1 * (u6[2] + u6[3]) + a2 * (u6[1] + u6[4]) - a3 * (u6[0] + u6[5]);
    const double uhat = (double)(sig * ut + one_m * uhcs);
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
      const float ghcs = psi * Gt[m] - a1 * (Gn[2] + Gn[3]) + a2 * (Gn[1] + Gn[4]) - a3 * (Gn[0] + Gn[5]);
      G.Gc[m] = (double)(sig * Gt[m] + one_m * ghcs);
    }
    // alpha slots in FP64: node fluxes alpha_j u_j, HCS, blend, quasi-conservative form
    {
      constexpr double dpsi = 256.0 / 175.0, d1 = 101.0 / 420.0, d2 = 1.0 / 105.0, d3 = 1.0 / 2100.0;
      const double sg = (double)sig, om = 1.0 - sg;
#pragma unroll
      for (int k = 0; k < N - 1; ++k) {
        double gn[6];
#pragma unroll
        for (int j = 0; j < 6; ++j) gn[j] = V[(L::AL + k) * nc + nd.c[j]] * (double)u6[j];
        const double ghcs = dpsi * Gt_a[k] - d1 * (gn[2] + gn[3]) + d2 * (gn[1] + gn[4]) - d3 * (gn[0] + gn[5]);
        const double gh = sg * Gt_a[k] + om * ghcs;
        G.gm[k] = gh - uhat * Vi[L::AL + k];
        G.gp[k] = gh - uhat * Vj[L::AL + k];
      }
    }
    if (pr.limiters) {
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
}

template <int N, int D, int DIR>
__global__ void __launch_bounds__(kFaceThreads)
    k_face32(const double* __restrict__ W, const double* __restrict__ V, const double* __restrict__ AUX,
             const float* __restrict__ P32, double* __restrict__ out, DevGrid g, DevFluid f, DevParams pr,
             const StepState* __restrict__ st, const uint8_t* __restrict__ gate) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  Nodes6 nd;
  if (!face_nodes<DIR>(g, t, nd)) return;
  const bool lin = gate != nullptr && gate[t] != 0;
  face32_body<N, D, DIR>(t, nd, W, V, AUX, P32, out, g, f, pr, st->lam[DIR], lin);
}

}  // namespace hrm
