// Kernel templates of the PP-WCNS-IS fractional step (arXiv 2208.04488).
//
// One RK stage is: k_prim (per cell: primitive variables, sound speed, and at
// the first stage the CFL max-wave-speed reduction) -> k_face for each direction
// (per midpoint: characteristic projection, WENO-IS, interpolation limiter,
// two HLLC solves, HCS reconstruction, shock-sensor blending, quasi-conservative
// fluxes and the flux limiter) -> k_update (per cell: flux difference with the
// non-conservative alpha term, SSP-RK combination, thermal relaxation,
// admissibility counters).
#pragma once

#include "hrm_device.cuh"

namespace hrm {

constexpr int kFaceThreads = 128;
constexpr int kCellThreads = 256;

// Face grid of direction DIR: n with n[DIR] + 1 entries along DIR.
template <int DIR>
__device__ __forceinline__ int64_t face_count(const DevGrid& g) {
  return (g.n[0] + (DIR == 0)) * (g.n[1] + (DIR == 1)) * (g.n[2] + (DIR == 2));
}

// ---------------------------------------------------------------- interpolation limiter

// Positivity-preserving interpolation limiter (Sec. 4.3.2, Alg. interp_limit_densities,
// Alg. interp_limit_vol_frac, hard switch) applied to the midpoint primitive
// state Vt against the first-order (node) state Vn; velocity and pressure are
// held, partial densities and volume fractions are limited, theta in FP64.
template <typename R, int N, int D>
__device__ __forceinline__ void interp_limit(R* Vt, const double* Vn, double rc2n, const DevFluid& f,
                                             const DevParams& pr) {
  using L = Lay<N, D>;
  constexpr int M = L::M;
#pragma unroll
  for (int k = 0; k < N; ++k) {
    const double lo = Vn[k], hi = (double)Vt[k];
    const double tgt = dmin(pr.eps_ar, lo);
    double th = 1.0;
    if (hi < tgt) th = (tgt - lo) / (hi - lo);
    Vt[k] = R((1.0 - th) * lo + th * hi);
  }
  double alt[N], aln[N];
  {
    double st = 0.0, sn = 0.0;
#pragma unroll
    for (int k = 0; k < N - 1; ++k) {
      alt[k] = (double)Vt[L::AL + k];
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
    double thk = 1.0;
    if (alt[k] < tgt) thk = (tgt - aln[k]) / (alt[k] - aln[k]);
    th = dmin(th, thk);
  }
#pragma unroll
  for (int k = 0; k < N - 1; ++k) Vt[L::AL + k] = R((1.0 - th) * aln[k] + th * alt[k]);
  // hard switch
  bool hs = false;
  {
    double st = 0.0;
#pragma unroll
    for (int k = 0; k < N - 1; ++k) {
      alt[k] = (double)Vt[L::AL + k];
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
  const double rc2 = rho_c2(S, P, (double)Vt[L::EN]);
  hs |= rc2 < dmin(pr.hs_rc2, rc2n);
  if (hs) {
#pragma unroll
    for (int m = 0; m < M; ++m) Vt[m] = R(Vn[m]);
  }
}

// ---------------------------------------------------------------- flux limiter helpers

// rho (e - qbar) of a conservative vector (Sec. 2).
template <int N, int D>
__device__ __forceinline__ double rhoe_tilde(const double* W, const DevFluid& f) {
  using L = Lay<N, D>;
  double rho = 0.0, kin = 0.0, rq = 0.0;
#pragma unroll
  for (int k = 0; k < N; ++k) {
    rho += W[k];
    rq += W[k] * f.q[k];
  }
#pragma unroll
  for (int d = 0; d < D; ++d) kin += W[L::MOM + d] * W[L::MOM + d];
  return W[L::EN] - 0.5 * kin / rho - rq;
}

__device__ __forceinline__ double theta_of(double lo, double hi, double eps) {
  const double tgt = dmin(eps, lo);
  return (hi < tgt) ? (tgt - lo) / (hi - lo) : 1.0;
}

// A midpoint flux G^-_{i+1/2} / G^+_{i+1/2} (Eq. G_pm): the conservative slots Gc
// are shared, the alpha slots differ (gm uses alpha_i, gp uses alpha_{i+1}).
template <int N, int D>
struct FluxPack {
  double Gc[Lay<N, D>::NC];
  double gm[N - 1 > 0 ? N - 1 : 1];
  double gp[N - 1 > 0 ? N - 1 : 1];
};

// Half-cell state W_n + s (G - F_n): with minus = true the alpha slots of G^-
// (cell i side), otherwise those of G^+ (cell i+1 side); F has zero alpha slots.
template <int N, int D>
__device__ __forceinline__ void half_state(const double* Wn, const double* Fn, const FluxPack<N, D>& G,
                                           double s, bool minus, double* out) {
  using L = Lay<N, D>;
#pragma unroll
  for (int m = 0; m < L::NC; ++m) out[m] = Wn[m] + s * (G.Gc[m] - Fn[m]);
#pragma unroll
  for (int k = 0; k < N - 1; ++k) out[L::AL + k] = Wn[L::AL + k] + s * (minus ? G.gm[k] : G.gp[k]);
}

template <int N, int D>
__device__ __forceinline__ void mix_pack(const FluxPack<N, D>& H, const FluxPack<N, D>& G, double th,
                                         FluxPack<N, D>& out) {
  using L = Lay<N, D>;
#pragma unroll
  for (int m = 0; m < L::NC; ++m) out.Gc[m] = (1.0 - th) * H.Gc[m] + th * G.Gc[m];
#pragma unroll
  for (int k = 0; k < N - 1; ++k) {
    out.gp[k] = (1.0 - th) * H.gp[k] + th * G.gp[k];
    out.gm[k] = (1.0 - th) * H.gm[k] + th * G.gm[k];
  }
}

template <int N, int D>
__device__ __forceinline__ void all_alpha_W(const double* W, double* al) {
  using L = Lay<N, D>;
  double s = 0.0;
#pragma unroll
  for (int k = 0; k < N - 1; ++k) {
    al[k] = W[L::AL + k];
    s += al[k];
  }
  al[N - 1] = 1.0 - s;
}

// Quasi-positivity-preserving flux limiter (Sec. 4.3.2, Alg.
// flux_limit_densities_vol_frac, Alg. flux_limit_energy, hard switch), FP64.
// Wi/Wj: W_i, W_{i+1}; Fi/Fj: conservative fluxes F(W_i), F(W_{i+1});
// G: high-order midpoint flux, H: first-order HLLC flux; the result replaces G.
//
// The limiter's guarantee rests on the first-order half-cell states being
// admissible, which holds for the HLLC flux in exact arithmetic with no margin
// at CFL 1/2. REPAIR (the precision form, whose H is an FP32 evaluation):
// where a first-order half-cell state comes out inadmissible, H is evaluated
// again in FP64 from the node states Vi, Vj, as the FP64 form does.
template <int N, int D, int DIR = 0, bool REPAIR = false>
__device__ __forceinline__ void flux_limit(const double* Wi, const double* Wj, const double* Fi,
                                           const double* Fj, double lam, FluxPack<N, D>& G,
                                           const FluxPack<N, D>& H_in, const DevFluid& f,
                                           const DevParams& pr, const double* Vi = nullptr,
                                           const double* Vj = nullptr) {
  using L = Lay<N, D>;
  constexpr int M = L::M;
  const double m2l = -2.0 * lam, p2l = 2.0 * lam;
  double Wp[M], Wm[M], WHp[M], WHm[M];
  FluxPack<N, D> H = H_in;
  half_state<N, D>(Wi, Fi, G, m2l, true, Wp);    // W_i^{+}
  half_state<N, D>(Wj, Fj, G, p2l, false, Wm);   // W_{i+1}^{-}
  half_state<N, D>(Wi, Fi, H, m2l, true, WHp);   // W_i^{HLLC,+}
  half_state<N, D>(Wj, Fj, H, p2l, false, WHm);  // W_{i+1}^{HLLC,-}
  // first-order states: volume fractions and rho e~ (also the limiter's lower ends)
  double aHp[N], aHm[N];
  all_alpha_W<N, D>(WHp, aHp);
  all_alpha_W<N, D>(WHm, aHm);
  double rHp = rhoe_tilde<N, D>(WHp, f), rHm = rhoe_tilde<N, D>(WHm, f);
  if constexpr (REPAIR) {
    bool bad = !(rHp > 0.0) || !(rHm > 0.0);
#pragma unroll
    for (int k = 0; k < N; ++k)
      bad |= !(WHp[k] >= 0.0) || !(WHm[k] >= 0.0) || !(aHp[k] >= 0.0) || !(aHm[k] >= 0.0);
    if (bad) {
      PrimState<double, N, D> a, b;
#pragma unroll
      for (int m = 0; m < M; ++m) {
        a.V[m] = Vi[m];
        b.V[m] = Vj[m];
      }
      double GH[M];
      const double uH = hllc<double, N, D, DIR>(f, a, b, GH);
#pragma unroll
      for (int m = 0; m < L::NC; ++m) H.Gc[m] = GH[m];
#pragma unroll
      for (int k = 0; k < N - 1; ++k) {
        H.gm[k] = GH[L::AL + k] - uH * Vi[L::AL + k];
        H.gp[k] = GH[L::AL + k] - uH * Vj[L::AL + k];
      }
      half_state<N, D>(Wi, Fi, H, m2l, true, WHp);
      half_state<N, D>(Wj, Fj, H, p2l, false, WHm);
      all_alpha_W<N, D>(WHp, aHp);
      all_alpha_W<N, D>(WHm, aHm);
      rHp = rhoe_tilde<N, D>(WHp, f);
      rHm = rhoe_tilde<N, D>(WHm, f);
    }
  }
  double th = 1.0;
#pragma unroll
  for (int k = 0; k < N; ++k) {
    th = dmin(th, dmin(theta_of(WHp[k], Wp[k], pr.eps_ar), theta_of(WHm[k], Wm[k], pr.eps_ar)));
  }
  {
    double ap[N], am[N];
    all_alpha_W<N, D>(Wp, ap);
    all_alpha_W<N, D>(Wm, am);
#pragma unroll
    for (int k = 0; k < N; ++k)
      th = dmin(th, dmin(theta_of(aHp[k], ap[k], pr.eps_a), theta_of(aHm[k], am[k], pr.eps_a)));
  }
  // with theta = 1 the mixed flux is G itself, bit for bit ((1 - 1) H + 1 G), and
  // the half-cell states need no recomputation
  FluxPack<N, D> Gs;
  if (th < 1.0) {
    mix_pack<N, D>(H, G, th, Gs);
    half_state<N, D>(Wi, Fi, Gs, m2l, true, Wp);   // W_i^{*,+}
    half_state<N, D>(Wj, Fj, Gs, p2l, false, Wm);  // W_{i+1}^{*,-}
  } else {
    Gs = G;
  }
  // energy stage
  const double th2 = dmin(theta_of(rHp, rhoe_tilde<N, D>(Wp, f), pr.eps_rhoe),
                          theta_of(rHm, rhoe_tilde<N, D>(Wm, f), pr.eps_rhoe));
  FluxPack<N, D> Gss;
  if (th2 < 1.0) {
    mix_pack<N, D>(H, Gs, th2, Gss);
    half_state<N, D>(Wi, Fi, Gss, m2l, true, Wp);   // W_i^{**,+}
    half_state<N, D>(Wj, Fj, Gss, p2l, false, Wm);  // W_{i+1}^{**,-}
  } else {
    Gss = Gs;
  }
  // hard switch
  bool hs = false;
  {
    double ap[N], am[N];
    all_alpha_W<N, D>(Wp, ap);
    all_alpha_W<N, D>(Wm, am);
#pragma unroll
    for (int k = 0; k < N; ++k) {
      hs |= Wp[k] < dmin(pr.hs_ar, WHp[k]);
      hs |= ap[k] < dmin(pr.hs_a, aHp[k]);
      hs |= Wm[k] < dmin(pr.hs_ar, WHm[k]);
      hs |= am[k] < dmin(pr.hs_a, aHm[k]);
    }
  }
  hs |= rhoe_tilde<N, D>(Wp, f) < dmin(pr.hs_rhoe, rHp);
  hs |= rhoe_tilde<N, D>(Wm, f) < dmin(pr.hs_rhoe, rHm);
  G = hs ? H : Gss;
}

// True when the flux limiter provably leaves G unchanged: every checked quantity
// of the high-order half-cell states W_i^{+}, W_{i+1}^{-} (alpha_k rho_k, all N
// alpha_k, rho e~) is at or above both its limiter threshold and its hard-switch
// threshold. Then no theta trigger fires (a_high >= eps >= min(eps, a_low)) and
// no hard switch either, whatever the first-order states, so the first-order
// flux is not needed. The states are those flux_limit forms, bit for bit; NaN
// fails the test.
template <int N, int D>
__device__ __forceinline__ bool flux_limit_noop(const double* Wi, const double* Wj, const double* Fi,
                                                const double* Fj, double lam, const FluxPack<N, D>& G,
                                                const DevFluid& f, const DevParams& pr) {
  using L = Lay<N, D>;
  constexpr int M = L::M;
  double Wp[M], Wm[M], ap[N], am[N];
  half_state<N, D>(Wi, Fi, G, -2.0 * lam, true, Wp);
  half_state<N, D>(Wj, Fj, G, 2.0 * lam, false, Wm);
  all_alpha_W<N, D>(Wp, ap);
  all_alpha_W<N, D>(Wm, am);
  const double tar = pr.eps_ar > pr.hs_ar ? pr.eps_ar : pr.hs_ar;
  const double ta = pr.eps_a > pr.hs_a ? pr.eps_a : pr.hs_a;
  const double tre = pr.eps_rhoe > pr.hs_rhoe ? pr.eps_rhoe : pr.hs_rhoe;
  bool ok = rhoe_tilde<N, D>(Wp, f) >= tre && rhoe_tilde<N, D>(Wm, f) >= tre;
#pragma unroll
  for (int k = 0; k < N; ++k) ok = ok && Wp[k] >= tar && Wm[k] >= tar && ap[k] >= ta && am[k] >= ta;
  return ok;
}

// ---------------------------------------------------------------- per-midpoint kernel

// Loads of the six node cells i-2..i+3 of a midpoint.
struct Nodes6 {
  int64_t c[6];
};

// Midpoint of this thread in a sweep launched over patch_grid blocks of
// kFaceThreads: linear, or patched as above. Past the end of a row or of the
// grid: the midpoint count (no midpoint).
template <int DIR>
__device__ __forceinline__ int64_t patch_midpoint(const DevGrid& g) {
  static_assert(kFaceThreads == 128, "four warps per patch");
  const int64_t f0 = g.n[0] + (DIR == 0), f1 = g.n[1] + (DIR == 1), f2 = g.n[2] + (DIR == 2);
  if (!patched(g, DIR)) return (int64_t)blockIdx.x * kFaceThreads + threadIdx.x;
  const int64_t nbx = (f0 + 31) / 32, b = blockIdx.x;
  const int64_t bx = b % nbx, rest = b / nbx;
  const int w = threadIdx.x >> 5;
  int64_t i1, i2;
  if (DIR == 1) {
    const int64_t nby = (f1 + 3) / 4;
    i1 = (rest % nby) * 4 + w;
    i2 = rest / nby;
  } else {
    i1 = rest % f1;
    i2 = (rest / f1) * 4 + w;
  }
  const int64_t i0 = bx * 32 + (threadIdx.x & 31);
  if (i0 >= f0 || i1 >= f1 || i2 >= f2) return f0 * f1 * f2;
  return (i2 * f1 + i1) * f0 + i0;
}

template <int DIR>
__device__ __forceinline__ bool face_nodes(const DevGrid& g, int64_t t, Nodes6& nd) {
  const int64_t f0 = g.n[0] + (DIR == 0), f1 = g.n[1] + (DIR == 1), f2 = g.n[2] + (DIR == 2);
  if (t >= f0 * f1 * f2) return false;
  const int64_t i0 = t % f0;
  const int64_t r = t / f0;
  const int64_t i1 = r % f1, i2 = r / f1;
  const int64_t fp = DIR == 0 ? i0 : (DIR == 1 ? i1 : i2);
  const bool dlo = g.bc[2 * DIR] == 2, dhi = g.bc[2 * DIR + 1] == 2;
  // cell of the Dirichlet slice that continues this line
  const int64_t tr = DIR == 0 ? i2 * g.n[1] + i1 : (DIR == 1 ? i2 * g.n[0] + i0 : i1 * g.n[0] + i0);
#pragma unroll
  for (int j = 0; j < 6; ++j) {
    const int64_t jj = fp - 3 + j;
    const int64_t q = bc_map(g, DIR, jj);
    nd.c[j] = DIR == 0 ? (i2 * g.n[1] + i1) * g.n[0] + q
                       : (DIR == 1 ? (i2 * g.n[1] + q) * g.n[0] + i0 : (q * g.n[1] + i1) * g.n[0] + i0);
    if (jj < 0 && dlo) nd.c[j] = g.goff[2 * DIR] + tr;
    if (jj >= g.n[DIR] && dhi) nd.c[j] = g.goff[2 * DIR + 1] + tr;
    nd.c[j] = HRM_IDX(g, nd.c[j], g.ncells);
  }
  return true;
}

// Conservative flux F^DIR of a node (Eq. F_x_F_y_def), NC slots.
template <int N, int D, int DIR>
__device__ __forceinline__ void node_flux(const double* W, const double* V, double* F) {
  using L = Lay<N, D>;
  const double un = V[L::MOM + DIR], p = V[L::EN];
#pragma unroll
  for (int k = 0; k < N; ++k) F[k] = W[k] * un;
#pragma unroll
  for (int d = 0; d < D; ++d) F[L::MOM + d] = W[L::MOM + d] * un + (d == DIR ? p : 0.0);
  F[L::EN] = (W[L::EN] + p) * un;
}

// Whether the six node states of a midpoint are bit-identical (every plane of W).
template <int N, int D>
__device__ __forceinline__ bool uniform_nodes(const double* __restrict__ W, int64_t nc, const Nodes6& nd) {
  bool same = true;
#pragma unroll
  for (int m = 0; m < Lay<N, D>::M; ++m) {
    const long long b = __double_as_longlong(W[m * nc + nd.c[2]]);
#pragma unroll
    for (int j = 0; j < 6; ++j)
      if (j != 2) same &= __double_as_longlong(W[m * nc + nd.c[j]]) == b;
  }
  return same;
}

// Outputs of a midpoint: M + N - 1 planes over the face grid of the direction --
// the NC conservative flux slots, the N-1 alpha slots of G^-_{i+1/2} (planes
// AL..M-1) and the N-1 alpha slots of G^+_{i+1/2} (planes M..M+N-2).
// One midpoint t of direction DIR (t inside the face grid); lam = lambda_DIR.
// lin: the midpoint is gated smooth -- the WENO-IS weights are replaced by the
// linear weights d_k; everything else is unchanged.
template <typename R, int N, int D, int DIR>
__device__ __forceinline__ void face_body(int64_t t, const Nodes6& nd, const double* __restrict__ W,
                                          const double* __restrict__ V, const double* __restrict__ AUX,
                                          double* __restrict__ out, const DevGrid& g, const DevFluid& f,
                                          const DevParams& pr, double lam, bool lin = false) {
  using L = Lay<N, D>;
  constexpr int M = L::M;
  const int64_t nc = g.ncells;
  const int64_t nf = face_count<DIR>(g);
  const double* __restrict__ Cc = AUX;           // sound speed
  const double* __restrict__ Rr = AUX + nc;      // mixture density
  const double* __restrict__ RC2 = AUX + 2 * nc; // rho c^2

  // node states i and i+1 (FP64)
  double Vi[M], Vj[M], Wi[M], Wj[M];
#pragma unroll
  for (int m = 0; m < M; ++m) {
    Vi[m] = V[m * nc + nd.c[2]];
    Vj[m] = V[m * nc + nd.c[3]];
    Wi[m] = W[m * nc + nd.c[2]];
    Wj[m] = W[m * nc + nd.c[3]];
  }

  // first-order HLLC flux and u_* from the node states (Sec. 4.1.1), evaluated
  // where it is used: the first-order scheme, and the flux limiter where it may act
  FluxPack<N, D> H;
  auto first_order = [&]() {
    PrimState<double, N, D> a, b;
#pragma unroll
    for (int m = 0; m < M; ++m) {
      a.V[m] = Vi[m];
      b.V[m] = Vj[m];
    }
    double GH[M];
    const double uH = hllc<double, N, D, DIR>(f, a, b, GH);
#pragma unroll
    for (int m = 0; m < L::NC; ++m) H.Gc[m] = GH[m];
#pragma unroll
    for (int k = 0; k < N - 1; ++k) {
      H.gm[k] = GH[L::AL + k] - uH * Vi[L::AL + k];
      H.gp[k] = GH[L::AL + k] - uH * Vj[L::AL + k];
    }
  };

  FluxPack<N, D> G;
  if (pr.scheme == 1) {
    first_order();
    G = H;
  } else if (uniform_nodes<N, D>(W, nc, nd)) {
    // six bit-identical node states: in exact arithmetic every step below returns
    // the node's physical flux with zero alpha slots -- constants are reproduced
    // by the interpolation (App. C), the HLLC flux of equal states is their flux
    // (Sec. 4.1.1), the HCS weights sum to one, alpha u - u alpha = 0 (Eq. G_pm),
    // and the node state is the limiters' own candidate (Sec. 4.3.2)
    const double un = Vi[L::MOM + DIR], p = Vi[L::EN];
#pragma unroll
    for (int k = 0; k < N; ++k) G.Gc[k] = Wi[k] * un;
#pragma unroll
    for (int d = 0; d < D; ++d) G.Gc[L::MOM + d] = Wi[L::MOM + d] * un;
    G.Gc[L::MOM + DIR] = G.Gc[L::MOM + DIR] + p;
    G.Gc[L::EN] = (Wi[L::EN] + p) * un;
#pragma unroll
    for (int k = 0; k < N - 1; ++k) {
      G.gm[k] = 0.0;
      G.gp[k] = 0.0;
    }
  } else {
    R p6[6], u6[6];
#pragma unroll
    for (int j = 0; j < 6; ++j) {
      p6[j] = R(V[L::EN * nc + nd.c[j]]);
      u6[j] = R(V[(L::MOM + DIR) * nc + nd.c[j]]);
    }
    // characteristic projection with the face-averaged state (App. D)
    const R rhob = R(0.5) * (R(Rr[nd.c[2]]) + R(Rr[nd.c[3]]));
    const R cb = R(0.5) * (R(Cc[nd.c[2]]) + R(Cc[nd.c[3]]));
    const R inv_rc = R(1) / (rhob * cb);
    const R rc2b = rhob * cb * cb;
    const R eps = R(pr.weno_eps);
    R UL[M], UR[M];
    R w6[6];
#pragma unroll
    for (int j = 0; j < 6; ++j) w6[j] = u6[j] - inv_rc * p6[j];
    UL[0] = weno_sel<R>(lin, w6[0], w6[1], w6[2], w6[3], w6[4], eps);
    UR[0] = weno_sel<R>(lin, w6[5], w6[4], w6[3], w6[2], w6[1], eps);
#pragma unroll
    for (int j = 0; j < 6; ++j) w6[j] = u6[j] + inv_rc * p6[j];
    UL[M - 1] = weno_sel<R>(lin, w6[0], w6[1], w6[2], w6[3], w6[4], eps);
    UR[M - 1] = weno_sel<R>(lin, w6[5], w6[4], w6[3], w6[2], w6[1], eps);
    R arb[N];
#pragma unroll
    for (int k = 0; k < N; ++k) {
#pragma unroll
      for (int j = 0; j < 6; ++j) w6[j] = R(V[k * nc + nd.c[j]]);
      arb[k] = R(0.5) * (w6[2] + w6[3]);
      const R coef = arb[k] / rc2b;
#pragma unroll
      for (int j = 0; j < 6; ++j) w6[j] = w6[j] - coef * p6[j];
      UL[1 + k] = weno_sel<R>(lin, w6[0], w6[1], w6[2], w6[3], w6[4], eps);
      UR[1 + k] = weno_sel<R>(lin, w6[5], w6[4], w6[3], w6[2], w6[1], eps);
    }
    {
      int t_ = 0;
#pragma unroll
      for (int d = 0; d < D; ++d) {
        if (d == DIR) continue;
#pragma unroll
        for (int j = 0; j < 6; ++j) w6[j] = R(V[(L::MOM + d) * nc + nd.c[j]]);
        UL[N + 1 + t_] = weno_sel<R>(lin, w6[0], w6[1], w6[2], w6[3], w6[4], eps);
        UR[N + 1 + t_] = weno_sel<R>(lin, w6[5], w6[4], w6[3], w6[2], w6[1], eps);
        ++t_;
      }
    }
#pragma unroll
    for (int k = 0; k < N - 1; ++k) {
#pragma unroll
      for (int j = 0; j < 6; ++j) w6[j] = R(V[(L::AL + k) * nc + nd.c[j]]);
      UL[N + D + k] = weno_sel<R>(lin, w6[0], w6[1], w6[2], w6[3], w6[4], eps);
      UR[N + D + k] = weno_sel<R>(lin, w6[5], w6[4], w6[3], w6[2], w6[1], eps);
    }
    // back to primitive variables, V~ = R U~
    PrimState<R, N, D> sl, sr;
    {
      R h[N];
#pragma unroll
      for (int k = 0; k < N; ++k) h[k] = arb[k] / (R(2) * cb);
      const R rc_2 = rhob * cb / R(2);
#pragma unroll
      for (int side = 0; side < 2; ++side) {
        const R* U = side == 0 ? UL : UR;
        R* Vt = side == 0 ? sl.V : sr.V;
#pragma unroll
        for (int k = 0; k < N; ++k) Vt[k] = (-h[k]) * U[0] + U[1 + k] + h[k] * U[M - 1];
        Vt[L::MOM + DIR] = R(0.5) * U[0] + R(0.5) * U[M - 1];
        int t_ = 0;
#pragma unroll
        for (int d = 0; d < D; ++d) {
          if (d == DIR) continue;
          Vt[L::MOM + d] = U[N + 1 + t_];
          ++t_;
        }
        Vt[L::EN] = (-rc_2) * U[0] + rc_2 * U[M - 1];
#pragma unroll
        for (int k = 0; k < N - 1; ++k) Vt[L::AL + k] = U[N + D + k];
      }
    }
    // positivity-preserving interpolation limiter (Sec. 4.3.2)
    if (pr.limiters) {
      interp_limit<R, N, D>(sl.V, Vi, RC2[nd.c[2]], f, pr);
      interp_limit<R, N, D>(sr.V, Vj, RC2[nd.c[3]], f, pr);
    }
    // high-order midpoint flux G~ and velocity u~
    R Gt[M];
    const R ut = hllc<R, N, D, DIR>(f, sl, sr, Gt);
    // explicit HCS reconstruction (Eqs. reconstructed_G, reconstructed_vel)
    constexpr double psi = 256.0 / 175.0;
    constexpr double a1 = 75.0 * psi / 128.0 - 37.0 / 60.0;
    constexpr double a2 = 25.0 * psi / 256.0 - 2.0 / 15.0;
    constexpr double a3 = 3.0 * psi / 256.0 - 1.0 / 60.0;
    // shock sensor (Sec. 4.3.1) on rho and p
    R sig = R(0);
    if (pr.blend) {
      R r6[6];
#pragma unroll
      for (int j = 0; j < 6; ++j) r6[j] = R(Rr[nd.c[j]]);
      auto half = [](R a, R b, R c, R d, R e) -> R {
        const R num = fabs(R(16) * b - a - R(30) * c + R(16) * d - e);
        const R den = fabs(a + R(16) * b + R(30) * c + R(16) * d + e);
        return den == R(0) ? R(0) : num / den;
      };
      const R sr_ = R(0.5) * (half(r6[1], r6[2], r6[3], r6[4], r6[5]) + half(r6[0], r6[1], r6[2], r6[3], r6[4]));
      const R sp_ = R(0.5) * (half(p6[1], p6[2], p6[3], p6[4], p6[5]) + half(p6[0], p6[1], p6[2], p6[3], p6[4]));
      const R prod = sr_ * sp_;
      R pw = prod;
      for (int e = 1; e < pr.qexp; ++e) pw = pw * prod;
      sig = tanh_r(R(pr.Cs) * pw);
    }
    const R one_m = R(1) - sig;
    const R uhcs = R(psi) * ut - R(a1) * (u6[2] + u6[3]) + R(a2) * (u6[1] + u6[4]) - R(a3) * (u6[0] + u6[5]);
    const double uhat = (double)(sig * ut + one_m * uhcs);
    // node fluxes G of the flux-source form at the six nodes, slot by slot
#pragma unroll
    for (int m = 0; m < M; ++m) {
      R Gn[6];
#pragma unroll
      for (int j = 0; j < 6; ++j) {
        const double un = (double)u6[j];
        double v;
        if (m < L::MOM) {
          v = W[m * nc + nd.c[j]] * un;
        } else if (m < L::EN) {
          v = W[m * nc + nd.c[j]] * un + ((m - L::MOM) == DIR ? (double)p6[j] : 0.0);
        } else if (m == L::EN) {
          v = (W[m * nc + nd.c[j]] + (double)p6[j]) * un;
        } else {
          v = W[m * nc + nd.c[j]] * un;
        }
        Gn[j] = R(v);
      }
      const R ghcs = R(psi) * Gt[m] - R(a1) * (Gn[2] + Gn[3]) + R(a2) * (Gn[1] + Gn[4]) - R(a3) * (Gn[0] + Gn[5]);
      const double gh = (double)(sig * Gt[m] + one_m * ghcs);
      if (m < L::NC) {
        G.Gc[m] = gh;
      } else {
        // quasi-conservative alpha slots (Eq. G_pm, high-order form)
        G.gm[m - L::AL] = gh - uhat * Vi[m];
        G.gp[m - L::AL] = gh - uhat * Vj[m];
      }
    }

    if (pr.limiters) {
      double Fi[L::NC], Fj[L::NC];
      node_flux<N, D, DIR>(Wi, Vi, Fi);
      node_flux<N, D, DIR>(Wj, Vj, Fj);
      if (!flux_limit_noop<N, D>(Wi, Wj, Fi, Fj, lam, G, f, pr)) {
        first_order();
        flux_limit<N, D>(Wi, Wj, Fi, Fj, lam, G, H, f, pr);
      }
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

// Midpoint of this thread in a sweep of a 2D or 3D grid launched over
// lane_patch_grid blocks: a block takes 32 x 4 midpoints (along x, then y; z
// from the block index) and each warp an 8 x 4 patch of them. Uniform and
// non-uniform stencils come in bands a few midpoints wide along the material
// interfaces and wave fronts; a warp of 32 midpoints along one row crossing such
// a band holds a few non-uniform lanes, which run the whole midpoint body, and
// an 8 x 4 patch holds more of the band and fewer idle lanes. Past the end of
// the grid: the midpoint count (no midpoint).
template <int DIR>
__device__ __forceinline__ int64_t lane_patch_midpoint(const DevGrid& g) {
  static_assert(kFaceThreads == 128, "four warps per block");
  const int64_t f0 = g.n[0] + (DIR == 0), f1 = g.n[1] + (DIR == 1), f2 = g.n[2] + (DIR == 2);
  const int64_t nbx = (f0 + 31) / 32, nby = (f1 + 3) / 4, b = blockIdx.x;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int64_t i0 = (b % nbx) * 32 + w * 8 + (lane & 7);
  const int64_t i1 = ((b / nbx) % nby) * 4 + (lane >> 3);
  const int64_t i2 = b / (nbx * nby);
  if (i0 >= f0 || i1 >= f1 || i2 >= f2) return f0 * f1 * f2;
  return (i2 * f1 + i1) * f0 + i0;
}

template <typename R, int N, int D, int DIR>
__global__ void __launch_bounds__(kFaceThreads)
    k_face(const double* __restrict__ W, const double* __restrict__ V, const double* __restrict__ AUX,
           double* __restrict__ out, DevGrid g, DevFluid f, DevParams pr, const StepState* __restrict__ st,
           const uint8_t* __restrict__ gate) {
  const int64_t t = D >= 2 ? lane_patch_midpoint<DIR>(g) : (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  Nodes6 nd;
  if (!face_nodes<DIR>(g, t, nd)) return;
  const bool lin = gate != nullptr && gate[t] != 0;
  face_body<R, N, D, DIR>(t, nd, W, V, AUX, out, g, f, pr, st->lam[DIR], lin);
}

// ---------------------------------------------------------------- thermal relaxation (Sec. 4.2)

// Precision-form relaxation (FP64 throughout): the same root p* and T* as
// relax_cell, with the quadratic A_p p^2 + B_p p + C_p = 0 multiplied by rho^2
// so that its coefficients need no division:
//   rho^2 A_p = rho C_v,  rho^2 B_p = -(R_e R_m - p_inf,1 rho (C_v + rho_1' R_1)),
//   rho^2 C_p = -R_e p_inf,1 (R_m - rho_1' R_1),
// with C_v = sum alpha_k rho_k c_v,k, R_m = sum alpha_k rho_k (c_p,k - c_v,k),
// rho_1' = alpha_1 rho_1 (species `liq`) and R_e = rho (rho e~) =
// rho (E - sum alpha_k rho_k q_k) - |rho u|^2 / 2. With
// Y = rho_1' (p* + gamma_1 p_inf,1) c_v,1 + (C_v - rho_1' c_v,1)(p* + p_inf,1),
// Eq. T_relax_e gives T* = R_e (p* + p_inf,1) / (rho Y), and the relaxed volume
// fractions alpha_k = alpha_k rho_k R_k T* / (p* + p_inf,k) share one division
// z = R_e / (rho Y p*). Two divisions and one square root per cell. Returns rho
// and R_e for a primitive evaluation that follows.
template <int N, int D>
__device__ __forceinline__ void relax_fast(double* W, const DevFluid& f, double& rho_out, double& Re_out,
                                           double* pT = nullptr) {
  using L = Lay<N, D>;
  const int l = f.liq;
  double rho = 0.0, Cv = 0.0, Rm = 0.0, rq = 0.0, m2 = 0.0;
#pragma unroll
  for (int k = 0; k < N; ++k) {
    rho += W[k];
    Cv = fma(W[k], f.cv[k], Cv);
    Rm = fma(W[k], f.Rg[k], Rm);
  }
  if (f.has_q) {
#pragma unroll
    for (int k = 0; k < N; ++k) rq = fma(W[k], f.q[k], rq);
  }
#pragma unroll
  for (int d = 0; d < D; ++d) m2 = fma(W[L::MOM + d], W[L::MOM + d], m2);
  const double Re = fma(rho, W[L::EN] - rq, -0.5 * m2);
  const double pinf1 = f.pinf[l], Wl = W[l], WlR1 = Wl * f.Rg[l];
  const double A = rho * Cv;
  const double B = fma(pinf1 * rho, Cv + WlR1, -(Re * Rm));
  const double C = -(Re * pinf1 * (Rm - WlR1));
  const double sq = sqrt(fma(B, B, -4.0 * A * C));
  const double ps = (B > 0.0) ? (-2.0 * C) / (B + sq) : (sq - B) / (2.0 * A);
  const double ppl = ps + pinf1;
  const double Y = fma(Wl * fma(f.gamma[l], pinf1, ps), f.cv[l], fma(-Wl, f.cv[l], Cv) * ppl);
  const double z = Re / (rho * Y * ps);
#pragma unroll
  for (int k = 0; k < N - 1; ++k)  // alpha_k = rho_k' R_k T* / (p* + p_inf,k), one stiffened gas at most
    W[L::AL + k] = W[k] * f.Rg[k] * (k == l ? ps : ppl) * z;
  if (pT) {
    pT[0] = ps;
    pT[1] = z * ps * ppl;
  }
  rho_out = rho;
  Re_out = Re;
}

// Infinite-rate thermal relaxation of one cell: keeps alpha_k rho_k, rho u, E and
// replaces the stored alpha_k by rho Y_k / rho_k(p*, T*). p* is the positive root of
// A_p p^2 + B_p p + C_p = 0 (Eqs. Ap_Bp_Cp_1-3, p_relax) in the cancellation-free
// form, T* from Eq. T_relax_e. Species `liq` is the stiffened gas.
// FAST (precision form): relax_fast.
template <int N, int D, bool FAST = false>
__device__ __forceinline__ void relax_cell(double* W, const DevFluid& f, double* pT = nullptr) {
  if constexpr (FAST) {
    double rho, Re;
    relax_fast<N, D>(W, f, rho, Re, pT);
    return;
  }
  using L = Lay<N, D>;
  const int l = f.liq;
  double rho = 0.0;
#pragma unroll
  for (int k = 0; k < N; ++k) rho += W[k];
  double Y[N];
#pragma unroll
  for (int k = 0; k < N; ++k) Y[k] = W[k] / rho;
  const double re = rhoe_tilde<N, D>(W, f);
  double cvb = 0.0, cpb = 0.0;
#pragma unroll
  for (int k = 0; k < N; ++k) {
    cvb += Y[k] * f.cv[k];
    cpb += Y[k] * f.cp[k];
  }
  const double pinf1 = f.pinf[l], R1 = f.Rg[l], Yl = Y[l];
  const double Ap = cvb;
  const double Bp = -(re * (cpb - cvb) - pinf1 * cvb - pinf1 * Yl * R1);
  const double Cp = -(re * pinf1 * ((cpb - cvb) - Yl * R1));
  const double sq = sqrt(Bp * Bp - 4.0 * Ap * Cp);
  const double ps = (Bp > 0.0) ? (-2.0 * Cp) / (Bp + sq) : (sq - Bp) / (2.0 * Ap);
  const double den = Yl * (ps + f.gamma[l] * pinf1) * f.cv[l] / (ps + pinf1) + cvb - Yl * f.cv[l];
  const double Ts = (re / rho) / den;
#pragma unroll
  for (int k = 0; k < N - 1; ++k) {
    const double rhok = (ps + f.pinf[k]) / (f.Rg[k] * Ts);
    W[L::AL + k] = W[k] / rhok;
  }
  if (pT) {
    pT[0] = ps;
    pT[1] = Ts;
  }
}

// Admissibility of a conservative state: bit 0 negative partial density, bit 1 a
// volume fraction outside [0, 1], bit 2 rho c^2 <= 0, bit 3 rho e~ <= 0 (NaN counts).
template <int N, int D>
__device__ __forceinline__ int admissibility_bits(const double* W, const DevFluid& f) {
  using L = Lay<N, D>;
  int b = 0;
#pragma unroll
  for (int k = 0; k < N; ++k)
    if (!(W[k] >= 0.0)) b |= 1;
  double al[N];
  all_alpha_W<N, D>(W, al);
#pragma unroll
  for (int k = 0; k < N; ++k)
    if (!(al[k] >= 0.0 && al[k] <= 1.0)) b |= 2;
  const double re = rhoe_tilde<N, D>(W, f);
  double S, P;
  mix_SP<double, N>(f, &W[L::AL], S, P);
  const double p = (re - P) / S;
  if (!(rho_c2(S, P, p) > 0.0)) b |= 4;
  if (!(re > 0.0)) b |= 8;
  return b;
}

__device__ __forceinline__ void count_bits(StepState* st, int b) {
  if (b) {
    for (int i = 0; i < 4; ++i)
      if (b & (1 << i)) atomicAdd(&st->counts[i], 1ull);
  }
}

// ---------------------------------------------------------------- per-cell update

// The precision form's FP64 arithmetic writes its multiply-adds as explicit
// fma(): its translation units are built without FMA contraction, so that every
// FP32 expression rounds as written whichever kernel it is inlined into.
// Precision form: W_out = a W^n + b (W_src + dt RHS) of one interior cell c,
// with W_src + dt RHS accumulated directly and dt/dx_d folded into one
// coefficient per direction (one multiply-add per slot and direction). Ws: the
// cell's W_src, already loaded. The SSP-RK stages that combine with W^n have
// b = 1 - a, so their combination is formed as acc + a (W^n - acc): two
// operations as before, and exactly acc when W^n equals acc.
template <int N, int D>
__device__ __forceinline__ void fast_combine(int64_t c, const double* Wn, const double* Ws,
                                             const double* __restrict__ F0, const double* __restrict__ F1,
                                             const double* __restrict__ F2, const DevGrid& g, double dt, double a,
                                             double b, double* Wo) {
  using L = Lay<N, D>;
  constexpr int M = L::M;
  const int64_t nc = g.ncells;
  const int64_t i0 = c % g.n[0];
  const int64_t r = c / g.n[0];
  const int64_t i1 = r % g.n[1], i2 = r / g.n[1];
  double acc[M];
#pragma unroll
  for (int m = 0; m < M; ++m) acc[m] = Ws[m];
#pragma unroll
  for (int d = 0; d < D; ++d) {
    const double* F = d == 0 ? F0 : (d == 1 ? F1 : F2);
    const int64_t f0 = g.n[0] + (d == 0), f1 = g.n[1] + (d == 1), f2 = g.n[2] + (d == 2);
    const int64_t nf = f0 * f1 * f2;
    const int64_t fl = HRM_IDX(g, (i2 * f1 + i1) * f0 + i0, nf);
    const int64_t fr = HRM_IDX(g, fl + (d == 0 ? 1 : (d == 1 ? f0 : f0 * f1)), nf);
    const double cd = -dt * g.inv_dx[d];
    // G^-_{i+1/2} - G^+_{i-1/2}: the alpha slots of the right face use alpha_i
    // (planes AL..), those of the left face alpha_i as its right neighbour (planes M..)
#pragma unroll
    for (int m = 0; m < L::NC; ++m) acc[m] = fma(cd, F[m * nf + fr] - F[m * nf + fl], acc[m]);
#pragma unroll
    for (int k = 0; k < N - 1; ++k) {
      const int m = L::AL + k;
      acc[m] = fma(cd, F[m * nf + fr] - F[(M + k) * nf + fl], acc[m]);
    }
  }
  if (a == 0.0 && b == 1.0) {
#pragma unroll
    for (int m = 0; m < M; ++m) Wo[m] = acc[m];
  } else if (a == 0.0) {
#pragma unroll
    for (int m = 0; m < M; ++m) Wo[m] = b * acc[m];
  } else {
#pragma unroll
    for (int m = 0; m < M; ++m) Wo[m] = fma(a, Wn[m * nc + c] - acc[m], acc[m]);
  }
}

// Whether every flux difference G^-_{i+1/2} - G^+_{i-1/2} of cell c is exactly
// +0: the two faces' values bit-equal and finite in every slot and direction.
// Integer compares only.
template <int N, int D>
__device__ __forceinline__ bool faces_unchanged(int64_t c, const double* __restrict__ F0,
                                                const double* __restrict__ F1, const double* __restrict__ F2,
                                                const DevGrid& g) {
  using L = Lay<N, D>;
  constexpr int M = L::M;
  const int64_t i0 = c % g.n[0];
  const int64_t r = c / g.n[0];
  const int64_t i1 = r % g.n[1], i2 = r / g.n[1];
  auto bits = [](double x) { return (unsigned long long)__double_as_longlong(x); };
  auto same_finite = [&](double x, double y) {
    const unsigned long long bx = bits(x);
    return (bx == bits(y)) & (((bx >> 52) & 0x7ffull) != 0x7ffull);
  };
  bool same = true;
#pragma unroll
  for (int d = 0; d < D; ++d) {
    const double* F = d == 0 ? F0 : (d == 1 ? F1 : F2);
    const int64_t f0 = g.n[0] + (d == 0), f1 = g.n[1] + (d == 1), f2 = g.n[2] + (d == 2);
    const int64_t nf = f0 * f1 * f2;
    const int64_t fl = HRM_IDX(g, (i2 * f1 + i1) * f0 + i0, nf);
    const int64_t fr = HRM_IDX(g, fl + (d == 0 ? 1 : (d == 1 ? f0 : f0 * f1)), nf);
#pragma unroll
    for (int m = 0; m < L::NC; ++m) same = same & same_finite(F[m * nf + fr], F[m * nf + fl]);
#pragma unroll
    for (int k = 0; k < N - 1; ++k) same = same & same_finite(F[(L::AL + k) * nf + fr], F[(M + k) * nf + fl]);
  }
  return same;
}

// Precision form: whether a stage returns cell c exactly as it is, so that its
// arithmetic can be left out. Every flux difference G^-_{i+1/2} - G^+_{i-1/2}
// is exactly zero when the two faces' values are bit-equal and finite; a stage
// that combines with W^n (with_wn) also needs W_src bit-equal to W^n. Then
// fast_combine returns W_src exactly (its weights sum to one), except that a
// component -0 would come back +0, so those are left to the arithmetic; and
// relax_fast, which recomputes the volume fractions from the conserved
// variables alone, returns the cell unchanged if it came out of relax_fast
// before -- the caller's condition. Only integer compares: no FP64 work.
template <int N, int D>
__device__ __forceinline__ bool stage_keeps_cell(int64_t c, const double* Wn, const double* Ws,
                                                 const double* __restrict__ F0, const double* __restrict__ F1,
                                                 const double* __restrict__ F2, const DevGrid& g, bool with_wn) {
  constexpr int M = Lay<N, D>::M;
  const int64_t nc = g.ncells;
  bool same = faces_unchanged<N, D>(c, F0, F1, F2, g);
  if (with_wn) {
#pragma unroll
    for (int m = 0; m < M; ++m) {
      const unsigned long long bs = (unsigned long long)__double_as_longlong(Ws[m]);
      same = same & (bs == (unsigned long long)__double_as_longlong(Wn[m * nc + c])) &
             (bs != 0x8000000000000000ull);
    }
  }
  return same;
}

// RHS_i = -sum_d (G^{d,-}_{i+1/2} - G^{d,+}_{i-1/2}) / dx_d (Eq. semi_W_G_pm_eqn),
// then W_out = a W^n + b (W_src + dt RHS) (SSP-RK stage in Shu-Osher form),
// optionally followed by the thermal relaxation and the admissibility count.
// MODE 1 writes RHS instead of the combination. In-place (W_out == W_src or W^n)
// is allowed: each thread reads its own cell before writing it.
// FAST (precision form): reciprocal of dx and of rho instead of divisions.
// One interior cell c < nint (Dirichlet slices keep their state).
template <int N, int D, int MODE, bool FAST = false>
__device__ __forceinline__ void update_body(int64_t c, const double* Wn, const double* Wsrc, double* Wout,
                                            const double* __restrict__ F0, const double* __restrict__ F1,
                                            const double* __restrict__ F2, const DevGrid& g, const DevFluid& f,
                                            StepState* st, double dt, double a, double b, int relax, int count,
                                            uint8_t* __restrict__ same = nullptr) {
  using L = Lay<N, D>;
  constexpr int M = L::M;
  const int64_t nc = g.ncells;
  const int64_t i0 = c % g.n[0];
  const int64_t r = c / g.n[0];
  const int64_t i1 = r % g.n[1], i2 = r / g.n[1];
  double Ws[M];
#pragma unroll
  for (int m = 0; m < M; ++m) Ws[m] = Wsrc[m * nc + c];
  if constexpr (FAST && MODE == 0) {
    const bool with_wn = a != 0.0;
    if ((!relax || st->wn_relaxed) && stage_keeps_cell<N, D>(c, Wn, Ws, F0, F1, F2, g, with_wn)) {
      // W_out = W_src exactly; already there in place, or (with_wn) in W^n
      if (Wout != Wsrc && !(with_wn && Wout == Wn)) {
#pragma unroll
        for (int m = 0; m < M; ++m) Wout[m * nc + c] = Ws[m];
      }
      if (count) count_bits(st, admissibility_bits<N, D>(Ws, f));
      return;
    }
    double Wo[M];
    fast_combine<N, D>(c, Wn, Ws, F0, F1, F2, g, dt, a, b, Wo);
    if (relax) relax_cell<N, D, FAST>(Wo, f);
    if (count) count_bits(st, admissibility_bits<N, D>(Wo, f));
#pragma unroll
    for (int m = 0; m < M; ++m) Wout[m * nc + c] = Wo[m];
    return;
  }
  double rhs[M];
#pragma unroll
  for (int m = 0; m < M; ++m) rhs[m] = 0.0;
  // Faces all bit-equal: every difference is +0, its quotient by dx too, and
  // the sums below would leave rhs at +0 -- the divisions are left out.
  const bool flat = faces_unchanged<N, D>(c, F0, F1, F2, g);
#pragma unroll
  for (int d = 0; d < D; ++d) {
    if (flat) break;
    const double* F = d == 0 ? F0 : (d == 1 ? F1 : F2);
    const int64_t f0 = g.n[0] + (d == 0), f1 = g.n[1] + (d == 1), f2 = g.n[2] + (d == 2);
    const int64_t nf = f0 * f1 * f2;
    const int64_t fl = HRM_IDX(g, (i2 * f1 + i1) * f0 + i0, nf);
    const int64_t fr = HRM_IDX(g, fl + (d == 0 ? 1 : (d == 1 ? f0 : f0 * f1)), nf);
    const double dx = g.dx[d], idx = g.inv_dx[d];
    // where dx is a power of two (a significand field of zero), 1/dx is exact and
    // df / dx and df * (1/dx) are the same correctly rounded number: the product
    // then stands for the quotient at no change of any result
    const bool scale = FAST || (__double_as_longlong(dx) & 0xFFFFFFFFFFFFFll) == 0;
    // G^-_{i+1/2} - G^+_{i-1/2}: the alpha slots of the right face use alpha_i
    // (planes AL..), those of the left face alpha_i as its right neighbour (planes M..)
#pragma unroll
    for (int m = 0; m < L::NC; ++m) {
      const double df = F[m * nf + fr] - F[m * nf + fl];
      rhs[m] = rhs[m] - (scale ? df * idx : df / dx);
    }
#pragma unroll
    for (int k = 0; k < N - 1; ++k) {
      const int m = L::AL + k;
      const double df = F[m * nf + fr] - F[(M + k) * nf + fl];
      rhs[m] = rhs[m] - (scale ? df * idx : df / dx);
    }
  }
  if (MODE == 1) {
#pragma unroll
    for (int m = 0; m < M; ++m) Wout[m * nc + c] = rhs[m];
    return;
  }
  double Wo[M];
  if (a == 0.0) {
#pragma unroll
    for (int m = 0; m < M; ++m) Wo[m] = b * (Ws[m] + dt * rhs[m]);
  } else {
#pragma unroll
    for (int m = 0; m < M; ++m) Wo[m] = a * Wn[m * nc + c] + b * (Ws[m] + dt * rhs[m]);
  }
  // relax_cell recomputes the volume fractions from the conserved variables
  // alone: where those are bit-equal to W^n's and W^n came out of relax_cell
  // (the host's flag), it would return W^n's volume fractions, taken directly.
  bool keep = false;
  if (relax && flat && st->wn_relaxed) {
    keep = true;
#pragma unroll
    for (int m = 0; m < L::NC; ++m)
      keep = keep & (__double_as_longlong(Wo[m]) == __double_as_longlong(Wn[m * nc + c]));
  }
  if (keep) {
#pragma unroll
    for (int k = 0; k < N - 1; ++k) Wo[L::AL + k] = Wn[(L::AL + k) * nc + c];
  } else if (relax) {
    relax_cell<N, D, FAST>(Wo, f);
  }
  if (count) count_bits(st, admissibility_bits<N, D>(Wo, f));
  if (same) {
    // the next stage's primitive pass keeps this cell's V and AUX where W_out is W_src
    bool eq = true;
#pragma unroll
    for (int m = 0; m < M; ++m) eq = eq & (__double_as_longlong(Wo[m]) == __double_as_longlong(Ws[m]));
    same[c] = eq ? 1 : 0;
  }
#pragma unroll
  for (int m = 0; m < M; ++m) Wout[m * nc + c] = Wo[m];
}

template <int N, int D, int MODE, bool FAST = false>
__global__ void __launch_bounds__(kCellThreads)
    k_update(const double* Wn, const double* Wsrc, double* Wout, const double* __restrict__ F0,
             const double* __restrict__ F1, const double* __restrict__ F2, DevGrid g, DevFluid f,
             StepState* st, double a, double b, int relax, int count, uint8_t* __restrict__ same = nullptr) {
  const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= g.nint) return;
  update_body<N, D, MODE, FAST>(c, Wn, Wsrc, Wout, F0, F1, F2, g, f, st, MODE == 1 ? 0.0 : st->dt, a, b, relax,
                                count, same);
}

}  // namespace hrm
