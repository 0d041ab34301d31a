// TEST INFRASTRUCTURE -- serial FP64 CPU oracle of the positivity-preserving
// fractional algorithm of Wong, Angel & Kiris (arXiv 2208.04488).
//
// This file is the slow, obviously-correct reference that the CUDA path is
// checked against. Only tests/, __graft_entry__.smoke() and bench.py's CPU
// baseline may load it. It shares no code, header or constant table with the
// CUDA library, and nothing in the product path may call it.
//
// Every step follows the paper in the paper's order, one face at a time, in a
// plain scalar loop, built with -O2 -ffp-contract=off:
//   Sec. 2           stiffened-gas EOS and mixture rules (Eq. species_stiffened_EOS)
//   Sec. 4.1.1       HLLC Riemann solver for the five-equation model (Eq. HLLC_states,
//                    Eq. s_star_definition), quasi-conservative fluxes (Eq. G_pm)
//   Sec. 4.1.2       CFL time step and directional split sigma/tau/lambda
//   Sec. 4.2         algebraic thermal relaxation (Eqs. Ap_Bp_Cp_1-3, p_relax, T_relax_e)
//   Sec. 4.3.1       explicit HCS flux difference (Eq. HCS6, reconstructed_G, reconstructed_vel),
//                    shock-sensor blending (Eq. flux_blending, velocity_blending)
//   Sec. 4.3.2       interpolation limiter (Alg. interp_limit_densities, interp_limit_vol_frac,
//                    hard switch) and flux limiter (Alg. flux_limit_densities_vol_frac,
//                    flux_limit_energy, hard switch)
//   Sec. 4.4         SSP-RK time stepping with relaxation after every stage
//   App. C           incremental-stencil WENO interpolation
//   App. D           characteristic decomposition of the primitive variables
// Where the paper is silent or ambiguous the reading taken is stated inline
// (the same list is kept in the design notes). Where a step's exact-arithmetic
// result is known in closed form it is taken directly, at the step itself: a
// constant stencil interpolates to its value (App. C), and a midpoint of six
// bit-identical node states gets the node's physical flux (face_flux).
//
// Built three times: normally (real == double); with -DOR_COUNT, where `real`
// is a counting wrapper so that a run reports the algorithmic number of
// floating-point operations the method performs; and with -DOR_OMP -fopenmp,
// where the independent grid lines of each sweep and the cells of the
// relaxation are shared among host threads (identical results).

#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>
#ifdef OR_OMP
#include <omp.h>
#endif

// tanh of the shock sensor (Sec. 4.3.1), evaluated explicitly so that its
// rounding does not depend on a math library: tanh|x| = m / (m + 2) with
// m = expm1(2|x|); expm1 by its Taylor series for arguments below 0.5, else
// exp by Cody-Waite argument reduction (exp(y) = 2^k exp(r), y = k ln2 + r,
// |r| <= ln2 / 2, ln2 split into a 32-bit head and a tail) and its Taylor
// series; tanh|x| = 1 above 22, where 1 - tanh is below half an ulp.
static double tanh_explicit(double x) {
  static const double kLn2 = 0.6931471805599453;
  static const double kLn2Hi = 0.6931471803691238;     // 32 significant bits of ln 2
  static const double kLn2Lo = 1.9082149292705877e-10;  // ln 2 - kLn2Hi
  static const double kInv[19] = {0.0,       1.0,        1.0 / 2.0,  1.0 / 3.0,  1.0 / 4.0,
                                  1.0 / 5.0, 1.0 / 6.0,  1.0 / 7.0,  1.0 / 8.0,  1.0 / 9.0,
                                  1.0 / 10.0, 1.0 / 11.0, 1.0 / 12.0, 1.0 / 13.0, 1.0 / 14.0,
                                  1.0 / 15.0, 1.0 / 16.0, 1.0 / 17.0, 1.0 / 18.0};
  const double ax = std::fabs(x);
  double t;
  if (ax > 22.0) {
    t = 1.0;
  } else {
    const double y = 2.0 * ax;
    double m;
    if (y < 0.5) {
      double s = 1.0;
      for (int k = 18; k >= 2; --k) s = 1.0 + (y * kInv[k]) * s;  // expm1(y) / y
      m = y * s;
    } else {
      const double k = std::nearbyint(y / kLn2);
      const double r = (y - k * kLn2Hi) - k * kLn2Lo;
      double s = 1.0;
      for (int j = 17; j >= 1; --j) s = 1.0 + (r * kInv[j]) * s;  // exp(r)
      m = std::ldexp(s, (int)k) - 1.0;
    }
    t = m / (m + 2.0);
  }
  return x < 0.0 ? -t : t;
}

#ifdef OR_COUNT
struct OrCounts { unsigned long long add, mul, div, sqrt, tanh; };
static OrCounts g_cnt = {0, 0, 0, 0, 0};
struct real {
  double v;
  real() : v(0.0) {}
  real(double x) : v(x) {}
};
static inline real operator+(real a, real b) { g_cnt.add++; return real(a.v + b.v); }
static inline real operator-(real a, real b) { g_cnt.add++; return real(a.v - b.v); }
static inline real operator-(real a) { return real(-a.v); }
static inline real operator*(real a, real b) { g_cnt.mul++; return real(a.v * b.v); }
static inline real operator/(real a, real b) { g_cnt.div++; return real(a.v / b.v); }
static inline bool operator<(real a, real b) { return a.v < b.v; }
static inline bool operator>(real a, real b) { return a.v > b.v; }
static inline bool operator<=(real a, real b) { return a.v <= b.v; }
static inline bool operator>=(real a, real b) { return a.v >= b.v; }
static inline bool operator==(real a, real b) { return a.v == b.v; }
static inline bool operator!=(real a, real b) { return a.v != b.v; }
static inline real rsqrt_(real a) { g_cnt.sqrt++; return real(std::sqrt(a.v)); }
static inline real rtanh_(real a) { g_cnt.tanh++; return real(tanh_explicit(a.v)); }
static inline real rabs_(real a) { return real(std::fabs(a.v)); }
static inline double val(real a) { return a.v; }
#else
typedef double real;
static inline real rsqrt_(real a) { return std::sqrt(a); }
static inline real rtanh_(real a) { return tanh_explicit(a); }
static inline real rabs_(real a) { return std::fabs(a); }
static inline double val(real a) { return a; }
#endif

static inline real rmin(real a, real b) { return (b < a) ? b : a; }
static inline real rmax(real a, real b) { return (a < b) ? b : a; }
static inline int rsign(real a) { return (a > real(0.0)) ? 1 : ((a < real(0.0)) ? -1 : 0); }

#define OR_MAXN 4
#define OR_MAXD 3
#define OR_MAXM (2 * OR_MAXN + OR_MAXD)

extern "C" {

// ---- plain-data descriptions passed in from Python (ctypes) -------------

// Species table (Table fluid_properties): gamma_k, p_inf_k, c_v,k, q_k.
// `liq` is the index of the single stiffened gas (p_inf > 0), or any index
// when all species are ideal gases.
struct or_fluid {
  int32_t N, D, liq, pad;
  double gamma[OR_MAXN], pinf[OR_MAXN], cv[OR_MAXN], q[OR_MAXN];
};

struct or_params {
  int32_t limiters;    // 1: interpolation and flux limiters on (Sec. 4.3.2)
  int32_t blend;       // 1: shock-sensor blending (Eqs. flux_blending, velocity_blending)
  int32_t relax_mode;  // 0 off, 1 after every RK stage (Sec. 4.4), 2 after the full step
  int32_t scheme;      // 0 PP-WCNS-IS, 1 first-order HLLC only (Sec. 4.1.1)
  int32_t integrator;  // 0 SSP-RK3, 1 forward Euler, 2 SSP-RK2 (Sec. 5.1)
  int32_t cfl_sound;   // sound speed of the CFL maxima: 0 five-equation c, 1 four-equation HRM c (Eq. 4_eqn_sos)
  int32_t pad1, pad2;
  double eps_ar, eps_a, eps_rhoe;   // limiter thresholds (Sec. 4.3.2)
  double hs_ar, hs_a, hs_rc2, hs_rhoe;  // hard-switch thresholds (Sec. 4.3.2)
  double weno_eps;                  // App. C
  double Cs, q_sensor;              // shock sensor constants (Sec. 4.3.1)
};

// Uniform Cartesian grid. n[d] cells in direction d (x fastest), spacing dx[d].
// bc[2d] / bc[2d+1]: low / high side, 0 = transmissive (zeroth-order
// extrapolation into the ghost cells), 1 = periodic, 2 = Dirichlet: every ghost
// cell of that side holds the prescribed state bnd[2d + side], the conservative
// vector W (M planes) of the boundary slice, one entry per cell of the side
// (the other directions' indices, lowest direction fastest).
struct or_grid {
  int32_t D, pad;
  int64_t n[3];
  double dx[3];
  int32_t bc[6];
  const double* bnd[6];
};

}  // extern "C"

// ---- derived constants of a species table (not part of the per-cell work) ----
struct FluidK {
  int N, D, M, liq;
  double inv_gm1[OR_MAXN];    // 1/(gamma_k-1)
  double gpinf_gm1[OR_MAXN];  // gamma_k p_inf_k/(gamma_k-1)
  double cv[OR_MAXN], cp[OR_MAXN], q[OR_MAXN], pinf[OR_MAXN];
  double gamma[OR_MAXN], Rgas[OR_MAXN];  // gamma_k and c_p,k - c_v,k = (gamma_k-1) c_v,k
};

static FluidK make_fluid(const or_fluid* f) {
  FluidK k;
  k.N = f->N;
  k.D = f->D;
  k.M = 2 * f->N + f->D;
  k.liq = f->liq;
  for (int s = 0; s < f->N; ++s) {
    k.inv_gm1[s] = 1.0 / (f->gamma[s] - 1.0);
    k.gpinf_gm1[s] = f->gamma[s] * f->pinf[s] / (f->gamma[s] - 1.0);
    k.cv[s] = f->cv[s];
    k.cp[s] = f->gamma[s] * f->cv[s];  // gamma_k = c_p,k / c_v,k (Sec. 2)
    k.q[s] = f->q[s];
    k.pinf[s] = f->pinf[s];
    k.gamma[s] = f->gamma[s];
    k.Rgas[s] = k.cp[s] - k.cv[s];
  }
  return k;
}

// Slots of W = (alpha_k rho_k [N], rho u_d [D], E, alpha_k [N-1]) (Sec. 2) and of
// V = (alpha_k rho_k [N], u_d [D], p, alpha_k [N-1]) (App. D).
static inline int sMOM(const FluidK& f, int d) { return f.N + d; }
static inline int sE(const FluidK& f) { return f.N + f.D; }
static inline int sAL(const FluidK& f, int k) { return f.N + f.D + 1 + k; }

// Volume fractions of all N species; alpha_N = 1 - sum of the others (Sec. 2).
static void all_alpha(const FluidK& f, const real* X, real* al) {
  real s = 0.0;
  for (int k = 0; k < f.N - 1; ++k) {
    al[k] = X[sAL(f, k)];
    s = s + al[k];
  }
  al[f.N - 1] = real(1.0) - s;
}

// Mixture rules (Sec. 2): S = 1/(gbar-1) = sum alpha_k/(gamma_k-1),
// P = gbar pbar_inf/(gbar-1) = sum alpha_k gamma_k p_inf_k/(gamma_k-1).
static void mixture(const FluidK& f, const real* al, real& S, real& P) {
  S = 0.0;
  P = 0.0;
  for (int k = 0; k < f.N; ++k) {
    S = S + al[k] * f.inv_gm1[k];
    P = P + al[k] * f.gpinf_gm1[k];
  }
}

// rho c^2 = gbar (p + pbar_inf) (Sec. 2), with gbar = 1 + 1/S and gbar pbar_inf = P/S.
static real rho_c2_of(real S, real P, real p) {
  real gbar = real(1.0) + real(1.0) / S;
  return gbar * p + P / S;
}

// rho(e - qbar) of a conservative vector (Sec. 2, expression below Eq. mathcal_G_set).
static real rhoe_tilde(const FluidK& f, const real* W) {
  real rho = 0.0, kin = 0.0, rq = 0.0;
  for (int k = 0; k < f.N; ++k) rho = rho + W[k];
  for (int d = 0; d < f.D; ++d) kin = kin + W[sMOM(f, d)] * W[sMOM(f, d)];
  for (int k = 0; k < f.N; ++k) rq = rq + W[k] * f.q[k];
  return W[sE(f)] - real(0.5) * kin / rho - rq;
}

// Primitive state of one cell from W (Sec. 2): V, rho, c, rho c^2.
struct Cell {
  real W[OR_MAXM], V[OR_MAXM];
  real rho, c, rc2;
};

static void cell_from_W(const FluidK& f, const real* W, Cell& C) {
  for (int m = 0; m < f.M; ++m) C.W[m] = W[m];
  real rho = 0.0;
  for (int k = 0; k < f.N; ++k) rho = rho + W[k];
  real al[OR_MAXN];
  all_alpha(f, W, al);
  real S, P;
  mixture(f, al, S, P);
  real re = rhoe_tilde(f, W);
  // mixture EOS: p/(gbar-1) + gbar pbar_inf/(gbar-1) = rho (e - qbar)
  real p = (re - P) / S;
  for (int k = 0; k < f.N; ++k) C.V[k] = W[k];
  for (int d = 0; d < f.D; ++d) C.V[sMOM(f, d)] = W[sMOM(f, d)] / rho;
  C.V[sE(f)] = p;
  for (int k = 0; k < f.N - 1; ++k) C.V[sAL(f, k)] = W[sAL(f, k)];
  C.rho = rho;
  C.rc2 = rho_c2_of(S, P, p);
  C.c = rsqrt_(C.rc2 / rho);
}

// Conservative vector, total energy and sound speed of a primitive state.
struct PState {
  real V[OR_MAXM], W[OR_MAXM];
  real rho, c, rc2, E;
};

static void pstate_from_V(const FluidK& f, const real* V, PState& s) {
  for (int m = 0; m < f.M; ++m) s.V[m] = V[m];
  real rho = 0.0;
  for (int k = 0; k < f.N; ++k) rho = rho + V[k];
  real al[OR_MAXN];
  all_alpha(f, V, al);
  real S, P;
  mixture(f, al, S, P);
  real p = V[sE(f)];
  real kin = 0.0, rq = 0.0;
  for (int d = 0; d < f.D; ++d) kin = kin + V[sMOM(f, d)] * V[sMOM(f, d)];
  for (int k = 0; k < f.N; ++k) rq = rq + V[k] * f.q[k];
  real E = (S * p + P) + real(0.5) * rho * kin + rq;
  for (int k = 0; k < f.N; ++k) s.W[k] = V[k];
  for (int d = 0; d < f.D; ++d) s.W[sMOM(f, d)] = rho * V[sMOM(f, d)];
  s.W[sE(f)] = E;
  for (int k = 0; k < f.N - 1; ++k) s.W[sAL(f, k)] = V[sAL(f, k)];
  s.rho = rho;
  s.E = E;
  s.rc2 = rho_c2_of(S, P, p);
  s.c = rsqrt_(s.rc2 / rho);
}

// Conservative flux F^d of Eq. F_x_F_y_def (zero in the alpha slots).
static void flux_F(const FluidK& f, int dir, const real* V, const real* W, real* F) {
  real un = V[sMOM(f, dir)];
  real p = V[sE(f)];
  for (int k = 0; k < f.N; ++k) F[k] = W[k] * un;
  for (int d = 0; d < f.D; ++d) F[sMOM(f, d)] = W[sMOM(f, d)] * un;
  F[sMOM(f, dir)] = F[sMOM(f, dir)] + p;
  F[sE(f)] = (W[sE(f)] + p) * un;
  for (int k = 0; k < f.N - 1; ++k) F[sAL(f, k)] = 0.0;
}

// Flux-source-form flux G^d (Eq. W_G_eqn): F^d plus alpha_k u_d in the alpha slots.
static void flux_G(const FluidK& f, int dir, const real* V, const real* W, real* G) {
  flux_F(f, dir, V, W, G);
  for (int k = 0; k < f.N - 1; ++k) G[sAL(f, k)] = V[sAL(f, k)] * V[sMOM(f, dir)];
}

// ---------------------------------------------------------------------------
// HLLC (Sec. 4.1.1). Returns G = F^HLLC + (0, ..., f_alpha) and s_*.
// Reading: sign(0) = 0, so at s_* = 0 the flux is the mean of the two star
// fluxes exactly as the (1 +- sign)/2 form is written; only the sides with a
// non-zero factor are evaluated.
// ---------------------------------------------------------------------------
static void hllc(const FluidK& f, int dir, const real* VL, const real* VR, real* G,
                 real* sstar_out) {
  PState L, R;
  pstate_from_V(f, VL, L);
  pstate_from_V(f, VR, R);
  real uL = VL[sMOM(f, dir)], uR = VR[sMOM(f, dir)];
  real pL = VL[sE(f)], pR = VR[sE(f)];
  // Einfeldt / Batten wave speeds with arithmetic averages (Sec. 4.1.1).
  real ubar = real(0.5) * (uL + uR);
  real cbar = real(0.5) * (L.c + R.c);
  real sL = rmin(ubar - cbar, uL - L.c);
  real sR = rmax(ubar + cbar, uR + R.c);
  // Eq. s_star_definition
  real ss = (pR - pL + L.rho * uL * (sL - uL) - R.rho * uR * (sR - uR)) /
            (L.rho * (sL - uL) - R.rho * (sR - uR));
  int sg = rsign(ss);
  real sminus = rmin(real(0.0), sL), splus = rmax(real(0.0), sR);
  real FL[OR_MAXM], FR[OR_MAXM];
  real partL[OR_MAXM], partR[OR_MAXM];
  for (int side = 0; side < 2; ++side) {
    if ((side == 0 && sg < 0) || (side == 1 && sg > 0)) continue;
    const PState& K = (side == 0) ? L : R;
    real uK = (side == 0) ? uL : uR;
    real pK = (side == 0) ? pL : pR;
    real sK = (side == 0) ? sL : sR;
    real sfac = (side == 0) ? sminus : splus;
    real* Fk = (side == 0) ? FL : FR;
    real* part = (side == 0) ? partL : partR;
    flux_F(f, dir, K.V, K.W, Fk);
    // star state W_{*,K}
    real chi = (sK - uK) / (sK - ss);
    real Ws[OR_MAXM];
    for (int k = 0; k < f.N; ++k) Ws[k] = chi * K.W[k];
    for (int d = 0; d < f.D; ++d) Ws[sMOM(f, d)] = chi * K.rho * K.V[sMOM(f, d)];
    Ws[sMOM(f, dir)] = chi * K.rho * ss;
    Ws[sE(f)] = chi * (K.E + (ss - uK) * (K.rho * ss + pK / (sK - uK)));
    for (int k = 0; k < f.N - 1; ++k) Ws[sAL(f, k)] = K.W[sAL(f, k)];
    for (int m = 0; m < f.M; ++m) part[m] = Fk[m] + sfac * (Ws[m] - K.W[m]);
  }
  for (int m = 0; m < f.M; ++m) {
    if (sg > 0)
      G[m] = partL[m];
    else if (sg < 0)
      G[m] = partR[m];
    else
      G[m] = real(0.5) * partL[m] + real(0.5) * partR[m];
  }
  // alpha fluxes: upwind alpha times s_* (Sec. 4.1.1)
  for (int k = 0; k < f.N - 1; ++k) {
    real aL = VL[sAL(f, k)], aR = VR[sAL(f, k)];
    real fa;
    if (sg > 0)
      fa = aL * ss;
    else if (sg < 0)
      fa = aR * ss;
    else
      fa = real(0.5) * (aL * ss) + real(0.5) * (aR * ss);
    G[sAL(f, k)] = fa;
  }
  *sstar_out = ss;
}

// ---------------------------------------------------------------------------
// Incremental-stencil WENO interpolation (App. C), left-biased midpoint value
// at x_{i+1/2} from u[0..4] = u_{i-2}, u_{i-1}, u_i, u_{i+1}, u_{i+2}.
// ---------------------------------------------------------------------------
// Whether the five stencil values are bit-identical.
static bool constant_stencil(const real* u) {
  uint64_t b[5];
  for (int j = 0; j < 5; ++j) {
    const double x = val(u[j]);
    std::memcpy(&b[j], &x, sizeof x);
  }
  return b[0] == b[2] && b[1] == b[2] && b[3] == b[2] && b[4] == b[2];
}

static real weno_is_left(const real* u, double eps, real* omega_out) {
  // A constant stencil: every sub-stencil interpolant reproduces the constant
  // and the weights sum to one (App. C), so the interpolated value is that
  // constant, returned as it is (the weighted sum below reaches it only to
  // rounding). The weights themselves (omega_out) are formed in full.
  if (!omega_out && constant_stencil(u)) return u[2];
  const real um2 = u[0], um1 = u[1], u0 = u[2], up1 = u[3], up2 = u[4];
  // sub-stencil interpolants S0..S3
  real s0 = real(0.5) * (u0 + up1);
  real s1 = real(0.5) * (real(3.0) * u0 - um1);
  real s2 = real(1.0 / 8.0) * (real(3.0) * u0 + real(6.0) * up1 - up2);
  real s3 = real(1.0 / 8.0) * (real(3.0) * um2 - real(10.0) * um1 + real(15.0) * u0);
  // linear weights d_k
  const double d0 = 15.0 / 32.0, d1 = 5.0 / 32.0, d2 = 5.0 / 16.0, d3 = 1.0 / 16.0;
  // smoothness indicators
  real b0 = (u0 - up1) * (u0 - up1);
  real b1 = (um1 - u0) * (um1 - u0);
  real t01a = um1 - real(2.0) * u0 + up1, t01b = um1 - up1;
  real b01 = real(13.0 / 12.0) * t01a * t01a + real(0.25) * t01b * t01b;
  real t2a = u0 - real(2.0) * up1 + up2, t2b = real(3.0) * u0 - real(4.0) * up1 + up2;
  real b2 = real(13.0 / 12.0) * t2a * t2a + real(0.25) * t2b * t2b;
  real t3a = um2 - real(2.0) * um1 + u0, t3b = um2 - real(4.0) * um1 + real(3.0) * u0;
  real b3 = real(13.0 / 12.0) * t3a * t3a + real(0.25) * t3b * t3b;
  real t5a = up2 - real(4.0) * up1 + real(6.0) * u0 - real(4.0) * um1 + um2;
  real t5b = up2 - real(2.0) * up1 + real(2.0) * um1 - um2;
  real tau5 = real(13.0 / 12.0) * t5a * t5a + real(0.25) * t5b * t5b;
  // nonlinear weights omega_k = eta_k / sum_s eta_s, with every eta_k multiplied
  // by the same positive factor (beta_0 + eps)(beta_1 + eps)(beta_01 + eps)
  // (beta_2 + eps)(beta_3 + eps), which leaves omega_k as it is and clears the
  // denominators of eta_k: eta_0 = d_0 (1 + tau_5^2 / ((beta_0 + eps)(beta_01 + eps)))
  // becomes d_0 ((beta_0 + eps)(beta_01 + eps) + tau_5^2)(beta_1 + eps)(beta_2 + eps)(beta_3 + eps), etc.
  const real a = b0 + real(eps), b = b1 + real(eps), c = b01 + real(eps);
  const real g2 = b2 + real(eps), g3 = b3 + real(eps);
  const real t2 = tau5 * tau5;
  const real g23 = g2 * g3;
  const real abc = (a * b) * c;
  real e0 = real(d0) * ((a * c + t2) * (b * g23));
  real e1 = real(d1) * ((b * c + t2) * (a * g23));
  real e2 = real(d2) * ((g2 + tau5) * (abc * g3));
  real e3 = real(d3) * ((g3 + tau5) * (abc * g2));
  real esum = e0 + e1 + e2 + e3;
  if (omega_out) {  // omega_k = e_k / sum of e
    omega_out[0] = e0 / esum;
    omega_out[1] = e1 / esum;
    omega_out[2] = e2 / esum;
    omega_out[3] = e3 / esum;
  }
  // sum_k omega_k S_k, with the common normalisation applied once
  return (e0 * s0 + e1 * s1 + e2 * s2 + e3 * s3) / esum;
}

// The same interpolation with every nonlinear weight replaced by its linear
// (optimal) weight d_k: the value a smoothness gate selects where it judges
// the stencil smooth (the nonlinear weights then differ little from d_k).
static real weno_lin_left(const real* u) {
  // a constant stencil: the linear weights sum to one as well (App. C)
  if (constant_stencil(u)) return u[2];
  const real um2 = u[0], um1 = u[1], u0 = u[2], up1 = u[3], up2 = u[4];
  real s0 = real(0.5) * (u0 + up1);
  real s1 = real(0.5) * (real(3.0) * u0 - um1);
  real s2 = real(1.0 / 8.0) * (real(3.0) * u0 + real(6.0) * up1 - up2);
  real s3 = real(1.0 / 8.0) * (real(3.0) * um2 - real(10.0) * um1 + real(15.0) * u0);
  const double d0 = 15.0 / 32.0, d1 = 5.0 / 32.0, d2 = 5.0 / 16.0, d3 = 1.0 / 16.0;
  return real(d0) * s0 + real(d1) * s1 + real(d2) * s2 + real(d3) * s3;
}

// ---------------------------------------------------------------------------
// Positivity-preserving interpolation limiter (Sec. 4.3.2, Alg.
// interp_limit_densities, Alg. interp_limit_vol_frac and the hard switch).
// Reading: the limiter acts on the primitive midpoint vector; the partial
// densities and volume fractions it changes are the same entries in V and W,
// velocity and pressure are held, and rho c^2 for the hard switch is
// gbar(alpha)(p + pbar_inf(alpha)) of the limited vector.
// Vt: interpolated midpoint state (modified in place); Vn: first-order (node) state.
// Returns 1 when the hard switch fired.
// ---------------------------------------------------------------------------
static int interp_limit(const FluidK& f, const or_params* P, real* Vt, const Cell& nodec) {
  const real* Vn = nodec.V;
  // Alg. interp_limit_densities: each partial density independently.
  for (int k = 0; k < f.N; ++k) {
    real a_lo = Vn[k], a_hi = Vt[k];
    real target = rmin(real(P->eps_ar), a_lo);
    real th = 1.0;
    if (a_hi < target) th = (target - a_lo) / (a_hi - a_lo);
    Vt[k] = (real(1.0) - th) * a_lo + th * a_hi;
  }
  // Alg. interp_limit_vol_frac: one theta for all volume fractions, k = 1..N
  // (alpha_N derived), combination applied to the N-1 stored alpha_k.
  real alt[OR_MAXN], aln[OR_MAXN];
  all_alpha(f, Vt, alt);
  all_alpha(f, Vn, aln);
  real th = 1.0;
  for (int k = 0; k < f.N; ++k) {
    real target = rmin(real(P->eps_a), aln[k]);
    real thk = 1.0;
    if (alt[k] < target) thk = (target - aln[k]) / (alt[k] - aln[k]);
    th = rmin(th, thk);
  }
  for (int k = 0; k < f.N - 1; ++k)
    Vt[sAL(f, k)] = (real(1.0) - th) * Vn[sAL(f, k)] + th * Vt[sAL(f, k)];
  // hard switch
  int hs = 0;
  all_alpha(f, Vt, alt);
  for (int k = 0; k < f.N; ++k) {
    if (Vt[k] < rmin(real(P->hs_ar), Vn[k])) hs = 1;
    if (alt[k] < rmin(real(P->hs_a), aln[k])) hs = 1;
  }
  real S, Pm;
  mixture(f, alt, S, Pm);
  real rc2 = rho_c2_of(S, Pm, Vt[sE(f)]);
  if (rc2 < rmin(real(P->hs_rc2), nodec.rc2)) hs = 1;
  if (hs)
    for (int m = 0; m < f.M; ++m) Vt[m] = Vn[m];
  return hs;
}

// ---------------------------------------------------------------------------
// Quasi-positivity-preserving flux limiter (Sec. 4.3.2, Alg.
// flux_limit_densities_vol_frac, Alg. flux_limit_energy, hard switch).
// Gm/Gp: high-order G^-_{i+1/2}, G^+_{i+1/2} (limited in place);
// Hm/Hp: first-order HLLC G^{HLLC,-}, G^{HLLC,+}; Wi/Wj = W_i, W_{i+1};
// Fi/Fj = F(W_i), F(W_{i+1}); lam = lambda_d.
// Reading: the garbled "theta^-" of the alpha branch is theta^{alpha_k,-}; theta
// solves (1-theta) a_low + theta a_high = min(eps, a_low) for theta.
// Returns a bit mask: 1 first stage limited, 2 energy stage limited, 4 hard switch.
// ---------------------------------------------------------------------------
static void half_state(const FluidK& f, const real* Wn, const real* G, const real* F, real lam2sgn,
                       real* out) {
  // W_i^{+} = W_i - 2 lam (G^- - F_i);  W_{i+1}^{-} = W_{i+1} + 2 lam (G^+ - F_{i+1})
  for (int m = 0; m < f.M; ++m) out[m] = Wn[m] + lam2sgn * (G[m] - F[m]);
}

static real theta_solve(real a_low, real a_high, real eps) {
  real target = rmin(eps, a_low);
  if (a_high < target) return (target - a_low) / (a_high - a_low);
  return 1.0;
}

static int flux_limit(const FluidK& f, const or_params* P, real lam, const real* Wi, const real* Wj,
                      const real* Fi, const real* Fj, real* Gm, real* Gp, const real* Hm,
                      const real* Hp) {
  int flags = 0;
  const real m2l = real(-2.0) * lam, p2l = real(2.0) * lam;
  real Wp[OR_MAXM], Wm[OR_MAXM], WHp[OR_MAXM], WHm[OR_MAXM];
  half_state(f, Wi, Gm, Fi, m2l, Wp);   // W_i^{+}
  half_state(f, Wj, Gp, Fj, p2l, Wm);   // W_{i+1}^{-}
  half_state(f, Wi, Hm, Fi, m2l, WHp);  // W_i^{HLLC,+}
  half_state(f, Wj, Hp, Fj, p2l, WHm);  // W_{i+1}^{HLLC,-}
  // Stage 1: partial densities and volume fractions, one theta.
  real th = 1.0;
  for (int k = 0; k < f.N; ++k) {
    real tp = theta_solve(WHp[k], Wp[k], real(P->eps_ar));
    real tm = theta_solve(WHm[k], Wm[k], real(P->eps_ar));
    th = rmin(th, rmin(tp, tm));
  }
  {
    real ap[OR_MAXN], am[OR_MAXN], aHp[OR_MAXN], aHm[OR_MAXN];
    all_alpha(f, Wp, ap);
    all_alpha(f, Wm, am);
    all_alpha(f, WHp, aHp);
    all_alpha(f, WHm, aHm);
    for (int k = 0; k < f.N; ++k) {
      real tp = theta_solve(aHp[k], ap[k], real(P->eps_a));
      real tm = theta_solve(aHm[k], am[k], real(P->eps_a));
      th = rmin(th, rmin(tp, tm));
    }
  }
  if (th < real(1.0)) flags |= 1;
  real Gsm[OR_MAXM], Gsp[OR_MAXM];
  for (int m = 0; m < f.M; ++m) {
    Gsp[m] = (real(1.0) - th) * Hp[m] + th * Gp[m];
    Gsm[m] = (real(1.0) - th) * Hm[m] + th * Gm[m];
  }
  // Stage 2: rho e~ (Alg. flux_limit_energy).
  real Wsp[OR_MAXM], Wsm[OR_MAXM];
  half_state(f, Wi, Gsm, Fi, m2l, Wsp);  // W_i^{*,+}
  half_state(f, Wj, Gsp, Fj, p2l, Wsm);  // W_{i+1}^{*,-}
  real rHp = rhoe_tilde(f, WHp), rHm = rhoe_tilde(f, WHm);
  real thp = theta_solve(rHp, rhoe_tilde(f, Wsp), real(P->eps_rhoe));
  real thm = theta_solve(rHm, rhoe_tilde(f, Wsm), real(P->eps_rhoe));
  real th2 = rmin(thp, thm);
  if (th2 < real(1.0)) flags |= 2;
  real Gssm[OR_MAXM], Gssp[OR_MAXM];
  for (int m = 0; m < f.M; ++m) {
    Gssp[m] = (real(1.0) - th2) * Hp[m] + th2 * Gsp[m];
    Gssm[m] = (real(1.0) - th2) * Hm[m] + th2 * Gsm[m];
  }
  // Hard switch with the smaller tolerances.
  real Wssp[OR_MAXM], Wssm[OR_MAXM];
  half_state(f, Wi, Gssm, Fi, m2l, Wssp);  // W_i^{**,+}
  half_state(f, Wj, Gssp, Fj, p2l, Wssm);  // W_{i+1}^{**,-}
  int hs = 0;
  {
    real a1[OR_MAXN], a2[OR_MAXN], aHp[OR_MAXN], aHm[OR_MAXN];
    all_alpha(f, Wssp, a1);
    all_alpha(f, Wssm, a2);
    all_alpha(f, WHp, aHp);
    all_alpha(f, WHm, aHm);
    for (int k = 0; k < f.N; ++k) {
      if (Wssp[k] < rmin(real(P->hs_ar), WHp[k])) hs = 1;
      if (a1[k] < rmin(real(P->hs_a), aHp[k])) hs = 1;
      if (Wssm[k] < rmin(real(P->hs_ar), WHm[k])) hs = 1;
      if (a2[k] < rmin(real(P->hs_a), aHm[k])) hs = 1;
    }
    if (rhoe_tilde(f, Wssp) < rmin(real(P->hs_rhoe), rHp)) hs = 1;
    if (rhoe_tilde(f, Wssm) < rmin(real(P->hs_rhoe), rHm)) hs = 1;
  }
  if (hs) {
    flags |= 4;
    for (int m = 0; m < f.M; ++m) {
      Gm[m] = Hm[m];
      Gp[m] = Hp[m];
    }
  } else {
    for (int m = 0; m < f.M; ++m) {
      Gm[m] = Gssm[m];
      Gp[m] = Gssp[m];
    }
  }
  return flags;
}

// Shock sensor (Sec. 4.3.1): normalised fourth-order second differences.
// u[0..5] = values at nodes i-2..i+3. Reading: a zero denominator gives 0.
static real sensor_half(real a, real b, real c, real d, real e) {
  real num = rabs_(real(16.0) * b - a - real(30.0) * c + real(16.0) * d - e);
  real den = rabs_(a + real(16.0) * b + real(30.0) * c + real(16.0) * d + e);
  if (den == real(0.0)) return 0.0;
  return num / den;
}
static real sensor_sigma(const real* u) {
  real sp = sensor_half(u[1], u[2], u[3], u[4], u[5]);  // i-1 .. i+3
  real sm = sensor_half(u[0], u[1], u[2], u[3], u[4]);  // i-2 .. i+2
  return real(0.5) * (sp + sm);
}

// Diagnostics of one face, for unit tests.
struct FaceDiag {
  real VL_weno[OR_MAXM], VR_weno[OR_MAXM], VL[OR_MAXM], VR[OR_MAXM];
  real Gt[OR_MAXM], ut, GH[OR_MAXM], uH, Ghcs[OR_MAXM], uhcs, sig;
  int hsL, hsR, flux_flags;
};

// Characteristic fields of the six-node stencil of a midpoint (App. D): the
// matrices come from the arithmetic averages of the partial densities, mixture
// density and sound speed at nodes i, i+1. Slot order of U: 0 -> u - p/(rho c),
// 1..N -> alpha_k rho_k - alpha_k rho_k p/(rho c^2), N+1.. -> tangential
// velocities (increasing direction), then the N-1 alpha_k, last -> u + p/(rho c).
static void project_stencil(const FluidK& f, int dir, const Cell* nd, real U[6][OR_MAXM], real* arb,
                            real& rhob, real& cb) {
  const int M = f.M, N = f.N, D = f.D;
  const int un = sMOM(f, dir), sp = sE(f);
  const Cell& ci = nd[2];
  const Cell& cj = nd[3];
  for (int k = 0; k < N; ++k) arb[k] = real(0.5) * (ci.V[k] + cj.V[k]);
  rhob = real(0.5) * (ci.rho + cj.rho);
  cb = real(0.5) * (ci.c + cj.c);
  int tang[2], nt = 0;
  for (int d = 0; d < D; ++d)
    if (d != dir) tang[nt++] = d;
  // entries of R^{-1}: 1/(rho c) and alpha_k rho_k/(rho c^2) of the averaged state
  const real inv_rc = real(1.0) / (rhob * cb);
  const real rc2b = rhob * cb * cb;
  real ark_rc2[OR_MAXN];
  for (int k = 0; k < N; ++k) ark_rc2[k] = arb[k] / rc2b;
  for (int j = 0; j < 6; ++j) {
    const real* V = nd[j].V;
    real p = V[sp];
    U[j][0] = V[un] - inv_rc * p;
    for (int k = 0; k < N; ++k) U[j][1 + k] = V[k] - ark_rc2[k] * p;
    for (int t = 0; t < nt; ++t) U[j][N + 1 + t] = V[sMOM(f, tang[t])];
    for (int k = 0; k < N - 1; ++k) U[j][N + D + k] = V[sAL(f, k)];
    U[j][M - 1] = V[un] + inv_rc * p;
  }
}

// Back-projection V = R U of one characteristic vector (App. D): the columns of
// R are built from the same averaged state as R^{-1} in project_stencil; its
// entries alpha_k rho_k/(2c) and rho c/2.
static void back_project(const FluidK& f, int dir, const real* arb, real rhob, real cb, const real* Ut,
                         real* Vt) {
  const int M = f.M, N = f.N, D = f.D;
  const int un = sMOM(f, dir), sp = sE(f);
  int tang[2], nt = 0;
  for (int d = 0; d < D; ++d)
    if (d != dir) tang[nt++] = d;
  real ark_2c[OR_MAXN];
  for (int k = 0; k < N; ++k) ark_2c[k] = arb[k] / (real(2.0) * cb);
  const real rc_2 = rhob * cb / real(2.0);
  for (int k = 0; k < N; ++k) Vt[k] = (-ark_2c[k]) * Ut[0] + Ut[1 + k] + ark_2c[k] * Ut[M - 1];
  Vt[un] = real(0.5) * Ut[0] + real(0.5) * Ut[M - 1];
  for (int t = 0; t < nt; ++t) Vt[sMOM(f, tang[t])] = Ut[N + 1 + t];
  Vt[sp] = (-rc_2) * Ut[0] + rc_2 * Ut[M - 1];
  for (int k = 0; k < N - 1; ++k) Vt[sAL(f, k)] = Ut[N + D + k];
}

// Whether the six node states of a midpoint are bit-identical.
static bool uniform_nodes(const FluidK& f, const Cell* nd) {
  for (int m = 0; m < f.M; ++m) {
    uint64_t b[6];
    for (int j = 0; j < 6; ++j) {
      const double x = val(nd[j].W[m]);
      std::memcpy(&b[j], &x, sizeof x);
    }
    for (int j = 0; j < 6; ++j)
      if (b[j] != b[2]) return false;
  }
  return true;
}

// ---------------------------------------------------------------------------
// One midpoint x_{i+1/2} in direction `dir` from the six node cells
// nd[0..5] = i-2 .. i+3. Produces the quasi-conservative fluxes
// Gm = G^-_{i+1/2} (used by cell i) and Gp = G^+_{i+1/2} (used by cell i+1).
// ---------------------------------------------------------------------------
// lin: the midpoint is gated smooth -- every WENO-IS weight is replaced by its
// linear weight d_k; everything else is unchanged.
static void face_flux(const FluidK& f, const or_params* P, int dir, real lam, const Cell* nd,
                      real* Gm, real* Gp, FaceDiag* dg, int lin = 0) {
  const int M = f.M, N = f.N;
  const Cell& ci = nd[2];
  const Cell& cj = nd[3];
  const int un = sMOM(f, dir), sp = sE(f);

  // A uniform stencil (six bit-identical node states) of the high-order scheme
  // takes the node's physical flux F^d with zero alpha slots: in exact arithmetic
  // that is what every step below returns. The WENO-IS and linear interpolations
  // reproduce a constant (App. C), so V~_L = V~_R = V; the HLLC flux of two equal
  // states is their physical flux (Sec. 4.1.1); the HCS weights sum to one
  // (psi - 2 a1 + 2 a2 - 2 a3 = 1), so G^HCS = G~ and any sensor blend of the two
  // returns it, with u^ the node velocity; the quasi-conservative alpha slots are
  // then alpha u - u alpha = 0 (Eq. G_pm); and the node state is each positivity
  // limiter's own first-order candidate, so neither limiter changes the result
  // (Sec. 4.3.2). The diagnostic path (dg) evaluates every step.
  if (!dg && P->scheme == 0 && uniform_nodes(f, nd)) {
    flux_F(f, dir, ci.V, ci.W, Gm);
    for (int m = 0; m < M; ++m) Gp[m] = Gm[m];
    return;
  }

  // First-order HLLC flux G^{HLLC} and u_* from the node states (Sec. 4.1.1).
  real GH[OR_MAXM], uH;
  hllc(f, dir, ci.V, cj.V, GH, &uH);

  real Ghat[OR_MAXM], uhat;
  if (P->scheme == 1) {
    for (int m = 0; m < M; ++m) Ghat[m] = GH[m];
    uhat = uH;
  } else {
    // ---- characteristic projection (App. D)
    real arb[OR_MAXN], rhob, cb;
    real U[6][OR_MAXM];
    project_stencil(f, dir, nd, U, arb, rhob, cb);
    // ---- WENO-IS left- and right-biased interpolation of each field (App. C)
    real UL[OR_MAXM], UR[OR_MAXM];
    for (int m = 0; m < M; ++m) {
      real sl[5] = {U[0][m], U[1][m], U[2][m], U[3][m], U[4][m]};
      real sr[5] = {U[5][m], U[4][m], U[3][m], U[2][m], U[1][m]};
      if (lin) {
        UL[m] = weno_lin_left(sl);
        UR[m] = weno_lin_left(sr);
      } else {
        UL[m] = weno_is_left(sl, P->weno_eps, nullptr);
        UR[m] = weno_is_left(sr, P->weno_eps, nullptr);
      }
    }
    // ---- back to primitive variables: V~ = R U~ (App. D)
    real VL[OR_MAXM], VR[OR_MAXM];
    back_project(f, dir, arb, rhob, cb, UL, VL);
    back_project(f, dir, arb, rhob, cb, UR, VR);
    if (dg)
      for (int m = 0; m < M; ++m) {
        dg->VL_weno[m] = VL[m];
        dg->VR_weno[m] = VR[m];
      }
    // ---- positivity-preserving interpolation limiter (Sec. 4.3.2)
    int hsL = 0, hsR = 0;
    if (P->limiters) {
      hsL = interp_limit(f, P, VL, ci);
      hsR = interp_limit(f, P, VR, cj);
    }
    if (dg) {
      for (int m = 0; m < M; ++m) {
        dg->VL[m] = VL[m];
        dg->VR[m] = VR[m];
      }
      dg->hsL = hsL;
      dg->hsR = hsR;
    }
    // ---- high-order midpoint flux G~ and velocity u~ (HLLC on V~_L, V~_R)
    real Gt[OR_MAXM], ut;
    hllc(f, dir, VL, VR, Gt, &ut);
    // ---- explicit HCS reconstruction (Eqs. reconstructed_G, reconstructed_vel)
    const double psi = 256.0 / 175.0;
    const double a1 = 75.0 * psi / 128.0 - 37.0 / 60.0;
    const double a2 = 25.0 * psi / 256.0 - 2.0 / 15.0;
    const double a3 = 3.0 * psi / 256.0 - 1.0 / 60.0;
    real Gn[6][OR_MAXM];
    for (int j = 0; j < 6; ++j) flux_G(f, dir, nd[j].V, nd[j].W, Gn[j]);
    real Ghcs[OR_MAXM];
    for (int m = 0; m < M; ++m)
      Ghcs[m] = real(psi) * Gt[m] - real(a1) * (Gn[2][m] + Gn[3][m]) +
                real(a2) * (Gn[1][m] + Gn[4][m]) - real(a3) * (Gn[0][m] + Gn[5][m]);
    real uhcs = real(psi) * ut - real(a1) * (nd[2].V[un] + nd[3].V[un]) +
                real(a2) * (nd[1].V[un] + nd[4].V[un]) - real(a3) * (nd[0].V[un] + nd[5].V[un]);
    // ---- shock-sensor blending (Eqs. flux_blending, velocity_blending)
    real sig = 0.0;
    if (P->blend) {
      real r6[6], p6[6];
      for (int j = 0; j < 6; ++j) {
        r6[j] = nd[j].rho;
        p6[j] = nd[j].V[sp];
      }
      real prod = sensor_sigma(r6) * sensor_sigma(p6);
      real powq = prod;  // [sigma(rho) sigma(p)]^q with integer q
      for (int e = 1; e < (int)P->q_sensor; ++e) powq = powq * prod;
      sig = rtanh_(real(P->Cs) * powq);
    }
    for (int m = 0; m < M; ++m) Ghat[m] = sig * Gt[m] + (real(1.0) - sig) * Ghcs[m];
    uhat = sig * ut + (real(1.0) - sig) * uhcs;
    if (dg) {
      for (int m = 0; m < M; ++m) {
        dg->Gt[m] = Gt[m];
        dg->Ghcs[m] = Ghcs[m];
      }
      dg->ut = ut;
      dg->uhcs = uhcs;
      dg->sig = sig;
    }
  }
  if (dg) {
    for (int m = 0; m < M; ++m) dg->GH[m] = GH[m];
    dg->uH = uH;
  }
  // ---- quasi-conservative fluxes G^-, G^+ (Eq. G_pm and its high-order form)
  real Hm[OR_MAXM], Hp[OR_MAXM];
  for (int m = 0; m < M; ++m) {
    Gm[m] = Ghat[m];
    Gp[m] = Ghat[m];
    Hm[m] = GH[m];
    Hp[m] = GH[m];
  }
  for (int k = 0; k < N - 1; ++k) {
    int s = sAL(f, k);
    Gm[s] = Ghat[s] - uhat * ci.V[s];
    Gp[s] = Ghat[s] - uhat * cj.V[s];
    Hm[s] = GH[s] - uH * ci.V[s];
    Hp[s] = GH[s] - uH * cj.V[s];
  }
  int flags = 0;
  if (P->limiters && P->scheme == 0) {
    real Fi[OR_MAXM], Fj[OR_MAXM];
    flux_F(f, dir, ci.V, ci.W, Fi);
    flux_F(f, dir, cj.V, cj.W, Fj);
    flags = flux_limit(f, P, lam, ci.W, cj.W, Fi, Fj, Gm, Gp, Hm, Hp);
  }
  if (dg) dg->flux_flags = flags;
}

// ---------------------------------------------------------------------------
// Grid-level helpers
// ---------------------------------------------------------------------------
static inline int64_t map_index(const or_grid* g, int d, int64_t j) {
  int64_t n = g->n[d];
  if (j < 0) return g->bc[2 * d] == 1 ? j + n : 0;
  if (j >= n) return g->bc[2 * d + 1] == 1 ? j - n : n - 1;
  return j;
}

static inline int64_t ncells(const or_grid* g) {
  int64_t c = 1;
  for (int d = 0; d < g->D; ++d) c *= g->n[d];
  return c;
}

static inline int64_t lin(const or_grid* g, const int64_t* ijk) {
  int64_t nx = g->n[0], ny = g->D > 1 ? g->n[1] : 1;
  int64_t j = g->D > 1 ? ijk[1] : 0, k = g->D > 2 ? ijk[2] : 0;
  return (k * ny + j) * nx + ijk[0];
}

static void load_W(const FluidK& f, const double* W, int64_t nc, int64_t c, real* out) {
  for (int m = 0; m < f.M; ++m) out[m] = real(W[(int64_t)m * nc + c]);
}

// Cells of the boundary slice normal to d and the index of the slice cell that
// continues line ijk (the other directions' indices, lowest fastest).
static int64_t slice_cells(const or_grid* g, int d) {
  int64_t s = 1;
  for (int e = 0; e < g->D; ++e)
    if (e != d) s *= g->n[e];
  return s;
}
static int64_t slice_index(const or_grid* g, int d, const int64_t* ijk) {
  int64_t s = 0, stride = 1;
  for (int e = 0; e < g->D; ++e) {
    if (e == d) continue;
    s += ijk[e] * stride;
    stride *= g->n[e];
  }
  return s;
}

// W of node j (possibly outside the grid) on the line through ijk along d.
static void load_node(const FluidK& f, const or_grid* g, const double* W, int d, const int64_t* ijk, int64_t j,
                      real* out) {
  const int side = j < 0 ? 0 : (j >= g->n[d] ? 1 : -1);
  if (side >= 0 && g->bc[2 * d + side] == 2) {
    load_W(f, g->bnd[2 * d + side], slice_cells(g, d), slice_index(g, d, ijk), out);
    return;
  }
  int64_t q[3] = {ijk[0], ijk[1], ijk[2]};
  q[d] = map_index(g, d, j);
  load_W(f, W, ncells(g), lin(g, q), out);
}

// L(W): the semi-discrete right-hand side of Eq. semi_W_G_pm_eqn, direction by
// direction: RHS_i = -sum_d (G^{d,-}_{i+1/2} - G^{d,+}_{i-1/2}) / dx_d.
// gate (nullable): per direction, one byte per midpoint over that direction's
// midpoint grid (n_d + 1 midpoints along d, x fastest); nonzero = gated smooth.
static void rhs_impl(const FluidK& f, const or_params* P, const or_grid* g, const double* W,
                     const real* lam, real* RHS, const uint8_t* const* gate = nullptr) {
  const int M = f.M;
  const int64_t nc = ncells(g);
  for (int64_t c = 0; c < nc * M; ++c) RHS[c] = 0.0;
  for (int dir = 0; dir < g->D; ++dir) {
    const int64_t n = g->n[dir];
    // iterate over all lines along dir (independent: each writes its own cells;
    // with -DOR_OMP they are shared among threads, which changes no result)
    int64_t nl = nc / n;
#ifdef OR_OMP
#pragma omp parallel
#endif
    {
    std::vector<Cell> line(n + 6);
    std::vector<real> Gm((n + 1) * M), Gp((n + 1) * M);
#ifdef OR_OMP
#pragma omp for schedule(static)
#endif
    for (int64_t l = 0; l < nl; ++l) {
      // the other two indices of line l
      int64_t ijk[3] = {0, 0, 0};
      int64_t rem = l;
      for (int d = 0; d < g->D; ++d) {
        if (d == dir) continue;
        ijk[d] = rem % g->n[d];
        rem /= g->n[d];
      }
      // node cells j = -3 .. n+2 with boundary conditions
      for (int64_t j = -3; j < n + 3; ++j) {
        real w[OR_MAXM];
        load_node(f, g, W, dir, ijk, j, w);
        cell_from_W(f, w, line[j + 3]);
      }
      // faces f = 0..n: face f lies between cells f-1 and f; stencil f-3..f+2
      for (int64_t fc = 0; fc <= n; ++fc) {
        int lin_gate = 0;
        if (gate && gate[dir]) {
          int64_t q[3] = {ijk[0], ijk[1], ijk[2]};
          q[dir] = fc;
          const int64_t f0 = g->n[0] + (dir == 0);
          const int64_t f1 = (g->D > 1 ? g->n[1] : 1) + (dir == 1);
          lin_gate = gate[dir][(q[2] * f1 + q[1]) * f0 + q[0]] != 0;
        }
        face_flux(f, P, dir, lam[dir], &line[fc], &Gm[fc * M], &Gp[fc * M], nullptr, lin_gate);
      }
      for (int64_t i = 0; i < n; ++i) {
        int64_t q[3] = {ijk[0], ijk[1], ijk[2]};
        q[dir] = i;
        int64_t c = lin(g, q);
        for (int m = 0; m < M; ++m)
          RHS[(int64_t)m * nc + c] =
              RHS[(int64_t)m * nc + c] - (Gm[(i + 1) * M + m] - Gp[i * M + m]) / real(g->dx[dir]);
      }
    }
    }
  }
}

// Thermal relaxation of one cell at infinite rate (Sec. 4.2). Keeps
// alpha_k rho_k, rho u and E; replaces the N-1 stored alpha_k by alpha_k^*.
// Reading: p^* is the positive root written in the cancellation-free form
// (-2C/(B + sqrt(disc)) when B > 0), T^* from Eq. T_relax_e.
static void relax_cell(const FluidK& f, real* W, real* pT_out) {
  const int N = f.N, l = f.liq;
  real rho = 0.0;
  for (int k = 0; k < N; ++k) rho = rho + W[k];
  real Y[OR_MAXN];
  for (int k = 0; k < N; ++k) Y[k] = W[k] / rho;
  real re = rhoe_tilde(f, W);  // rho (e - qbar)
  real cvb = 0.0, cpb = 0.0;
  for (int k = 0; k < N; ++k) {
    cvb = cvb + Y[k] * real(f.cv[k]);
    cpb = cpb + Y[k] * real(f.cp[k]);
  }
  const real pinf1 = f.pinf[l];
  const real R1 = f.Rgas[l];
  // Eqs. Ap_Bp_Cp_1 .. Ap_Bp_Cp_3 (species `liq` plays the role of species 1)
  real Ap = cvb;
  real Bp = -(re * (cpb - cvb) - pinf1 * cvb - pinf1 * Y[l] * R1);
  real Cp = -(re * pinf1 * ((cpb - cvb) - Y[l] * R1));
  real disc = Bp * Bp - real(4.0) * Ap * Cp;
  real sq = rsqrt_(disc);
  real ps;
  if (Bp > real(0.0))
    ps = real(-2.0) * Cp / (Bp + sq);
  else
    ps = (sq - Bp) / (real(2.0) * Ap);
  // Eq. T_relax_e: T* = (e - qbar) / [Y_1 (p*+gamma_1 p_inf1) c_v1/(p*+p_inf1) + cvbar - Y_1 c_v1]
  const real g1 = f.gamma[l];
  real den = Y[l] * (ps + g1 * pinf1) * real(f.cv[l]) / (ps + pinf1) + cvb - Y[l] * real(f.cv[l]);
  real Ts = (re / rho) / den;
  // rho_k^* (Eq. rho_k_thermally_relaxed), alpha_k^* = rho Y_k / rho_k^*
  for (int k = 0; k < N - 1; ++k) {
    real rhok = (ps + real(f.pinf[k])) / (real(f.Rgas[k]) * Ts);  // (gamma_k - 1) c_v,k = R_k
    W[sAL(f, k)] = W[k] / rhok;
  }
  if (pT_out) {
    pT_out[0] = ps;
    pT_out[1] = Ts;
  }
}

static void relax_grid(const FluidK& f, int64_t nc, double* W) {
#ifdef OR_OMP
#pragma omp parallel for schedule(static)
#endif
  for (int64_t c = 0; c < nc; ++c) {
    real w[OR_MAXM];
    load_W(f, W, nc, c, w);
    relax_cell(f, w, nullptr);
    for (int m = 0; m < f.M; ++m) W[(int64_t)m * nc + c] = val(w[m]);
  }
}

// Four-equation HRM sound speed of a cell (Eq. 4_eqn_sos) at its equilibrium
// state (Sec. 4.2): out = {c4, p, T, Gamma, Psi_1..Psi_N}; Psi_k and Gamma by
// implicit differentiation of the p* quadratic (Sec. 3 definitions).
static void c4eq_impl(const FluidK& f, const real* W, real* out) {
  const int N = f.N, l = f.liq;
  real w[OR_MAXM];
  for (int m = 0; m < f.M; ++m) w[m] = W[m];
  real pT[2];
  relax_cell(f, w, pT);  // equilibrium p, T of this (alpha_k rho_k, rho u, E)
  real p = pT[0];
  real rho = 0.0;
  for (int k = 0; k < N; ++k) rho = rho + w[k];
  real Y[OR_MAXN];
  for (int k = 0; k < N; ++k) Y[k] = w[k] / rho;
  real re = rhoe_tilde(f, w);
  real cvb = 0.0, cpb = 0.0;
  for (int k = 0; k < N; ++k) {
    cvb = cvb + Y[k] * real(f.cv[k]);
    cpb = cpb + Y[k] * real(f.cp[k]);
  }
  const real pinf1 = f.pinf[l];
  const real R1 = f.Rgas[l];
  const real Rb = cpb - cvb;
  real Ap = cvb;
  real Bp = -(re * Rb - pinf1 * cvb - pinf1 * Y[l] * R1);
  real denom = real(2.0) * Ap * p + Bp;
  // e-derivatives at fixed partial densities: d(rho e~)/de = rho
  real dB_de = -(rho * Rb);
  real dC_de = -(pinf1 * rho * (Rb - Y[l] * R1));
  real Gam = (-(dB_de * p + dC_de) / denom) / rho;
  real c2 = Gam * p / rho;
  for (int k = 0; k < N; ++k) {
    // derivatives at fixed e and other partial densities
    real e_spec = re / rho;  // e - qbar
    real qbar = 0.0;
    for (int s = 0; s < N; ++s) qbar = qbar + Y[s] * real(f.q[s]);
    real drhoe = (e_spec + qbar) - real(f.q[k]);  // d(rho e - sum ar q)/d ar_k = e - q_k
    real dcv = (real(f.cv[k]) - cvb) / rho;
    real dRb = (real(f.Rgas[k]) - Rb) / rho;
    real dY1 = ((k == l ? real(1.0) : real(0.0)) - Y[l]) / rho;
    real dA = dcv;
    real dB = -(drhoe * Rb + re * dRb - pinf1 * dcv - pinf1 * R1 * dY1);
    real dC = -(pinf1 * (drhoe * (Rb - Y[l] * R1) + re * (dRb - R1 * dY1)));
    real Psi = -(dA * p * p + dB * p + dC) / denom;
    out[4 + k] = Psi;
    c2 = c2 + Y[k] * Psi;
  }
  out[0] = rsqrt_(c2);
  out[1] = p;
  out[2] = pT[1];
  out[3] = Gam;
}


// Max wave speed per direction (Sec. 4.1.2): tau_d = max(|u_d| + c)/dx_d with the
// five-equation sound speed.
// Reading: the prescribed states of Dirichlet sides enter the maximum too (their
// waves enter the domain at once).
static void tau_impl(const FluidK& f, const or_grid* g, const double* W, real* tau, int sound = 0) {
  const int64_t nc = ncells(g);
  for (int d = 0; d < g->D; ++d) tau[d] = 0.0;
  auto visit = [&](const double* X, int64_t n, int64_t c) {
    real w[OR_MAXM];
    load_W(f, X, n, c, w);
    Cell C;
    cell_from_W(f, w, C);
    real cw = C.c;  // five-equation c (sound 0) or the four-equation HRM c (sound 1)
    if (sound == 1) {
      real o[4 + OR_MAXN];
      c4eq_impl(f, w, o);
      cw = o[0];
    }
    for (int d = 0; d < g->D; ++d) {
      real s = (rabs_(C.V[sMOM(f, d)]) + cw) / real(g->dx[d]);
      tau[d] = rmax(tau[d], s);
    }
  };
  for (int64_t c = 0; c < nc; ++c) visit(W, nc, c);
  for (int b = 0; b < 2 * g->D; ++b)
    if (g->bc[b] == 2) {
      const int64_t ns = slice_cells(g, b / 2);
      for (int64_t c = 0; c < ns; ++c) visit(g->bnd[b], ns, c);
    }
}

// Directional split: sigma_d = tau_d / sum tau, lambda_d = dt/(sigma_d dx_d)
// (Sec. 4.1.2; for a given dt the split comes from the step-start state).
static void lambdas(const or_grid* g, const real* tau, real dt, real* lam) {
  real st = 0.0;
  for (int d = 0; d < g->D; ++d) st = st + tau[d];
  for (int d = 0; d < g->D; ++d) {
    real sigma = tau[d] / st;
    lam[d] = dt / (sigma * real(g->dx[d]));
  }
}

extern "C" {

// --------------------------- exported API ---------------------------------

void or_params_default(or_params* p) {
  memset(p, 0, sizeof(*p));
  p->limiters = 1;
  p->blend = 1;
  p->relax_mode = 1;
  p->scheme = 0;
  p->integrator = 0;
  p->eps_ar = 1.0e-10;  // Sec. 4.3.2
  p->eps_a = 1.0e-10;
  p->eps_rhoe = 1.0e-8;
  p->hs_ar = 1.0e-11;
  p->hs_a = 1.0e-11;
  p->hs_rc2 = 1.0e-9;
  p->hs_rhoe = 1.0e-9;
  p->weno_eps = 1.0e-15;  // App. C
  p->Cs = 1.0e12;         // Sec. 4.3.1
  p->q_sensor = 2.0;
}

// out[0..3] = rho, c, rho c^2, rho(e - qbar); V[M] primitive vector.
void or_prim_cell(const or_fluid* fl, const double* W, double* V, double* out) {
  FluidK f = make_fluid(fl);
  real w[OR_MAXM];
  for (int m = 0; m < f.M; ++m) w[m] = W[m];
  Cell C;
  cell_from_W(f, w, C);
  for (int m = 0; m < f.M; ++m) V[m] = val(C.V[m]);
  out[0] = val(C.rho);
  out[1] = val(C.c);
  out[2] = val(C.rc2);
  out[3] = val(rhoe_tilde(f, w));
}

// W[M], out[0..2] = rho, c, E from a primitive vector.
void or_cons_cell(const or_fluid* fl, const double* V, double* W, double* out) {
  FluidK f = make_fluid(fl);
  real v[OR_MAXM];
  for (int m = 0; m < f.M; ++m) v[m] = V[m];
  PState s;
  pstate_from_V(f, v, s);
  for (int m = 0; m < f.M; ++m) W[m] = val(s.W[m]);
  out[0] = val(s.rho);
  out[1] = val(s.c);
  out[2] = val(s.E);
}

double or_weno_left(const double* u, double eps, double* omega) {
  real r[5], om[4];
  for (int j = 0; j < 5; ++j) r[j] = u[j];
  real v = weno_is_left(r, eps, om);
  if (omega)
    for (int k = 0; k < 4; ++k) omega[k] = val(om[k]);
  return val(v);
}

double or_hllc(const or_fluid* fl, int dir, const double* VL, const double* VR, double* G) {
  FluidK f = make_fluid(fl);
  real l[OR_MAXM], r[OR_MAXM], g[OR_MAXM], ss;
  for (int m = 0; m < f.M; ++m) {
    l[m] = VL[m];
    r[m] = VR[m];
  }
  hllc(f, dir, l, r, g, &ss);
  for (int m = 0; m < f.M; ++m) G[m] = val(g[m]);
  return val(ss);
}

double or_sensor(const double* u6) {
  real r[6];
  for (int j = 0; j < 6; ++j) r[j] = u6[j];
  return val(sensor_sigma(r));
}

// One face from six node conservative states W6[j*M + m], j = i-2..i+3.
// diag (optional, 8*M+8 doubles): VL_weno, VR_weno, VL, VR, Gt, GH, Ghcs, [ut, uH, uhcs, sig,
// hsL, hsR, flux_flags, 0].
void or_face(const or_fluid* fl, const or_params* P, int dir, double lam, const double* W6,
             double* Gm, double* Gp, double* diag) {
  FluidK f = make_fluid(fl);
  Cell nd[6];
  for (int j = 0; j < 6; ++j) {
    real w[OR_MAXM];
    for (int m = 0; m < f.M; ++m) w[m] = W6[j * f.M + m];
    cell_from_W(f, w, nd[j]);
  }
  real gm[OR_MAXM], gp[OR_MAXM];
  FaceDiag dg;
  memset(&dg, 0, sizeof(dg));
  face_flux(f, P, dir, real(lam), nd, gm, gp, &dg);
  for (int m = 0; m < f.M; ++m) {
    Gm[m] = val(gm[m]);
    Gp[m] = val(gp[m]);
  }
  if (diag) {
    int M = f.M;
    for (int m = 0; m < M; ++m) {
      diag[0 * M + m] = val(dg.VL_weno[m]);
      diag[1 * M + m] = val(dg.VR_weno[m]);
      diag[2 * M + m] = val(dg.VL[m]);
      diag[3 * M + m] = val(dg.VR[m]);
      diag[4 * M + m] = val(dg.Gt[m]);
      diag[5 * M + m] = val(dg.GH[m]);
      diag[6 * M + m] = val(dg.Ghcs[m]);
    }
    double* t = diag + 7 * M;
    t[0] = val(dg.ut);
    t[1] = val(dg.uH);
    t[2] = val(dg.uhcs);
    t[3] = val(dg.sig);
    t[4] = dg.hsL;
    t[5] = dg.hsR;
    t[6] = dg.flux_flags;
  }
}

// Interpolation limiter of one biased midpoint state (Sec. 4.3.2, the two
// interpolation algorithms and the hard switch): Vt (M, in/out) is the
// interpolated primitive vector, Wn the conservative vector of its node (W_i
// for the left-biased, W_{i+1} for the right-biased state). Returns 1 when the
// hard switch fired.
int or_interp_limit(const or_fluid* fl, const or_params* P, double* Vt, const double* Wn) {
  FluidK f = make_fluid(fl);
  real w[OR_MAXM], v[OR_MAXM];
  for (int m = 0; m < f.M; ++m) {
    w[m] = Wn[m];
    v[m] = Vt[m];
  }
  Cell c;
  cell_from_W(f, w, c);
  int hs = interp_limit(f, P, v, c);
  for (int m = 0; m < f.M; ++m) Vt[m] = val(v[m]);
  return hs;
}

// Flux limiter of one midpoint (Sec. 4.3.2, the two flux algorithms and the
// hard switch): W_i, W_{i+1}, the high-order G^-_{i+1/2}, G^+_{i+1/2} (in/out)
// and the first-order G^{HLLC,-}, G^{HLLC,+}; F_i and F_{i+1} (direction dir)
// are evaluated from W_i and W_{i+1}. Returns flux_limit's flag mask.
int or_flux_limit(const or_fluid* fl, const or_params* P, int dir, double lam, const double* Wi,
                  const double* Wj, double* Gm, double* Gp, const double* Hm, const double* Hp) {
  FluidK f = make_fluid(fl);
  real wi[OR_MAXM], wj[OR_MAXM], gm[OR_MAXM], gp[OR_MAXM], hm[OR_MAXM], hp[OR_MAXM];
  for (int m = 0; m < f.M; ++m) {
    wi[m] = Wi[m];
    wj[m] = Wj[m];
    gm[m] = Gm[m];
    gp[m] = Gp[m];
    hm[m] = Hm[m];
    hp[m] = Hp[m];
  }
  Cell ci, cj;
  cell_from_W(f, wi, ci);
  cell_from_W(f, wj, cj);
  real Fi[OR_MAXM], Fj[OR_MAXM];
  flux_F(f, dir, ci.V, ci.W, Fi);
  flux_F(f, dir, cj.V, cj.W, Fj);
  int flags = flux_limit(f, P, real(lam), ci.W, cj.W, Fi, Fj, gm, gp, hm, hp);
  for (int m = 0; m < f.M; ++m) {
    Gm[m] = val(gm[m]);
    Gp[m] = val(gp[m]);
  }
  return flags;
}

// The projection matrices of a midpoint in direction dir from its nodes W_i,
// W_{i+1} (App. D), as the face computation applies them: column m of Rinv is
// the characteristic vector project_stencil makes of the unit primitive vector
// e_m, column m of R the primitive vector back_project makes of the unit
// characteristic vector e_m (both M*M, row-major). avg receives the averaged
// state the matrices use: alpha_k rho_k (N), rho, c.
void or_char_matrices(const or_fluid* fl, int dir, const double* Wi, const double* Wj, double* Rinv,
                      double* R, double* avg) {
  FluidK f = make_fluid(fl);
  const int M = f.M;
  real wi[OR_MAXM], wj[OR_MAXM];
  for (int m = 0; m < M; ++m) {
    wi[m] = Wi[m];
    wj[m] = Wj[m];
  }
  Cell nd[6];
  cell_from_W(f, wi, nd[2]);
  cell_from_W(f, wj, nd[3]);
  nd[0] = nd[1] = nd[4] = nd[5] = nd[2];
  real arb[OR_MAXN], rhob = 0.0, cb = 0.0;
  for (int col = 0; col < M; ++col) {
    for (int m = 0; m < M; ++m) nd[0].V[m] = real(m == col ? 1.0 : 0.0);
    real U[6][OR_MAXM];
    project_stencil(f, dir, nd, U, arb, rhob, cb);
    for (int m = 0; m < M; ++m) Rinv[m * M + col] = val(U[0][m]);
  }
  for (int col = 0; col < M; ++col) {
    real e[OR_MAXM], v[OR_MAXM];
    for (int m = 0; m < M; ++m) e[m] = real(m == col ? 1.0 : 0.0);
    back_project(f, dir, arb, rhob, cb, e, v);
    for (int m = 0; m < M; ++m) R[m * M + col] = val(v[m]);
  }
  for (int k = 0; k < f.N; ++k) avg[k] = val(arb[k]);
  avg[f.N] = val(rhob);
  avg[f.N + 1] = val(cb);
}

void or_rhs_gated(const or_fluid* fl, const or_params* P, const or_grid* g, const double* W,
                  const double* lam, const uint8_t* gx, const uint8_t* gy, const uint8_t* gz, double* RHS) {
  FluidK f = make_fluid(fl);
  int64_t nc = ncells(g);
  std::vector<real> r(nc * f.M);
  real l[3] = {lam[0], lam[1], lam[2]};
  const uint8_t* gates[3] = {gx, gy, gz};
  rhs_impl(f, P, g, W, l, r.data(), gates);
  for (int64_t c = 0; c < nc * f.M; ++c) RHS[c] = val(r[c]);
}

void or_rhs(const or_fluid* fl, const or_params* P, const or_grid* g, const double* W,
            const double* lam, double* RHS) {
  or_rhs_gated(fl, P, g, W, lam, nullptr, nullptr, nullptr, RHS);
}

// In place; pT (optional, 2 doubles) receives p* and T* of the last cell.
void or_relax_cell(const or_fluid* fl, double* W, double* pT) {
  FluidK f = make_fluid(fl);
  real w[OR_MAXM], o[2];
  for (int m = 0; m < f.M; ++m) w[m] = W[m];
  relax_cell(f, w, o);
  for (int m = 0; m < f.M; ++m) W[m] = val(w[m]);
  if (pT) {
    pT[0] = val(o[0]);
    pT[1] = val(o[1]);
  }
}

void or_relax(const or_fluid* fl, const or_grid* g, double* W) {
  FluidK f = make_fluid(fl);
  relax_grid(f, ncells(g), W);
}

// tau[d] and dt = CFL / sum tau (Sec. 4.1.2), with the wave speed's sound speed
// chosen: 0 five-equation c, 1 the four-equation HRM c (Eq. 4_eqn_sos). Returns dt.
double or_dt_sound(const or_fluid* fl, const or_grid* g, const double* W, double cfl, int sound, double* tau) {
  FluidK f = make_fluid(fl);
  real t[3] = {0.0, 0.0, 0.0};
  tau_impl(f, g, W, t, sound);
  real st = 0.0;
  for (int d = 0; d < g->D; ++d) {
    st = st + t[d];
    if (tau) tau[d] = val(t[d]);
  }
  return val(real(cfl) / st);
}

// tau[d] and dt with the five-equation c (Sec. 4.1.2). Returns dt.
double or_dt(const or_fluid* fl, const or_grid* g, const double* W, double cfl, double* tau) {
  return or_dt_sound(fl, g, W, cfl, 0, tau);
}

// lambda_d for a given dt from the state W (Sec. 4.1.2).
void or_lambdas(const or_fluid* fl, const or_grid* g, const double* W, double dt, double* lam) {
  FluidK f = make_fluid(fl);
  real t[3] = {0.0, 0.0, 0.0}, l[3] = {0.0, 0.0, 0.0};
  tau_impl(f, g, W, t);
  lambdas(g, t, real(dt), l);
  for (int d = 0; d < 3; ++d) lam[d] = val(l[d]);
}

// nsteps full time steps of size dt (Sec. 4.4): each stage is a forward-Euler
// step of the hyperbolic system followed by the thermal relaxation
// (relax_mode 1); SSP-RK3 in the Shu-Osher form, SSP-RK2 or forward Euler.
// lambda_d come from the state at the start of each step.
// gx, gy, gz (nullable): a fixed smoothness gate per direction (see rhs_impl),
// applied at every stage of every step.
}  // extern "C"

// The time integrators (Sec. 4.4, Sec. 5.1): SSP-RK3 in Shu-Osher form, SSP-RK2
// or forward Euler, relaxation after every stage (relax_mode 1), after the
// step (2) or never (0). rhs(Wstage, t_stage, L) supplies L(W); the stage
// times are t^n, t^n + dt and t^n + dt/2 (SSP-RK3), t^n and t^n + dt (SSP-RK2).
template <typename Rhs>
static void step_impl(const FluidK& f, const or_params* P, const or_grid* g, double* W, double dt, int nsteps,
                      double t0, Rhs&& rhs) {
  const int64_t nc = ncells(g), tot = nc * f.M;
  std::vector<double> W0(tot), W1(tot), W2(tot);
  std::vector<real> L(tot);
  for (int s = 0; s < nsteps; ++s) {
    const double tn = t0 + s * dt;
    for (int64_t c = 0; c < tot; ++c) W0[c] = W[c];
    const int relax_stage = (P->relax_mode == 1);
    // stage 1: W1 = W0 + dt L(W0)
    rhs(W0.data(), tn, L.data(), true);
    for (int64_t c = 0; c < tot; ++c) W1[c] = val(real(W0[c]) + real(dt) * L[c]);
    if (P->integrator == 1) {
      if (P->relax_mode != 0) relax_grid(f, nc, W1.data());
      for (int64_t c = 0; c < tot; ++c) W[c] = W1[c];
      continue;
    }
    if (relax_stage) relax_grid(f, nc, W1.data());
    rhs(W1.data(), tn + dt, L.data(), false);
    if (P->integrator == 2) {
      // SSP-RK2: W^{n+1} = 1/2 W0 + 1/2 (W1 + dt L(W1))
      for (int64_t c = 0; c < tot; ++c)
        W[c] = val(real(0.5) * real(W0[c]) + real(0.5) * (real(W1[c]) + real(dt) * L[c]));
      if (P->relax_mode != 0) relax_grid(f, nc, W);
      continue;
    }
    // SSP-RK3 stage 2: W2 = 3/4 W0 + 1/4 (W1 + dt L(W1))
    for (int64_t c = 0; c < tot; ++c)
      W2[c] = val(real(0.75) * real(W0[c]) + real(0.25) * (real(W1[c]) + real(dt) * L[c]));
    if (relax_stage) relax_grid(f, nc, W2.data());
    // stage 3: W^{n+1} = 1/3 W0 + 2/3 (W2 + dt L(W2))
    rhs(W2.data(), tn + 0.5 * dt, L.data(), false);
    for (int64_t c = 0; c < tot; ++c)
      W[c] = val(real(1.0 / 3.0) * real(W0[c]) + real(2.0 / 3.0) * (real(W2[c]) + real(dt) * L[c]));
    if (P->relax_mode != 0) relax_grid(f, nc, W);
  }
}

extern "C" {

// gx, gy, gz (nullable): a fixed smoothness gate per direction (see rhs_impl),
// applied at every stage of every step. lambda_d come from the state at the
// start of each step.
void or_step_gated(const or_fluid* fl, const or_params* P, const or_grid* g, double* W, double dt,
                   int nsteps, const uint8_t* gx, const uint8_t* gy, const uint8_t* gz) {
  const uint8_t* gates[3] = {gx, gy, gz};
  const uint8_t* const* gate = (gx || gy || gz) ? gates : nullptr;
  FluidK f = make_fluid(fl);
  real lam[3] = {0.0, 0.0, 0.0};
  step_impl(f, P, g, W, dt, nsteps, 0.0, [&](const double* Ws, double, real* L, bool first) {
    if (first) {
      real t[3] = {0.0, 0.0, 0.0};
      tau_impl(f, g, Ws, t, P->cfl_sound);
      lambdas(g, t, real(dt), lam);
    }
    rhs_impl(f, P, g, Ws, lam, L, gate);
  });
}

// Temporal convergence test of Sec. 5.1: the spatial operator replaced by the
// exact convective derivatives of the advected solution alpha_1 = a0 + a1
// sin(k (x - u t)) at constant u, p and species densities (two species, 1D):
// d(a_k r_k u)/dx = r_k u da_k/dx, d(rho u^2 + p)/dx = u^2 drho/dx,
// d((E + p) u)/dx = u d(rho e)/dx + u^3/2 drho/dx, u da_1/dx, with
// d(rho e)/dx = sum_k (rho_k e_k) da_k/dx and rho_k e_k = p/(g_k - 1) +
// g_k pinf_k/(g_k - 1) + rho_k q_k, evaluated at each stage's time.
// adv = {a0, a1, k, u, p, rho_1, rho_2, x0 (left end of the domain)}; t0: time
// of the initial state.
void or_step_exact(const or_fluid* fl, const or_params* P, const or_grid* g, double* W, double dt, int nsteps,
                   double t0, const double* adv) {
  FluidK f = make_fluid(fl);
  const int64_t n = g->n[0];
  const double a1 = adv[1], k = adv[2], u = adv[3], p = adv[4], r1 = adv[5], r2 = adv[6], x0 = adv[7];
  double re[2];
  for (int s = 0; s < 2; ++s)
    re[s] = p * f.inv_gm1[s] + f.gpinf_gm1[s] + (s == 0 ? r1 : r2) * f.q[s];
  step_impl(f, P, g, W, dt, nsteps, t0, [&](const double*, double t, real* L, bool) {
    for (int64_t i = 0; i < n; ++i) {
      const double x = x0 + (i + 0.5) * g->dx[0];
      const double da1 = a1 * k * std::cos(k * (x - u * t)), da2 = -da1;
      const double drho = r1 * da1 + r2 * da2;
      const double drhoe = re[0] * da1 + re[1] * da2;
      L[0 * n + i] = -(r1 * u * da1);
      L[1 * n + i] = -(r2 * u * da2);
      L[2 * n + i] = -(u * u * drho);
      L[3 * n + i] = -(u * drhoe + u * u * u / 2.0 * drho);
      L[4 * n + i] = -(u * da1);
    }
  });
}

void or_step(const or_fluid* fl, const or_params* P, const or_grid* g, double* W, double dt,
             int nsteps) {
  or_step_gated(fl, P, g, W, dt, nsteps, nullptr, nullptr, nullptr);
}

// Admissibility counters (Sec. 2, sets G and script-G): counts[0] cells with a
// negative partial density, [1] a volume fraction outside [0, 1], [2] rho c^2 <= 0,
// [3] rho(e - qbar) <= 0.
void or_admissibility(const or_fluid* fl, const or_grid* g, const double* W, int64_t* counts) {
  FluidK f = make_fluid(fl);
  const int64_t nc = ncells(g);
  for (int i = 0; i < 4; ++i) counts[i] = 0;
  for (int64_t c = 0; c < nc; ++c) {
    real w[OR_MAXM];
    load_W(f, W, nc, c, w);
    int bad_ar = 0, bad_a = 0;
    for (int k = 0; k < f.N; ++k)
      if (w[k] < real(0.0)) bad_ar = 1;
    real al[OR_MAXN];
    all_alpha(f, w, al);
    for (int k = 0; k < f.N; ++k)
      if (al[k] < real(0.0) || al[k] > real(1.0)) bad_a = 1;
    Cell C;
    cell_from_W(f, w, C);
    counts[0] += bad_ar;
    counts[1] += bad_a;
    counts[2] += (C.rc2 <= real(0.0)) || !(C.rc2 == C.rc2);
    real re = rhoe_tilde(f, w);
    counts[3] += (re <= real(0.0)) || !(re == re);
  }
}

// Four-equation HRM sound speed (Eq. 4_eqn_sos) by implicit differentiation of
// the p* quadratic (expressions below Fig. compare_sound_speed_flow_models).
// out: [0] c_4eq, [1] p, [2] T, [3] Gamma, [4..4+N) Psi_k.
void or_c4eq_cell(const or_fluid* fl, const double* W, double* out) {
  FluidK f = make_fluid(fl);
  real w[OR_MAXM], o[4 + OR_MAXN];
  for (int m = 0; m < f.M; ++m) w[m] = W[m];
  c4eq_impl(f, w, o);
  for (int i = 0; i < 4 + f.N; ++i) out[i] = val(o[i]);
}

// Initial state in pressure and temperature equilibrium (Sec. 5): from the
// primitive planes prim = (alpha_1..alpha_{N-1}, u_1..u_D, p, T) of `nc` cells,
// rho_k = (p + p_inf_k)/((gamma_k - 1) c_v,k T) (Eq. rho_k_thermally_relaxed),
// alpha_N = 1 - sum of the others, and E from the mixture EOS (Sec. 2):
// E = sum alpha_k (p + gamma_k p_inf_k)/(gamma_k - 1) + sum alpha_k rho_k q_k + rho |u|^2 / 2.
void or_ic_from_prim(const or_fluid* fl, int64_t nc, const double* prim, double* W) {
  FluidK f = make_fluid(fl);
  const int N = f.N, D = f.D;
  for (int64_t c = 0; c < nc; ++c) {
    real al[OR_MAXN];
    real s = 0.0;
    for (int k = 0; k < N - 1; ++k) {
      al[k] = prim[(int64_t)k * nc + c];
      s = s + al[k];
    }
    al[N - 1] = real(1.0) - s;
    real p = prim[(int64_t)(N + D - 1) * nc + c];
    real T = prim[(int64_t)(N + D) * nc + c];
    real rho = 0.0, E = 0.0;
    real ar[OR_MAXN];
    for (int k = 0; k < N; ++k) {
      real rhok = (p + real(f.pinf[k])) / (real(f.Rgas[k]) * T);
      ar[k] = al[k] * rhok;
      rho = rho + ar[k];
      E = E + al[k] * (p + real(f.gamma[k]) * real(f.pinf[k])) * real(f.inv_gm1[k]) + ar[k] * real(f.q[k]);
    }
    real kin = 0.0;
    for (int d = 0; d < D; ++d) {
      real u = prim[(int64_t)(N - 1 + d) * nc + c];
      kin = kin + u * u;
      W[(int64_t)sMOM(f, d) * nc + c] = val(rho * u);
    }
    E = E + real(0.5) * rho * kin;
    for (int k = 0; k < N; ++k) W[(int64_t)k * nc + c] = val(ar[k]);
    W[(int64_t)sE(f) * nc + c] = val(E);
    for (int k = 0; k < N - 1; ++k) W[(int64_t)sAL(f, k) * nc + c] = val(al[k]);
  }
}

// Operations performed by the midpoint computations alone (everything of
// face_flux: projection, WENO, limiters, two HLLC solves, HCS, blending, flux
// limiter) over every face of direction `dir`; the primitive variables of the
// node cells are computed outside the counted region. out[0..4] = add, mul, div,
// sqrt, tanh; returns the number of faces. Zero counts in the normal build.
// gated: every midpoint gated to the linear WENO weights (the operation count
// of a gated midpoint).
int64_t or_faces_flops_gated(const or_fluid* fl, const or_params* P, const or_grid* g, const double* W,
                             const double* lam, int dir, int gated, double* out) {
  FluidK f = make_fluid(fl);
  const int M = f.M;
  const int64_t nc = ncells(g), n = g->n[dir], nl = nc / n;
  std::vector<Cell> line(n + 6);
  std::vector<real> Gm(M), Gp(M);
  double acc[5] = {0, 0, 0, 0, 0};
  for (int64_t l = 0; l < nl; ++l) {
    int64_t ijk[3] = {0, 0, 0};
    int64_t rem = l;
    for (int d = 0; d < g->D; ++d) {
      if (d == dir) continue;
      ijk[d] = rem % g->n[d];
      rem /= g->n[d];
    }
    for (int64_t j = -3; j < n + 3; ++j) {
      int64_t q[3] = {ijk[0], ijk[1], ijk[2]};
      q[dir] = map_index(g, dir, j);
      real w[OR_MAXM];
      load_W(f, W, nc, lin(g, q), w);
      cell_from_W(f, w, line[j + 3]);
    }
#ifdef OR_COUNT
    OrCounts before = g_cnt;
#endif
    for (int64_t fc = 0; fc <= n; ++fc)
      face_flux(f, P, dir, real(lam[dir]), &line[fc], Gm.data(), Gp.data(), nullptr, gated);
#ifdef OR_COUNT
    acc[0] += (double)(g_cnt.add - before.add);
    acc[1] += (double)(g_cnt.mul - before.mul);
    acc[2] += (double)(g_cnt.div - before.div);
    acc[3] += (double)(g_cnt.sqrt - before.sqrt);
    acc[4] += (double)(g_cnt.tanh - before.tanh);
#endif
  }
  for (int i = 0; i < 5; ++i) out[i] = acc[i];
  return nl * (n + 1);
}

int64_t or_faces_flops(const or_fluid* fl, const or_params* P, const or_grid* g, const double* W,
                       const double* lam, int dir, double* out) {
  return or_faces_flops_gated(fl, P, g, W, lam, dir, 0, out);
}

// Learned smoothness detector data. For the midpoints idx[0..n) of direction
// dir (indices over that direction's midpoint grid, n_d + 1 along d, x
// fastest): feat[30 s ..] the normalised stencil features -- for q in
// (alpha_1, alpha_2, rho, u_dir, p) over the six nodes i-2 .. i+3,
// (q_j - mean q) / (max q - min q + 1e-30) evaluated on the differences
// q_j - q_i, zero where alpha_2 does not exist --
// and dev[s] = the largest |omega_k - d_k| of the WENO-IS weights (App. C)
// over both biases and all characteristic fields of the midpoint (App. D).
void or_stencil_sample(const or_fluid* fl, const or_params* P, const or_grid* g, const double* W,
                       int dir, int64_t n, const int64_t* idx, double* feat, double* dev) {
  FluidK f = make_fluid(fl);
  const int64_t nc = ncells(g);
  int64_t ext[3] = {1, 1, 1};
  for (int d = 0; d < g->D; ++d) ext[d] = g->n[d];
  const int64_t f0 = ext[0] + (dir == 0), f1 = ext[1] + (dir == 1);
  const double dk[4] = {15.0 / 32.0, 5.0 / 32.0, 5.0 / 16.0, 1.0 / 16.0};
  for (int64_t s = 0; s < n; ++s) {
    const int64_t t = idx[s];
    const int64_t q[3] = {t % f0, (t / f0) % f1, t / (f0 * f1)};
    Cell nd[6];
    for (int j = 0; j < 6; ++j) {
      real w[OR_MAXM];
      load_node(f, g, W, dir, q, q[dir] - 3 + j, w);
      cell_from_W(f, w, nd[j]);
    }
    for (int a = 0; a < 5; ++a) {
      double v[6];
      const bool present = a >= 2 || a < f.N - 1;
      for (int j = 0; j < 6; ++j) {
        if (!present)
          v[j] = 0.0;
        else if (a < 2)
          v[j] = val(nd[j].V[sAL(f, a)]);
        else if (a == 2)
          v[j] = val(nd[j].rho);
        else if (a == 3)
          v[j] = val(nd[j].V[sMOM(f, dir)]);
        else
          v[j] = val(nd[j].V[sE(f)]);
      }
      // differences from node i first, so that a uniform stencil gives exact
      // zeros (the normalisation is invariant under the shift)
      double dq[6], mean = 0.0, lo = 0.0, hi = 0.0;
      for (int j = 0; j < 6; ++j) {
        dq[j] = v[j] - v[2];
        mean += dq[j];
        lo = dq[j] < lo ? dq[j] : lo;
        hi = dq[j] > hi ? dq[j] : hi;
      }
      mean /= 6.0;
      for (int j = 0; j < 6; ++j) feat[30 * s + 6 * a + j] = (dq[j] - mean) / ((hi - lo) + 1e-30);
    }
    real U[6][OR_MAXM], arb[OR_MAXN], rhob, cb;
    project_stencil(f, dir, nd, U, arb, rhob, cb);
    double mx = 0.0;
    for (int m = 0; m < f.M; ++m) {
      for (int side = 0; side < 2; ++side) {
        real s5[5];
        for (int j = 0; j < 5; ++j) s5[j] = side == 0 ? U[j][m] : U[5 - j][m];
        real om[4];
        weno_is_left(s5, P->weno_eps, om);
        for (int k = 0; k < 4; ++k) {
          const double d = std::fabs(val(om[k]) - dk[k]);
          if (!(d <= mx)) mx = d;  // NaN propagates
        }
      }
    }
    dev[s] = mx;
  }
}

// Linear-weight interpolation of a left-biased five-point stencil (the gated value).
double or_weno_lin(const double* u) {
  real r[5];
  for (int j = 0; j < 5; ++j) r[j] = u[j];
  return val(weno_lin_left(r));
}

// Threads the line loops use (1 unless built with -DOR_OMP -fopenmp).
int or_threads(void) {
#ifdef OR_OMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

double or_tanh(double x) { return tanh_explicit(x); }

#ifdef OR_COUNT
void or_count_reset(void) { memset(&g_cnt, 0, sizeof(g_cnt)); }
void or_count_get(unsigned long long* out) {
  out[0] = g_cnt.add;
  out[1] = g_cnt.mul;
  out[2] = g_cnt.div;
  out[3] = g_cnt.sqrt;
  out[4] = g_cnt.tanh;
}
#endif

}  // extern "C"
