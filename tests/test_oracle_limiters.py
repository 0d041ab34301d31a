"""Pins of the oracle's positivity limiters, hard switches, characteristic
projection and shock sensor against what the paper's definitions fix.

* Interpolation limiter (Sec. 4.3.2, Alg. interp_limit_densities, Alg.
  interp_limit_vol_frac, the interpolation hard switch).
* Flux limiter (Sec. 4.3.2, Alg. flux_limit_densities_vol_frac, Alg.
  flux_limit_energy, the flux hard switch).
* Characteristic decomposition (App. D): the matrix A of the quasi-linear
  primitive system and its eigen-decomposition A = R Lambda R^{-1}.
* Shock sensor (Sec. 4.3.1).

Every expected value comes from the defining equations: a limited quantity
equals min(eps, first-order value) where its theta solve acts, a hard switch
returns the first-order state or flux exactly, R^{-1} A R is diagonal with the
acoustic eigenvalues at both ends, the sensor's normalised fourth-order second
differences vanish on affine data. Each docstring names a plausible mistake in
the oracle that the test fails under; every one was planted in a copy of the
oracle and seen to fail.
"""
import numpy as np
import pytest

from paper_2208_04488_gb300 import problems as P

EPS = np.finfo(np.float64).eps


def _fluid(orc, fl, D=1):
    gamma, pinf, cv, q = P._species(fl)
    return orc.make_fluid(gamma, pinf, cv, q, D=D)


def _wa(orc, D=1):
    """The paper's water and air (Table fluid_properties)."""
    return _fluid(orc, [P.PAPER_WATER, P.PAPER_AIR], D=D)


def _wa0(orc, D=1):
    """The paper's water (with q = 0, so that a partial density does not enter
    rho e~) and air: the flux-limiter tests change one quantity at a time."""
    return _fluid(orc, [dict(P.PAPER_WATER, q=0.0), P.PAPER_AIR], D=D)


def _W(orc, f, V):
    W, _ = orc.cons_cell(f, np.asarray(V, dtype=np.float64))
    return W


def _roundoff(*vals):
    return 16 * EPS * max(abs(v) for v in vals)


# =====================================================================
# Interpolation limiter (Sec. 4.3.2)
# =====================================================================

def test_interp_density_theta_per_species(orc):
    """Alg. interp_limit_densities: a negative interpolated alpha_1 rho_1 is
    pulled to exactly min(eps, alpha_1 rho_1(W_i)) by its own theta, while an
    admissible alpha_2 rho_2, the velocity and the pressure are left as they are.

    Mutation caught: one theta shared by all species (alpha_2 rho_2 would move)."""
    f = _wa(orc)
    p = orc.make_params()
    Vn = np.array([800.0, 0.6, 5.0, 2.0e5, 0.7])
    Vt = np.array([-5.0, 0.9, 7.0, 2.5e5, 0.7])
    V, hs = orc.interp_limit(f, p, Vt, _W(orc, f, Vn))
    assert hs == 0
    target = min(p.eps_ar, Vn[0])
    assert abs(V[0] - target) <= _roundoff(Vn[0], Vt[0])
    assert V[1] == Vt[1] and V[2] == Vt[2] and V[3] == Vt[3] and V[4] == Vt[4]


def test_interp_density_target_is_the_node_value_below_eps(orc):
    """Alg. interp_limit_densities: when the node's partial density is itself
    below eps the target is that node value, min(eps, alpha_k rho_k(W_i)).

    Mutation caught: target = eps (the limited value would be eps = 1e-10, not 1e-12)."""
    f = _wa(orc)
    p = orc.make_params()
    Vn = np.array([900.0, 1e-12, 0.0, 1.0e5, 1.0 - 1e-9])
    Vt = np.array([901.0, -1e-3, 0.0, 1.0e5, 1.0 - 1e-9])
    V, hs = orc.interp_limit(f, p, Vt, _W(orc, f, Vn))
    assert hs == 0
    assert abs(V[1] - 1e-12) <= _roundoff(Vt[1], Vn[1])
    assert V[0] == Vt[0]


def test_interp_volume_fractions_one_theta_including_derived_alpha(orc):
    """Alg. interp_limit_vol_frac over k = 1..N, with alpha_N = 1 - sum of the
    others: three species, the interpolated alpha_1, alpha_2 push the derived
    alpha_3 negative. One theta limits alpha_3 to exactly min(eps, alpha_3(W_i))
    and moves alpha_1 and alpha_2 by the same convex combination.

    Mutations caught: alpha_N left out of the theta loop (no limiting at all);
    a theta per stored alpha (alpha_1, alpha_2 would not move)."""
    f = _fluid(orc, [P.PAPER_WATER, P.PAPER_AIR, P.PAPER_SF6])
    p = orc.make_params()
    # V = (a1r1, a2r2, a3r3, u, p, a1, a2)
    Vn = np.array([500.0, 0.4, 1.2, 3.0, 1.0e6, 0.5, 0.3])
    Vt = np.array([500.0, 0.4, 1.2, 3.0, 1.0e6, 0.7, 0.5])
    V, hs = orc.interp_limit(f, p, Vt, _W(orc, f, Vn))
    assert hs == 0
    a3n, a3t = 1 - Vn[5] - Vn[6], 1 - Vt[5] - Vt[6]
    a3 = 1 - V[5] - V[6]
    assert abs(a3 - min(p.eps_a, a3n)) <= _roundoff(1.0)
    th1 = (V[5] - Vn[5]) / (Vt[5] - Vn[5])
    th2 = (V[6] - Vn[6]) / (Vt[6] - Vn[6])
    th3 = (min(p.eps_a, a3n) - a3n) / (a3t - a3n)
    assert 0.0 < th3 < 1.0
    assert th1 == pytest.approx(th3, rel=1e-12) and th2 == pytest.approx(th3, rel=1e-12)
    assert np.array_equal(V[:5], Vt[:5])


def test_interp_volume_fraction_theta_is_the_smallest(orc):
    """Alg. interp_limit_vol_frac takes theta = min over k: with alpha_1 mildly
    and the derived alpha_2 strongly out of bounds, the binding one (alpha_2) is
    at its target and alpha_1 ends inside [0, 1].

    Mutation caught: the last species' theta instead of the minimum."""
    f = _wa(orc)
    p = orc.make_params()
    Vn = np.array([600.0, 0.5, 0.0, 1.0e5, 0.4])
    Vt = np.array([600.0, 0.5, 0.0, 1.0e5, 1.6])  # alpha_1 > 1, alpha_2 = -0.6
    V, hs = orc.interp_limit(f, p, Vt, _W(orc, f, Vn))
    assert hs == 0
    assert abs((1 - V[4]) - min(p.eps_a, 1 - Vn[4])) <= _roundoff(1.6)
    assert 0.0 <= V[4] <= 1.0
    # alpha_1 mildly negative, alpha_2 = 1 - alpha_1 fine: alpha_1 binds
    Vt2 = np.array([600.0, 0.5, 0.0, 1.0e5, -0.2])
    V2, _ = orc.interp_limit(f, p, Vt2, _W(orc, f, Vn))
    assert abs(V2[4] - p.eps_a) <= _roundoff(0.4)


def test_interp_hard_switch_returns_the_node_state_exactly(orc):
    """Interpolation hard switch (Sec. 4.3.2): a limited state with rho c^2 < 0
    (pressure below -pbar_inf, which the convex limiters do not touch) is
    replaced by the node's primitive state bit for bit; an admissible state is
    returned unchanged and the switch stays off.

    Mutation caught: the switch resetting only the limited entries."""
    f = _wa(orc)
    p = orc.make_params()
    Vn = np.array([800.0, 0.6, 5.0, 2.0e5, 0.7])
    Wn = _W(orc, f, Vn)
    Vnode, _ = orc.prim_cell(f, Wn)
    Vt = np.array([810.0, 0.62, 4.0, -2.0 * P.PAPER_WATER["pinf"], 0.69])
    V, hs = orc.interp_limit(f, p, Vt, Wn)
    assert hs == 1
    assert np.array_equal(V, Vnode)
    Vok = np.array([810.0, 0.62, 4.0, 2.1e5, 0.69])
    V2, hs2 = orc.interp_limit(f, p, Vok, Wn)
    assert hs2 == 0 and np.array_equal(V2, Vok)


def _rough_stencils(orc, f, count, seed):
    """Seeded six-node stencils whose partial densities, volume fractions and
    pressures jump over many orders of magnitude."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(count):
        W6 = []
        for _j in range(6):
            a1 = 10 ** rng.uniform(-12, 0) if rng.random() < 0.5 else 1 - 10 ** rng.uniform(-12, -0.3)
            ar1 = a1 * 10 ** rng.uniform(-3, 3.2)
            ar2 = (1 - a1) * 10 ** rng.uniform(-4, 1.5)
            W6.append(_W(orc, f, [ar1, ar2, rng.normal(0, 300), 10 ** rng.uniform(3, 9.5), a1]))
        out.append(np.array(W6))
    return out


def test_interp_limiter_sides_use_their_own_node(orc):
    """Sec. 4.3.2: the left-biased midpoint state is limited towards (and hard-
    switched to) V_i, the right-biased one towards V_{i+1}. On seeded rough
    stencils, where both limiters and both hard switches fire, each side of the
    face equals the limiter applied to its WENO value with its own node, and a
    hard-switched side equals that node's V exactly.

    Mutation caught: the right-biased state limited with node i."""
    f = _wa(orc)
    p = orc.make_params()
    fired = {"hsL": 0, "hsR": 0, "L": 0, "R": 0}
    for W6 in _rough_stencils(orc, f, 600, seed=3):
        _, _, d = orc.face(f, p, 0, 1e-4, W6)
        VL, hsL = orc.interp_limit(f, p, d["VL_weno"], W6[2])
        VR, hsR = orc.interp_limit(f, p, d["VR_weno"], W6[3])
        assert np.array_equal(VL, d["VL"]) and hsL == d["hsL"]
        assert np.array_equal(VR, d["VR"]) and hsR == d["hsR"]
        if hsL:
            assert np.array_equal(d["VL"], orc.prim_cell(f, W6[2])[0])
        if hsR:
            assert np.array_equal(d["VR"], orc.prim_cell(f, W6[3])[0])
        fired["hsL"] += hsL
        fired["hsR"] += hsR
        fired["L"] += (not hsL) and not np.array_equal(d["VL"], d["VL_weno"])
        fired["R"] += (not hsR) and not np.array_equal(d["VR"], d["VR_weno"])
    assert min(fired.values()) >= 5, fired


# =====================================================================
# Flux limiter (Sec. 4.3.2)
# =====================================================================

LAM = 1.0e-3  # lambda = dt/dx [s/m]


def _flux_setup(orc, f, Vi, Vj, dir_=0):
    """W_i, W_{i+1} and their physical fluxes F_i, F_{i+1} (Eq. F_x_F_y_def,
    zero in the alpha slots). Passing G^HLLC = F makes the first-order
    half-cell states the node states themselves."""
    N, D = f.N, f.D

    def F(W):
        V, _ = orc.prim_cell(f, W)
        un, pr = V[N + dir_], V[N + D]
        out = np.zeros(W.size)
        out[:N + D] = W[:N + D] * un
        out[N + dir_] += pr
        out[N + D] = (W[N + D] + pr) * un
        return out

    Wi, Wj = _W(orc, f, Vi), _W(orc, f, Vj)
    return Wi, Wj, F(Wi), F(Wj)


def _half(W, G, F, sgn):
    """W_i^{+} = W_i - 2 lam (G^- - F_i) (sgn -1); W_{i+1}^{-} = W_{i+1} + 2 lam (G^+ - F_{i+1}) (sgn +1)."""
    return W + sgn * 2.0 * LAM * (G - F)


def _thetas(Gout, Gin, H):
    """theta of every component where the convex combination (1-theta) H + theta G is defined."""
    m = np.abs(Gin - H) > 1e-9 * (np.abs(Gin) + np.abs(H) + 1e-300)
    return (Gout[m] - H[m]) / (Gin[m] - H[m])


def test_flux_limit_noop_on_admissible_half_states(orc):
    """Alg. flux_limit_densities_vol_frac and flux_limit_energy with every
    half-cell state admissible: theta = 1 in both stages, no hard switch, the
    fluxes come back bit for bit."""
    f = _wa0(orc)
    p = orc.make_params()
    Wi, Wj, Fi, Fj = _flux_setup(orc, f, [800.0, 0.6, 0.0, 2e5, 0.7], [700.0, 0.7, 0.0, 1.5e5, 0.6])
    Gm, Gp = Fi + 0.01 * np.abs(Fi + 1), Fj - 0.01 * np.abs(Fj + 1)
    gm, gp, flags = orc.flux_limit(f, p, 0, LAM, Wi, Wj, Gm, Gp, Fi, Fj)
    assert flags == 0
    assert np.array_equal(gm, Gm) and np.array_equal(gp, Gp)


def test_flux_limit_density_stage_one_theta_both_sides(orc):
    """Alg. flux_limit_densities_vol_frac: G^- drives alpha_1 rho_1 of W_i^{+}
    negative. One theta, taken for all components and for both G^- and G^+,
    brings alpha_1 rho_1(W_i^{*,+}) to exactly min(eps, alpha_1 rho_1(W_i^{HLLC,+}))
    (Sec. 4.3.2, the convex combination G^* = (1-theta) G^HLLC + theta G).

    Mutations caught: target = eps where the first-order value is smaller
    (second case); separate thetas for G^- and G^+."""
    f = _wa0(orc)
    p = orc.make_params()
    for ar1_i in (800.0, 3e-11):
        Wi, Wj, Fi, Fj = _flux_setup(orc, f, [ar1_i, 0.6, 0.0, 2e5, 0.7], [700.0, 0.7, 0.0, 1.5e5, 0.6])
        Gm = Fi.copy()
        Gm[0] += (Wi[0] + 5.0) / (2 * LAM)  # W_i^{+} alpha_1 rho_1 = -5
        Gp = Fj.copy()
        Gp[1] += 10.0  # harmless change on the other side
        gm, gp, flags = orc.flux_limit(f, p, 0, LAM, Wi, Wj, Gm, Gp, Fi, Fj)
        assert flags == 1
        Wp = _half(Wi, gm, Fi, -1)
        assert abs(Wp[0] - min(p.eps_ar, Wi[0])) <= _roundoff(Wi[0], 5.0)
        th = np.concatenate([_thetas(gm, Gm, Fi), _thetas(gp, Gp, Fj)])
        assert th.size >= 2 and np.allclose(th, th[0], rtol=1e-12, atol=0)


def test_flux_limit_volume_fraction_of_the_right_cell(orc):
    """Alg. flux_limit_densities_vol_frac, volume-fraction branch on the cell
    i+1 side (the theta^{alpha_k,-} solve; read for the garbled "theta^-"): G^+
    pushes alpha_1(W_{i+1}^{-}) above 1, i.e. the derived alpha_2 below 0, and
    theta brings alpha_2(W_{i+1}^{*,-}) to exactly min(eps, alpha_2(W_{i+1}^{HLLC,-})).

    Mutation caught: the minus-side alpha theta ignored."""
    f = _wa0(orc)
    p = orc.make_params()
    Wi, Wj, Fi, Fj = _flux_setup(orc, f, [800.0, 0.6, 0.0, 2e5, 0.7], [700.0, 0.7, 0.0, 1.5e5, 0.6])
    Gp = Fj.copy()
    Gp[4] += (1.3 - Wj[4]) / (2 * LAM)  # alpha_1(W_{i+1}^-) = 1.3
    gm, gp, flags = orc.flux_limit(f, p, 0, LAM, Wi, Wj, Fi.copy(), Gp, Fi, Fj)
    assert flags == 1
    Wm = _half(Wj, gp, Fj, +1)
    assert abs((1.0 - Wm[4]) - min(p.eps_a, 1.0 - Wj[4])) <= _roundoff(1.3)


def test_flux_limit_energy_stage_reads_the_stage_one_state(orc):
    """Alg. flux_limit_energy after Alg. flux_limit_densities_vol_frac: G^-
    makes both alpha_2 rho_2 and rho e~ of W_i^{+} negative. Stage one limits
    the density; the energy theta is then solved on W_i^{*,+} (the state of the
    stage-one flux), so rho e~(W_i^{**,+}) equals min(eps_rhoe, rho e~(W_i^{HLLC,+}))
    to round-off (u = 0: rho e~ is affine along the combination). The state is
    air at 10 Pa, so the round-off of E is far below eps_rhoe.

    Mutation caught: the energy theta solved on the unlimited W_i^{+}."""
    f = _wa0(orc)
    p = orc.make_params()
    Vi = [1e-9, 1.2e-4, 0.0, 10.0, 1e-12]
    Wi, Wj, Fi, Fj = _flux_setup(orc, f, Vi, [1e-9, 1.0e-4, 0.0, 8.0, 1e-12])
    Gm = Fi.copy()
    Gm[1] += (Wi[1] + 1e-3) / (2 * LAM)  # alpha_2 rho_2(W_i^+) = -1e-3
    Gm[3] += (Wi[3] + 20.0 * Wi[3]) / (2 * LAM)  # rho e~(W_i^+) = -20 E_i
    gm, gp, flags = orc.flux_limit(f, p, 0, LAM, Wi, Wj, Gm, Fj.copy(), Fi, Fj)
    assert flags == 3
    Wss = _half(Wi, gm, Fi, -1)
    _, info = orc.prim_cell(f, Wss)
    _, infoH = orc.prim_cell(f, Wi)
    assert abs(info["rhoe"] - min(p.eps_rhoe, infoH["rhoe"])) <= _roundoff(Wi[3], 20.0 * Wi[3])
    assert Wss[1] >= min(p.eps_ar, Wi[1]) * (1 - 1e-6)


def test_flux_limit_energy_includes_kinetic_energy(orc):
    """Alg. flux_limit_energy limits rho e~ = E - |rho u|^2/(2 rho) - sum alpha_k
    rho_k q_k, not E: with u != 0 and only the energy flux changed, rho e~ of
    W_i^{**,+} is min(eps_rhoe, rho e~(W_i^{HLLC,+})) to round-off.

    Mutation caught: the kinetic term dropped from rho e~."""
    f = _wa0(orc)
    p = orc.make_params()
    Wi, Wj, Fi, Fj = _flux_setup(orc, f, [1e-9, 1.2e-4, 40.0, 10.0, 1e-12], [1e-9, 1.0e-4, 40.0, 8.0, 1e-12])
    _, infoH = orc.prim_cell(f, Wi)
    Gm = Fi.copy()
    Gm[3] += (infoH["rhoe"] + 30.0) / (2 * LAM)  # rho e~(W_i^+) = -30
    gm, _, flags = orc.flux_limit(f, p, 0, LAM, Wi, Wj, Gm, Fj.copy(), Fi, Fj)
    assert flags == 2
    _, info = orc.prim_cell(f, _half(Wi, gm, Fi, -1))
    assert abs(info["rhoe"] - min(p.eps_rhoe, infoH["rhoe"])) <= _roundoff(Wi[3], 30.0)


def test_flux_hard_switch_replaces_both_fluxes_exactly(orc):
    """Flux hard switch (Sec. 4.3.2): when W_{i+1}^{**,-} alone fails a hard-
    switch test, both G^{**,-} and G^{**,+} become the first-order HLLC fluxes
    bit for bit. The test raises the volume-fraction hard-switch tolerance to
    0.5 so the limited alpha_2 = eps fails it.

    Mutations caught: only the failing side replaced; the minus side's tests
    left out."""
    f = _wa0(orc)
    p = orc.make_params(hs_a=0.5)
    Wi, Wj, Fi, Fj = _flux_setup(orc, f, [800.0, 0.6, 0.0, 2e5, 0.7], [700.0, 0.7, 0.0, 1.5e5, 0.6])
    Gp = Fj.copy()
    Gp[4] += (1.3 - Wj[4]) / (2 * LAM)
    Gm = Fi.copy()
    Gm[1] += 3.0
    Hm, Hp = Fi + 1.0, Fj + 2.0  # first-order fluxes, distinct from both inputs
    Hm[4] = Fi[4]
    Hp[4] = Fj[4]
    gm, gp, flags = orc.flux_limit(f, p, 0, LAM, Wi, Wj, Gm, Gp, Hm, Hp)
    assert flags & 4
    assert np.array_equal(gm, Hm) and np.array_equal(gp, Hp)


# =====================================================================
# Characteristic decomposition (App. D)
# =====================================================================

def _A(f, dir_, arb, rho, c, u):
    """The matrix of the quasi-linear primitive system in direction dir_
    (App. D, A for x and B for y; z alike), at the averaged state."""
    N, D = f.N, f.D
    M = 2 * N + D
    un, sp = N + dir_, N + D
    A = u * np.eye(M)
    A[:N, un] = arb
    A[un, sp] = 1.0 / rho
    A[sp, un] = rho * c * c
    return A


@pytest.mark.parametrize("N,D", [(2, 1), (2, 2), (3, 2), (3, 3)])
def test_projection_diagonalises_the_primitive_system(orc, N, D):
    """App. D: at the averages of the partial densities, mixture density and
    sound speed of nodes i and i+1, R^{-1} A R = diag(u - c, u, ..., u, u + c)
    and R R^{-1} = R^{-1} R = I, in every direction; the averages are the
    arithmetic means of alpha_k rho_k, rho and c (not of c^2).

    Mutations caught: a sign flip in one entry of R; the averaged c taken
    from the mean of c^2; tangential velocities out of order."""
    fl = [P.PAPER_WATER, P.PAPER_AIR, P.PAPER_SF6][:N]
    f = _fluid(orc, fl, D=D)
    prim, _ = P.random_admissible_states(N, D, 24, seed=100 + 10 * N + D, fluids=fl)
    W = orc.ic_from_prim(f, prim)
    M = 2 * N + D
    for s in range(0, W.shape[1], 2):
        Wi, Wj = W[:, s].copy(), W[:, s + 1].copy()
        Vi, ii = orc.prim_cell(f, Wi)
        Vj, ij = orc.prim_cell(f, Wj)
        arb = 0.5 * (Vi[:N] + Vj[:N])
        rho = 0.5 * (ii["rho"] + ij["rho"])
        c = 0.5 * (ii["c"] + ij["c"])
        for dir_ in range(D):
            Rinv, R, avg = orc.char_matrices(f, dir_, Wi, Wj)
            np.testing.assert_allclose(avg[:N], arb, rtol=1e-15)
            assert avg[N] == pytest.approx(rho, rel=1e-15)
            assert avg[N + 1] == pytest.approx(c, rel=1e-15)
            u = 0.5 * (Vi[N + dir_] + Vj[N + dir_])
            Lam = Rinv @ _A(f, dir_, avg[:N], avg[N], avg[N + 1], u) @ R
            expect = np.full(M, u)
            expect[0], expect[-1] = u - c, u + c
            scale = abs(u) + c
            np.testing.assert_allclose(np.diag(Lam), expect, rtol=0, atol=1e-12 * scale)
            assert np.abs(Lam - np.diag(np.diag(Lam))).max() <= 1e-9 * scale * max(1.0, avg[N] * c)
            I = np.eye(M)
            np.testing.assert_allclose(R @ Rinv, I, rtol=0, atol=1e-12)
            np.testing.assert_allclose(Rinv @ R, I, rtol=0, atol=1e-12)


def test_projection_round_trip_on_a_constant_stencil(orc):
    """App. D with App. C: on a constant stencil the WENO values of the
    characteristic fields equal the node value, so V~_L = V~_R = R R^{-1} V_i
    reproduces V_i to round-off (and the face flux is the physical flux)."""
    f = _fluid(orc, [P.PAPER_WATER, P.PAPER_AIR, P.PAPER_SF6], D=2)
    prim, _ = P.random_admissible_states(3, 2, 6, seed=41, fluids=[P.PAPER_WATER, P.PAPER_AIR, P.PAPER_SF6])
    W = orc.ic_from_prim(f, prim)
    p = orc.make_params()
    for s in range(W.shape[1]):
        W6 = np.repeat(W[:, s][None, :], 6, axis=0)
        V, _ = orc.prim_cell(f, W[:, s])
        for dir_ in (0, 1):
            _, _, d = orc.face(f, p, dir_, 1e-4, W6)
            np.testing.assert_allclose(d["VL_weno"], V, rtol=1e-12, atol=1e-12 * np.abs(V).max())
            np.testing.assert_allclose(d["VR_weno"], V, rtol=1e-12, atol=1e-12 * np.abs(V).max())


# =====================================================================
# Shock sensor (Sec. 4.3.1)
# =====================================================================

def test_sensor_bounded_for_positive_data(orc):
    """Sec. 4.3.1: for positive data each normalised second difference has
    |numerator| <= denominator (triangle inequality), so sigma lies in [0, 1]."""
    rng = np.random.default_rng(9)
    for _ in range(3000):
        u = 10 ** rng.uniform(-6, 9, size=6)
        s = orc.sensor(u)
        assert 0.0 <= s <= 1.0


def test_sensor_vanishes_on_affine_data(orc):
    """Sec. 4.3.1: -u_{j-2} + 16 u_{j-1} - 30 u_j + 16 u_{j+1} - u_{j+2} is a
    fourth-order second difference and is exactly 0 on affine data (exact
    integer arithmetic here).

    Mutation caught: a wrong coefficient (e.g. 32 for 30)."""
    for a, b in ((3.0, 2.0), (1000.0, -7.0), (5.0, 0.0)):
        u = np.array([a + b * j for j in range(-2, 4)])
        assert orc.sensor(u) == 0.0


def test_sensor_mirror_symmetry_and_stencil_extent(orc):
    """Sec. 4.3.1: sigma(u) = (sigma^+ + sigma^-)/2 with sigma^+ on nodes
    i-1..i+3 and sigma^- on i-2..i+2. Mirroring the six nodes maps sigma^+ to
    sigma^-, so sigma is mirror-invariant; a spike at node i-2 enters only
    sigma^- and one at i+3 only sigma^+, with equal values.

    Mutation caught: both halves on the same five nodes (a spike at i+3 would
    give 0)."""
    rng = np.random.default_rng(17)
    for _ in range(200):
        u = 10 ** rng.uniform(0, 6, size=6)
        assert orc.sensor(u[::-1].copy()) == pytest.approx(orc.sensor(u), rel=1e-13)
    lo = np.array([2.0, 1, 1, 1, 1, 1])
    hi = lo[::-1].copy()
    assert orc.sensor(lo) > 0.0
    assert orc.sensor(lo) == orc.sensor(hi)
    # a spike at an interior node enters both halves: more than at an end node
    mid = np.array([1.0, 1, 2.0, 1, 1, 1])
    assert orc.sensor(mid) > orc.sensor(lo)


def test_sensor_blend_factor_at_shock_and_contact(orc):
    """Sec. 4.3.1, Eqs. flux_blending and velocity_blending: at a joint jump
    of rho and p (a shock) sigma^s = tanh(C_s [sigma(rho) sigma(p)]^q) is 1 and
    the blended flux is the second-order G~ exactly; across a contact with
    uniform pressure sigma(p) is round-off, so sigma^s is negligible (the HCS
    flux is used).

    Mutation caught: q = 1 (sigma^s ~ 1e-5 at the contact)."""
    f = _wa(orc)
    p = orc.make_params(limiters=0)
    left = _W(orc, f, [1.0e-8, 1.2, 0.0, 1.0e5, 1e-8])
    right = _W(orc, f, [1.0e-8, 5.0, 300.0, 8.0e5, 1e-8])
    W6 = np.array([left, left, left, right, right, right])
    Gm, Gp, d = orc.face(f, p, 0, 1e-4, W6)
    assert d["sig"] == 1.0
    assert np.array_equal(Gm[:4], d["Gt"][:4])
    # contact: water | air at equal pressure and velocity
    a = _W(orc, f, [1000.0 * (1 - 1e-8), 1.2e-8, 10.0, 1.0e5, 1 - 1e-8])
    b = _W(orc, f, [1000.0 * 1e-8, 1.2 * (1 - 1e-8), 10.0, 1.0e5, 1e-8])
    W6 = np.array([a, a, a, b, b, b])
    _, _, d = orc.face(f, p, 0, 1e-4, W6)
    assert d["sig"] < 1e-12
