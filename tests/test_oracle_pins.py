"""Pins of the CPU oracle against what the paper and the mathematics fix.

Each test names the passage it follows. None of them compares the oracle with
itself or with the CUDA path: the expected values are the paper's printed
numbers, closed forms, textbook results or invariants.
"""
import math

import numpy as np
import pytest

from paper_2208_04488_gb300 import problems as P
from tests import exact_riemann as ER


def _fluid(orc, fl, D=1):
    gamma, pinf, cv, q = P._species(fl)
    return orc.make_fluid(gamma, pinf, cv, q, D=D)


def _W_from_prim(orc, f, prim_cols):
    prim = np.asarray(prim_cols, dtype=np.float64)
    if prim.ndim == 1:
        prim = prim[:, None]
    return orc.ic_from_prim(f, prim)


# ---------------------------------------------------------------- initial-condition tables

def test_ic_table_temporal_convergence(orc):
    """Table exact_1D_convergence (Sec. 5.1): rho_1, rho_2 at 101325 Pa, 298 K."""
    f = _fluid(orc, [P.PAPER_WATER, P.PAPER_AIR])
    W = _W_from_prim(orc, f, [0.5, 0.0, 101325.0, 298.0])
    assert W[0, 0] / 0.5 == pytest.approx(1022.7724412751677, rel=1e-15)
    assert W[1, 0] / 0.5 == pytest.approx(1.1817862212832324, rel=1e-15)


def test_ic_table_shock_tubes(orc):
    """Tables IC_1D_gas_liquid_shock_tube_problem and IC_1D_extreme_... (Sec. 5.4, 5.5)."""
    for extreme, ar2_left in ((False, 5.2511071660640894e-5), (True, 9.7235797802400965e-5)):
        pr = P.shock_tube_1d_paper(n=100, extreme=extreme)
        f, g, W = orc.setup(pr)
        assert W[0, 0] == pytest.approx(9.9999998999999991e2, rel=1e-15)
        assert W[1, 0] == pytest.approx(ar2_left, rel=2e-9)
        assert W[0, -1] == pytest.approx(1.7538240816326533e-4, rel=1e-14)
        assert W[1, -1] == pytest.approx(1.9999999799999998e1, rel=1e-15)
    pr = P.shock_tube_1d_paper(n=100)
    # temperatures quoted in the text (Sec. 5.4, Sec. 5.5)
    assert pr.extra["TL"] == pytest.approx(661.89, abs=0.005)
    assert pr.extra["TR"] == pytest.approx(17.378, abs=0.0005)
    assert P.shock_tube_1d_paper(n=10, extreme=True).extra["TL"] == pytest.approx(357448, abs=0.5)


def test_ic_table_three_species_and_cylinder(orc):
    """Tables IC_1D_extreme_shock_interface_interaction (Sec. 5.6) and
    IC_2D_shock_water_cylinder (Sec. 5.7), rows at 101325 Pa and 298 K."""
    f3 = _fluid(orc, [P.PAPER_WATER, P.PAPER_AIR, P.PAPER_SF6])
    # 0.15 <= x < 0.3: water with minor air and SF6
    W = _W_from_prim(orc, f3, [1 - 2e-8, 1e-8, 0.0, 1.01325e5, 298.0])
    assert W[0, 0] == pytest.approx(1.0227724208197188e3, rel=1e-14)
    assert W[1, 0] == pytest.approx(1.1817862212832324e-8, rel=1e-14)
    assert W[2, 0] == pytest.approx(5.6328080779493768e-8, rel=1e-14)
    # x >= 0.3: air/SF6 mixture
    W = _W_from_prim(orc, f3, [1e-8, 0.5 - 5e-9, 0.0, 1.01325e5, 298.0])
    assert W[0, 0] == pytest.approx(1.0227724412751677e-5, rel=1e-14)
    assert W[1, 0] == pytest.approx(0.59089310473268508, rel=1e-14)
    assert W[2, 0] == pytest.approx(2.8164040108106478, rel=1e-14)
    f2 = _fluid(orc, [P.PAPER_WATER, P.PAPER_AIR], D=2)
    W = _W_from_prim(orc, f2, [1e-8, 0.0, 0.0, 1.01325e5, 298.0])  # pre-shock air
    assert W[0, 0] == pytest.approx(1.0227724412751677e-5, rel=1e-14)
    assert W[1, 0] == pytest.approx(1.1817862094653702, rel=1e-14)
    W = _W_from_prim(orc, f2, [1 - 1e-8, 0.0, 0.0, 1.01325e5, 298.0])  # water cylinder
    assert W[0, 0] == pytest.approx(1.0227724310474432e3, rel=1e-14)
    assert W[1, 0] == pytest.approx(1.1817862212832324e-8, rel=1e-7)
    # acoustic problem, x >= -0.5 (Table IC_1D_acoustic_wave_propagation_problem):
    # its air column matches the fluid table at 101325 Pa, 298 K; its water
    # column (684.46 = 0.5 x 1368.92) does not, so only the air entry is a pin.
    f1 = _fluid(orc, [P.PAPER_WATER, P.PAPER_AIR])
    W = _W_from_prim(orc, f1, [0.5, 0.0, 101325.0, 298.0])
    assert W[1, 0] == pytest.approx(0.5908931106416162, rel=1e-14)


def test_ic_table_material_interface(orc):
    """Table IC_1D_material_interface_advection_no_temp_diff (App. A)."""
    pr = P.material_interface_1d(n=100)
    f, g, W = orc.setup(pr)
    mid = 50
    assert W[0, mid] == pytest.approx(1.0227724310474432e3, rel=1e-14)
    assert W[1, mid] == pytest.approx(1.1817862272214237e-8, rel=1e-7)
    assert W[0, 0] == pytest.approx(1.0227724412751677e-5, rel=1e-14)
    assert W[1, 0] == pytest.approx(1.1817862094653702, rel=1e-14)
    assert W[2, 0] / (W[0, 0] + W[1, 0]) == pytest.approx(100.0, rel=1e-14)


# ---------------------------------------------------------------- sound speeds

def test_sound_speeds_water_air(orc):
    """Sec. 5.3: at alpha = 0.5 (101325 Pa, 298 K) the five-equation sound
    speed is 913.05 m/s and the four-equation HRM one 19.897 m/s; the HRM
    sound speed at alpha_1 = 1e-8 is c_ref = 346.46 m/s."""
    f = _fluid(orc, [P.PAPER_WATER, P.PAPER_AIR])
    W = _W_from_prim(orc, f, [0.5, 0.0, 101325.0, 298.0])[:, 0]
    V, o = orc.prim_cell(f, W)
    assert o["c"] == pytest.approx(913.05, abs=0.005)
    c4 = orc.c4eq_cell(f, W)
    assert c4["c4"] == pytest.approx(19.897, abs=0.0005)
    assert c4["p"] == pytest.approx(101325.0, rel=1e-12)
    assert c4["T"] == pytest.approx(298.0, rel=1e-12)
    W = _W_from_prim(orc, f, [1e-8, 0.0, 101325.0, 298.0])[:, 0]
    assert orc.c4eq_cell(f, W)["c4"] == pytest.approx(346.46, abs=0.005)


def test_c4eq_matches_finite_differences(orc):
    """Eq. 4_eqn_sos with Psi_k and Gamma from the implicit derivative of the
    p* quadratic equals central finite differences of the relaxed pressure
    p(alpha_k rho_k, e) (Sec. 3 definitions of Psi_k and Gamma)."""
    f = _fluid(orc, [P.BENCH_WATER, P.BENCH_AIR, P.BENCH_HELIUM])
    prim, _ = P.random_admissible_states(3, 1, 20, seed=7)
    W = orc.ic_from_prim(f, prim)
    for c in range(W.shape[1]):
        w = W[:, c].copy()
        res = orc.c4eq_cell(f, w)
        rho = w[:3].sum()
        e = (w[4] - 0.5 * w[3] ** 2 / rho) / rho  # specific internal energy (q = 0)

        def p_of(ar, e_):
            ww = w.copy()
            ww[:3] = ar
            r = ar.sum()
            ww[3] = r * (w[3] / rho)
            ww[4] = r * e_ + 0.5 * ww[3] ** 2 / r
            return orc.relax_cell(f, ww)[1]

        # central differences over a range of steps; the best one (truncation vs
        # round-off) must agree to 1e-6
        for k in range(3):
            errs = []
            for rel in (1e-2, 1e-3, 1e-4, 1e-5, 1e-6):
                h = rel * min(w[k], rho)
                ap, am = w[:3].copy(), w[:3].copy()
                ap[k] += h
                am[k] -= h
                fd = (p_of(ap, e) - p_of(am, e)) / (2 * h)
                errs.append(abs(fd / res["Psi"][k] - 1.0))
            assert errs and min(errs) < 1e-6, (k, errs)
        errs = []
        for rel in (1e-3, 1e-4, 1e-5, 1e-6):
            he = rel * e
            fdG = (p_of(w[:3], e + he) - p_of(w[:3], e - he)) / (2 * he) / rho
            errs.append(abs(fdG / res["Gamma"] - 1.0))
        assert min(errs) < 1e-6


# ---------------------------------------------------------------- WENO-IS (App. C)

def test_weno_linear_and_quadratic_exact(orc):
    """Linear and quadratic data have tau_5 = 0, so the weights are the linear
    d_k and the scheme returns the 5-point interpolant: exact at x_{i+1/2}."""
    x = np.arange(-2, 3, dtype=float)
    for coef in ([0.0, 2.0, 1.5], [3.0, -1.0, 0.0], [1.0, 0.0, 0.0]):
        u = coef[0] * x ** 2 + coef[1] * x + coef[2]
        v, om = orc.weno_left(u)
        exact = coef[0] * 0.25 + coef[1] * 0.5 + coef[2]
        assert v == pytest.approx(exact, rel=1e-14, abs=1e-14)
        np.testing.assert_allclose(om, [15 / 32, 5 / 32, 5 / 16, 1 / 16], rtol=1e-14)


def test_weno_linear_weights_form_lagrange_interpolant(orc):
    """sum_k d_k u^k equals the 5-point Lagrange interpolant at x_{i+1/2}
    (weights computed here by solving the Vandermonde system)."""
    nodes = np.arange(-2, 3, dtype=float)
    A = np.vander(nodes, 5, increasing=True).T
    lag = np.linalg.solve(A, 0.5 ** np.arange(5))
    np.testing.assert_allclose(lag, np.array([3, -20, 90, 60, -5]) / 128.0, atol=1e-14)
    u = np.array([1.0, 2.0, 4.0, 8.0, 16.0])
    # a constant offset of u (tau_5 changes only through differences) keeps this exact
    v_lin = float(lag @ u)
    # huge eps -> eta_k = d_k (tau_5 / eps ~ 1e-48); the weights are formed as
    # products of five (beta + eps), so eps stays below ~1e61 (no overflow)
    v, _ = orc.weno_left(u, eps=1e50)
    assert v == pytest.approx(v_lin, rel=1e-14)


def test_weno_fifth_order_on_smooth_data(orc):
    """Interpolation error of sin(x + 0.3) at x_{i+1/2} decreases as h^5 (App. C)."""
    errs = []
    for h in (0.2, 0.1, 0.05, 0.025):
        xs = np.arange(-2, 3) * h
        u = np.sin(xs + 0.3)
        v, _ = orc.weno_left(u)
        errs.append(abs(v - math.sin(0.5 * h + 0.3)))
    rates = [math.log2(errs[i] / errs[i + 1]) for i in range(3)]
    assert min(rates) > 4.6, (errs, rates)


def test_weno_essentially_non_oscillatory_at_jump(orc):
    """A jump between x_i and x_{i+1}: the left-biased value stays on the
    smooth side (the stencils S1, S3 that avoid the jump carry the weight)."""
    v, om = orc.weno_left([0.0, 0.0, 0.0, 1.0, 1.0])
    assert abs(v) < 1e-12
    assert om[1] + om[3] > 1 - 1e-12


# ---------------------------------------------------------------- HLLC (Sec. 4.1.1)

def _two_species_V(orc, f, a1, u, p, T, v=None):
    cols = [a1, u] + ([v] if v is not None else []) + [p, T]
    W = _W_from_prim(orc, f, cols)[:, 0]
    V, o = orc.prim_cell(f, W)
    return W, V, o


def test_hllc_equal_states_give_physical_flux(orc):
    f = _fluid(orc, [P.PAPER_WATER, P.PAPER_AIR], D=2)
    W, V, o = _two_species_V(orc, f, 0.3, 55.0, 2.0e5, 310.0, v=-12.0)
    for d in (0, 1):
        G, s = orc.hllc(f, d, V, V)
        un = V[2 + d]
        p = V[4]
        expect = np.array([W[0] * un, W[1] * un, W[2] * un, W[3] * un, (W[4] + p) * un,
                           V[5] * un])
        expect[2 + d] += p
        np.testing.assert_allclose(G, expect, rtol=1e-13, atol=1e-9)
        assert s == pytest.approx(un, rel=1e-13)


def test_uniform_stencil_face_is_the_physical_flux(orc):
    """App. C, Sec. 4.1.1, Eqs. reconstructed_G and G_pm, Sec. 4.3.2: a midpoint whose
    six node states are equal, evaluated step by step (projection, WENO-IS, both
    positivity limiters, two HLLC solves, HCS, sensor blend and flux limiter -- the
    single-face entry point always evaluates them all), returns the node's physical
    flux F^d in the conservative slots and zero in the alpha slots of both G^- and
    G^+, to rounding. The grid sweeps take that flux directly at bit-identical
    stencils; this pins the shortcut to the full evaluation."""
    params = orc.make_params()
    for fl, D, seed in (([P.BENCH_WATER, P.BENCH_AIR, P.BENCH_HELIUM], 2, 5),
                        ([P.PAPER_WATER, P.PAPER_AIR], 3, 6)):
        N = len(fl)
        f = _fluid(orc, fl, D=D)
        prim, _ = P.random_admissible_states(N, D, 24, seed=seed, fluids=fl)
        W = orc.ic_from_prim(f, prim)
        worst = 0.0
        for c in range(W.shape[1]):
            Wn = W[:, c]
            V, o = orc.prim_cell(f, Wn)
            p = V[N + D]
            for d in range(D):
                un = V[N + d]
                a = abs(un) + o["c"]
                lam = 0.4 / a
                Gm, Gp, _ = orc.face(f, params, d, lam, np.stack([Wn] * 6))
                F = np.zeros_like(Wn)
                F[:N + D + 1] = Wn[:N + D + 1] * un
                F[N + d] += p
                F[N + D] += p * un
                rho = Wn[:N].sum()
                scale = np.concatenate([Wn[:N] * a, np.full(D, rho * a * a + p),
                                        [(abs(Wn[N + D]) + p) * a], np.full(N - 1, a)])
                for G in (Gm, Gp):
                    err = np.abs(G - F) / scale
                    worst = max(worst, err.max())
        assert worst < 1e-12, worst


def test_grid_sweep_matches_the_full_face_evaluation(orc):
    """Eq. semi_W_G_pm_eqn: the grid right-hand side, whose sweep takes the physical
    flux directly at bit-identical stencils, equals -(G^-_{i+1/2} - G^+_{i-1/2}) / dx
    assembled from the single-face entry point (every step evaluated) to rounding.
    On the gas/liquid shock tube after a step the uniform regions on both sides of
    the waves meet non-uniform stencils, so cells with one face of each kind are
    checked too."""
    pr = P.shock_tube_1d_paper(120)
    f, g, W = orc.setup(pr)
    p = orc.make_params()
    dt, _ = orc.dt(f, g, W, 0.4)
    W = orc.step(f, p, g, W, dt, 1)
    lam = dt / g.dx[0]
    R = orc.rhs(f, p, g, W, [lam])
    n, N, D = W.shape[1], f.N, 1
    Gm, Gp, uni = {}, {}, {}
    for fc in range(3, n - 2):  # face fc lies between cells fc-1 and fc
        W6 = np.ascontiguousarray(W[:, fc - 3:fc + 3].T)
        Gm[fc], Gp[fc], _ = orc.face(f, p, 0, lam, W6)
        uni[fc] = bool((W6 == W6[2]).all())
    mixed = 0
    for i in range(3, n - 3):
        Rf = -(Gm[i + 1] - Gp[i]) / g.dx[0]
        Vc, o = orc.prim_cell(f, W[:, i])
        a = abs(Vc[N]) + o["c"]
        pc, rho = Vc[N + D], W[:N, i].sum()
        scale = np.concatenate([np.full(N, rho * a), np.full(D, rho * a * a + pc),
                                [(abs(W[N + D, i]) + pc) * a], np.full(N - 1, a)]) / g.dx[0]
        assert (np.abs(R[:, i] - Rf) <= 1e-12 * scale).all(), (i, (R[:, i] - Rf) / scale)
        mixed += uni[i] != uni[i + 1]
    assert sum(uni.values()) > 20 and mixed >= 2, (sum(uni.values()), mixed)


def test_grid_sweep_matches_the_full_face_evaluation_2d(orc):
    """As above in 2D, where each direction's flux takes that direction's velocity and
    puts p in that direction's momentum slot: on the three-species shock-bubble after
    one step (128 x 64), the grid right-hand side of every cell three cells from the sides equals
    -sum_d (G^-_{d,+1/2} - G^+_{d,-1/2}) / dx_d assembled from fully evaluated faces of
    both directions, with uniform and non-uniform stencils meeting in both."""
    pr = P.shock_bubble_2d(128, 64)
    f, g, W = orc.setup(pr)
    p = orc.make_params()
    dt, _ = orc.dt(f, g, W, pr.cfl)
    W = orc.step(f, p, g, W, dt, 1)
    lam = orc.lambdas(f, g, W, dt)
    R = orc.rhs(f, p, g, W, lam)
    nx, ny = pr.n
    N, D = f.N, 2

    faces = {}

    def face(d, i, j):  # face between cells (i-1, j) and (i, j) for d = 0, (i, j-1) and (i, j) for d = 1
        if (d, i, j) not in faces:
            idx = [j * nx + (i + k) for k in range(-3, 3)] if d == 0 else [(j + k) * nx + i for k in range(-3, 3)]
            W6 = np.ascontiguousarray(W[:, idx].T)
            Gm, Gp, _ = orc.face(f, p, d, lam[d], W6)
            faces[(d, i, j)] = (Gm, Gp, bool((W6 == W6[2]).all()))
        return faces[(d, i, j)]

    mixed = [0, 0]
    uniform = [0, 0]
    for j in range(3, ny - 3):
        for i in range(3, nx - 3):
            c = j * nx + i
            Rf = np.zeros(W.shape[0])
            for d in range(D):
                lo = face(d, i, j)
                hi = face(d, i + 1, j) if d == 0 else face(d, i, j + 1)
                Rf = Rf - (hi[0] - lo[1]) / g.dx[d]
                mixed[d] += lo[2] != hi[2]
                uniform[d] += lo[2]
            Vc, o = orc.prim_cell(f, W[:, c])
            a = abs(Vc[N]) + abs(Vc[N + 1]) + o["c"]
            pc, rho = Vc[N + D], W[:N, c].sum()
            scale = np.concatenate([np.full(N, rho * a), np.full(D, rho * a * a + pc),
                                    [(abs(W[N + D, c]) + pc) * a], np.full(N - 1, a)]) / min(g.dx[:D])
            assert (np.abs(R[:, c] - Rf) <= 1e-12 * scale).all(), (i, j, (R[:, c] - Rf) / scale)
    assert min(uniform) > 100 and min(mixed) >= 4, (uniform, mixed)


def test_grid_sweep_matches_the_full_face_evaluation_3d(orc):
    """As above in 3D: a water sphere in moving air (u = (40, -25, 15) m/s, uniform p
    and T, 16^3 cells, the sphere's surface a jump), where every direction has
    uniform and non-uniform stencils side by side; the grid right-hand side of every
    cell three cells from the sides equals the one assembled from fully evaluated faces
    of all three directions."""
    n = 16
    f = _fluid(orc, [P.PAPER_WATER, P.PAPER_AIR], D=3)
    x = np.arange(n) + 0.5
    Z, Y, X = np.meshgrid(x, x, x, indexing="ij")
    inside = ((X - 8.2) ** 2 + (Y - 7.9) ** 2 + (Z - 8.1) ** 2 < 4.0 ** 2).ravel()
    nc = n ** 3
    prim = np.stack([np.where(inside, 1.0 - 1e-8, 1e-8), np.full(nc, 40.0), np.full(nc, -25.0),
                     np.full(nc, 15.0), np.full(nc, 1.0e5), np.full(nc, 300.0)])
    W = orc.ic_from_prim(f, prim)
    g = orc.make_grid([n, n, n], [1e-3, 1e-3, 1e-3])
    p = orc.make_params()
    lam = [2e-4, 2e-4, 2e-4]
    R = orc.rhs(f, p, g, W, lam)
    N, D = f.N, 3
    stride = [1, n, n * n]
    faces = {}

    def face(d, c):  # face of direction d between cell c - stride[d] and cell c
        if (d, c) not in faces:
            W6 = np.ascontiguousarray(W[:, [c + k * stride[d] for k in range(-3, 3)]].T)
            Gm, Gp, _ = orc.face(f, p, d, lam[d], W6)
            faces[(d, c)] = (Gm, Gp, bool((W6 == W6[2]).all()))
        return faces[(d, c)]

    mixed = [0, 0, 0]
    for k in range(3, n - 3):
        for j in range(3, n - 3):
            for i in range(3, n - 3):
                c = (k * n + j) * n + i
                Rf = np.zeros(W.shape[0])
                for d in range(D):
                    lo, hi = face(d, c), face(d, c + stride[d])
                    Rf = Rf - (hi[0] - lo[1]) / g.dx[d]
                    mixed[d] += lo[2] != hi[2]
                Vc, o = orc.prim_cell(f, W[:, c])
                a = abs(Vc[N]) + abs(Vc[N + 1]) + abs(Vc[N + 2]) + o["c"]
                pc, rho = Vc[N + D], W[:N, c].sum()
                scale = np.concatenate([np.full(N, rho * a), np.full(D, rho * a * a + pc),
                                        [(abs(W[N + D, c]) + pc) * a], np.full(N - 1, a)]) / g.dx[0]
                assert (np.abs(R[:, c] - Rf) <= 1e-12 * scale).all(), (i, j, k, (R[:, c] - Rf) / scale)
    assert min(mixed) >= 20, mixed


def test_hllc_resolves_isolated_contact(orc):
    """Equal p and u, different composition: HLLC is exact for a contact, so
    s_* = u and the flux is the upwind (left) physical flux."""
    f = _fluid(orc, [P.PAPER_WATER, P.PAPER_AIR])
    WL, VL, _ = _two_species_V(orc, f, 1 - 1e-8, 40.0, 1e6, 300.0)
    WR, VR, _ = _two_species_V(orc, f, 1e-8, 40.0, 1e6, 900.0)
    G, s = orc.hllc(f, 0, VL, VR)
    assert s == pytest.approx(40.0, rel=1e-12)
    expect = np.array([WL[0] * 40, WL[1] * 40, WL[2] * 40 + 1e6, (WL[3] + 1e6) * 40, VL[4] * 40])
    np.testing.assert_allclose(G, expect, rtol=1e-11)


def test_hllc_mirror_states_zero_mass_flux(orc):
    """Mirror-symmetric states (u_L = -u_R): s_* = 0 and no mass crosses."""
    f = _fluid(orc, [P.PAPER_WATER, P.PAPER_AIR])
    _, VL, _ = _two_species_V(orc, f, 0.4, 120.0, 3e5, 300.0)
    VR = VL.copy()
    VR[2] = -VL[2]
    G, s = orc.hllc(f, 0, VL, VR)
    assert abs(s) < 1e-10
    assert abs(G[0]) < 1e-9 * abs(VL[0] * VL[2]) and abs(G[1]) < 1e-9 * abs(VL[1] * VL[2])
    assert abs(G[3]) < 1e-6


def test_first_order_update_quasi_positive(orc):
    """Sec. 4.1.2: with CFL <= 0.5 the half-cell updates W_i -+ 2 lambda (G^HLLC -+ F_i)
    of random admissible pairs stay in script-G (positive partial densities,
    bounded volume fractions, positive rho e~)."""
    f = _fluid(orc, [P.BENCH_WATER, P.BENCH_AIR, P.BENCH_HELIUM])
    params = orc.make_params(scheme=1, limiters=0)
    prim, _ = P.random_admissible_states(3, 1, 400, seed=11)
    # make neighbours strongly different: shuffle pressures over 5 decades
    W = orc.ic_from_prim(f, prim)
    rng = np.random.default_rng(3)
    bad = 0
    for t in range(200):
        i, j = rng.integers(0, W.shape[1], 2)
        Wi, Wj = W[:, i], W[:, j]
        Vi, oi = orc.prim_cell(f, Wi)
        Vj, oj = orc.prim_cell(f, Wj)
        lam = 0.5 / max(abs(Vi[3]) + oi["c"], abs(Vj[3]) + oj["c"])
        W6 = np.stack([Wi, Wi, Wi, Wj, Wj, Wj])
        Gm, Gp, dg = orc.face(f, params, 0, lam, W6)
        for Wn, G, sgn in ((Wi, Gm, -1.0), (Wj, Gp, 1.0)):
            Vn, _ = orc.prim_cell(f, Wn)
            F = np.array([Wn[0] * Vn[3], Wn[1] * Vn[3], Wn[2] * Vn[3], Wn[3] * Vn[3] + Vn[4],
                          (Wn[4] + Vn[4]) * Vn[3], 0.0, 0.0])
            Wh = Wn + sgn * 2 * lam * (G - F)
            al = np.array([Wh[5], Wh[6], 1 - Wh[5] - Wh[6]])
            rhoe = Wh[4] - 0.5 * Wh[3] ** 2 / Wh[:3].sum()
            if (Wh[:3] < 0).any() or (al < -1e-14).any() or (al > 1 + 1e-14).any() or rhoe <= 0:
                bad += 1
    assert bad == 0


# ---------------------------------------------------------------- relaxation (Sec. 4.2)

def _relax_checks(orc, f, W):
    N = f.N
    out, ps, Ts = orc.relax_cell(f, W)
    # conserved: partial densities, momentum, energy unchanged bit for bit
    np.testing.assert_array_equal(out[:N + f.D + 1], W[:N + f.D + 1])
    al = np.append(out[N + f.D + 1:], 1.0 - out[N + f.D + 1:].sum())
    assert (al >= 0).all() and (al <= 1).all()
    # pressure and temperature equilibrium: every species at p*, T*
    rho_k = out[:N] / al
    for k in range(N - 1):
        Tk = (ps + f.pinf[k]) / ((f.gamma[k] - 1.0) * rho_k[k] * f.cv[k])
        assert Tk == pytest.approx(Ts, rel=1e-13)
    # volume constraint (Eq. thermal_relax_constraint_1): sum_k alpha_k rho_k / rho_k(p*, T*) = 1,
    # which also puts the derived species N at T*
    rho_star = np.array([(ps + f.pinf[k]) / ((f.gamma[k] - 1.0) * f.cv[k] * Ts) for k in range(N)])
    # (B_p and C_p cancel p_inf-sized terms when p* << p_inf, hence 1e-10)
    assert np.sum(out[:N] / rho_star) == pytest.approx(1.0, abs=1e-10)
    # the five-equation mixture pressure of the relaxed state equals p*
    V, o = orc.prim_cell(f, out)
    assert V[N + f.D] == pytest.approx(ps, rel=1e-9, abs=1e-9 * max(f.pinf))
    # T* of Eq. T_relax_rho agrees with Eq. T_relax_e
    rho = W[:N].sum()
    Y = W[:N] / rho
    cv = np.array(f.cv[:N])
    cp = cv * np.array(f.gamma[:N])
    l = f.liq
    T_rho = 1.0 / rho / (Y[l] * (f.gamma[l] - 1) * cv[l] / (ps + f.pinf[l])
                         + (np.dot(Y, cp) - np.dot(Y, cv) - Y[l] * (cp[l] - cv[l])) / ps)
    assert T_rho == pytest.approx(Ts, rel=1e-9)
    assert ps > 0 and Ts > 0
    # idempotent
    again, ps2, Ts2 = orc.relax_cell(f, out)
    np.testing.assert_allclose(again, out, rtol=1e-12, atol=1e-20)
    return out, ps, Ts


def test_relaxation_equilibrium_and_conservation(orc):
    f = _fluid(orc, [P.BENCH_WATER, P.BENCH_AIR, P.BENCH_HELIUM])
    prim, _ = P.random_admissible_states(3, 2, 50, seed=5)
    f.D = 2
    W = orc.ic_from_prim(f, prim)
    rng = np.random.default_rng(9)
    for c in range(W.shape[1]):
        w = W[:, c].copy()
        # take it out of thermal equilibrium: move volume fraction, keep W conserved parts
        w[6] = min(max(w[6] * rng.uniform(0.5, 1.5), 1e-9), 0.999)
        w[7] = min(max(w[7] * rng.uniform(0.5, 1.5), 1e-9), 1.0 - w[6] - 1e-9)
        _relax_checks(orc, f, w)


def test_relaxation_keeps_equilibrium_states(orc):
    """A state already in p-T equilibrium is a fixed point (Sec. 4.2)."""
    f = _fluid(orc, [P.PAPER_WATER, P.PAPER_AIR, P.PAPER_SF6])
    prim, _ = P.random_admissible_states(3, 1, 30, seed=2,
                                         fluids=[P.PAPER_WATER, P.PAPER_AIR, P.PAPER_SF6])
    W = orc.ic_from_prim(f, prim)
    for c in range(W.shape[1]):
        out, ps, Ts = orc.relax_cell(f, W[:, c])
        assert ps == pytest.approx(prim[3, c], rel=1e-9)
        assert Ts == pytest.approx(prim[4, c], rel=1e-9)
        np.testing.assert_allclose(out[4:], W[4:, c], rtol=1e-9)


def test_relaxation_ideal_gases_closed_form(orc):
    """All ideal gases: C_p = 0 and p* = rho e~ (cbar_p - cbar_v)/cbar_v."""
    f = _fluid(orc, [P.PAPER_AIR, P.BENCH_HELIUM])
    W = np.array([0.7, 0.05, 30.0, 2.5e5, 0.3])
    out, ps, Ts = orc.relax_cell(f, W)
    rho = 0.75
    Y = W[:2] / rho
    cv = np.array(f.cv[:2])
    cp = cv * np.array(f.gamma[:2])
    rhoe = W[3] - 0.5 * W[2] ** 2 / rho
    assert ps == pytest.approx(rhoe * (Y @ cp - Y @ cv) / (Y @ cv), rel=1e-14)


# ---------------------------------------------------------------- shock sensor

def test_sensor_constant_and_zero_denominator(orc):
    assert orc.sensor(np.full(6, 3.0)) == 0.0
    assert orc.sensor(np.zeros(6)) == 0.0  # zero denominator reads as 0
    # linear data: the fourth-order second difference vanishes
    assert orc.sensor(np.arange(6, dtype=float) + 10.0) == pytest.approx(0.0, abs=1e-16)


# ---------------------------------------------------------------- time step (Sec. 4.1.2)

def test_dt_closed_form(orc):
    f = _fluid(orc, [P.PAPER_WATER, P.PAPER_AIR], D=2)
    W = _W_from_prim(orc, f, [0.3, 20.0, -50.0, 1e5, 300.0])
    _, o = orc.prim_cell(f, W[:, 0])
    Wg = np.repeat(W, 12, axis=1)
    g = orc.make_grid([4, 3], [0.1, 0.05])
    dt, tau = orc.dt(f, g, Wg, 0.5)
    t0 = (20 + o["c"]) / 0.1
    t1 = (50 + o["c"]) / 0.05
    assert dt == pytest.approx(0.5 / (t0 + t1), rel=1e-15)
    lam = orc.lambdas(f, g, Wg, dt)
    # lambda_d = CFL / (|u_d| + c)_max when dt is the CFL step
    assert lam[0] == pytest.approx(0.5 / (20 + o["c"]), rel=1e-14)
    assert lam[1] == pytest.approx(0.5 / (50 + o["c"]), rel=1e-14)


def test_explicit_tanh_matches_the_function(orc):
    """The sensor's tanh (Sec. 4.3.1) is evaluated explicitly (Cody-Waite
    reduction and Taylor series); it must be tanh to within a few ulps over the
    whole range, including the odd symmetry and the saturated tails."""
    import math
    xs = np.concatenate([np.linspace(-40, 40, 8001), np.logspace(-300, 1.6, 2000)])
    for x in xs:
        for v in (x, -x):
            t = orc.tanh(v)
            ref = math.tanh(v)
            assert abs(t - ref) <= 4 * np.spacing(abs(ref)) + 1e-300, (v, t, ref)
            assert orc.tanh(-v) == -t



def test_ic_table_undex(orc):
    """Table IC_2D_three_species_extreme_UNDEX_problem (Sec. 5.10): partial
    densities of the water, air and detonation-product regions (the minor
    third species, whose alpha is derived as 1 - alpha_1 - alpha_2, to the
    rounding of that difference)."""
    pr = P.undex_2d(48, 60)
    f, g, W = orc.setup(pr)
    x, y = P.cell_centers(pr.n, pr.lo, pr.hi)
    water = int(np.argmax((y < -3.0)))
    air = int(np.argmax((y > 5.0)))
    det = int(np.argmin(np.hypot(x, y + 0.5)))
    exp = {water: (1.0227724208197188e3, 1.1817862212832324e-8, 1.7000838926174497e-8),
           air: (1.0227724412751677e-5, 1.1817861976475079, 1.7000838926174497e-8),
           det: (8.9361901785714267e-7, 8.6891757696127126e-6, 1.2499999749999999e3)}
    for c, (a, b, d) in exp.items():
        assert W[0, c] == pytest.approx(a, rel=1e-14)
        assert W[1, c] == pytest.approx(b, rel=1e-14)
        assert W[2, c] == pytest.approx(d, rel=1e-14 if c == det else 1e-7)


def test_ic_and_inflow_tables_mach100_jet(orc):
    """Tables IC_2D_Mach_100_water_jet and BC_2D_Mach_100_water_jet (Sec. 5.9):
    partial densities of the ambient air and of the jet and ambient parts of the
    Dirichlet inflow, from p = 101325 Pa, T = 298 K and the volume fractions."""
    pr = P.mach100_jet_2d(64, 32)
    f, g, W = orc.setup(pr)
    assert W[0, 100] == pytest.approx(1.0227724412751677e-5, rel=1e-14)
    assert W[1, 100] == pytest.approx(1.1817862094653702, rel=1e-14)
    Wb = g._keep[0]  # left side, one state per row
    jet, amb = 16, 0  # rows at y = +0.0039 L and y = -0.246 L
    assert Wb[0, jet] == pytest.approx(1.0227724310474432e3, rel=1e-14)
    assert Wb[1, jet] == pytest.approx(1.1817862272214237e-8, rel=1e-14)
    assert Wb[2, jet] == pytest.approx((1.0227724310474432e3 + 1.1817862272214237e-8) * 1.5e5, rel=1e-14)
    assert Wb[0, amb] == pytest.approx(1.0227724412751677e-5, rel=1e-14)
    assert Wb[1, amb] == pytest.approx(1.1817862094653702, rel=1e-14)
    assert Wb[2, amb] == 0.0
    # the jet occupies the rows whose centres satisfy |y| <= 0.05 L
    ycen = -0.25 + (np.arange(32) + 0.5) / 64.0
    np.testing.assert_array_equal(Wb[2] > 0.0, np.abs(ycen) <= 0.05)


def test_cfl_with_four_equation_sound_speed(orc):
    """The CFL option with the four-equation HRM sound speed (Eq. 4_eqn_sos):
    for a uniform water-air mixture at rest (alpha = 0.5, 101325 Pa, 298 K)
    tau = c/dx with the printed speeds of Sec. 5.3, 19.897 m/s against the
    five-equation 913.05 m/s."""
    f = _fluid(orc, [P.PAPER_WATER, P.PAPER_AIR])
    W = np.repeat(_W_from_prim(orc, f, [0.5, 0.0, 101325.0, 298.0]), 16, axis=1)
    g = orc.make_grid([16], [0.01])
    dt5, tau5 = orc.dt(f, g, W, 0.5)
    dt4, tau4 = orc.dt(f, g, W, 0.5, sound=1)
    assert tau4[0] * 0.01 == pytest.approx(19.897, abs=0.0005)
    assert tau5[0] * 0.01 == pytest.approx(913.05, abs=0.005)
    assert dt4 == pytest.approx(0.5 * 0.01 / (tau4[0] * 0.01), rel=1e-15)
