"""Whole-scheme pins of the CPU oracle: the paper's printed convergence table,
conservation, positivity, equilibrium preservation and the exact Riemann
solution. The expected values come from the paper or from mathematics, never
from the oracle itself or from the CUDA path."""
import math
import os

import numpy as np
import pytest

from paper_2208_04488_gb300 import problems as P
from tests import exact_riemann as ER

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden_convergence():
    rows = np.loadtxt(os.path.join(GOLDEN, "convergence_2d.txt"))
    return {int(r[0]): r[1:] for r in rows}


def run_advection_2d(orc, n):
    pr = P.advection_2d_smooth(n)
    f, g, W = orc.setup(pr)
    nsteps = int(round(pr.t_end / pr.dt))
    W1 = orc.step(f, orc.make_params(), g, W, pr.dt, nsteps)
    _, _, We = orc.setup(P.advection_2d_smooth(n, t=pr.t_end))
    rho, rho_e = W1[0] + W1[1], We[0] + We[1]
    return (np.sqrt(np.mean((rho - rho_e) ** 2)), np.max(np.abs(rho - rho_e)),
            np.sqrt(np.mean((W1[5] - We[5]) ** 2)), np.max(np.abs(W1[5] - We[5])))


@pytest.mark.parametrize("n", [8, 16, 32, 64])
def test_spatial_convergence_table(orc, n):
    """Sec. 5.2, Table 2D_errors_and_rate_of_convergence_advection: the L2 and
    Linf errors of rho and alpha_1 printed by the paper (4 significant digits)."""
    ref = _golden_convergence()[n]
    got = run_advection_2d(orc, n)
    for g_, r_ in zip(got, ref):
        assert g_ == pytest.approx(r_, rel=1.5e-3), (n, got, ref)


@pytest.mark.slow
def test_spatial_convergence_table_128(orc):
    ref = _golden_convergence()[128]
    got = run_advection_2d(orc, 128)
    for g_, r_ in zip(got, ref):
        assert g_ == pytest.approx(r_, rel=1.5e-3), (got, ref)


def test_uniform_state_has_zero_rhs(orc):
    """Uniform states are steady: every midpoint flux is the same, so the flux
    difference vanishes exactly (Eq. semi_W_G_pm_eqn), in 1D, 2D and 3D."""
    for n, bc in (([17], [0, 0]), ([9, 7], [1, 1, 0, 0]), ([5, 6, 7], [0, 0, 1, 1, 0, 0])):
        D = len(n)
        gamma, pinf, cv, q = P._species([P.BENCH_WATER, P.BENCH_AIR, P.BENCH_HELIUM])
        f = orc.make_fluid(gamma, pinf, cv, q, D=D)
        nc = int(np.prod(n))
        prim = np.array([0.3, 0.5] + [37.0, -12.0, 5.0][:D] + [2.0e5, 320.0])[:, None]
        W = orc.ic_from_prim(f, np.repeat(prim, nc, axis=1))
        g = orc.make_grid(n, [0.1] * D, bc)
        R = orc.rhs(f, orc.make_params(), g, W, [1e-5] * 3)
        assert np.max(np.abs(R)) == 0.0


def _blobs_2d(orc, n=24, seed=1):
    rng = np.random.default_rng(seed)
    gamma, pinf, cv, q = P._species([P.BENCH_WATER, P.BENCH_AIR, P.BENCH_HELIUM])
    f = orc.make_fluid(gamma, pinf, cv, q, D=2)
    x, y = P.cell_centers([n, n], [0, 0], [1, 1])
    aw = np.where(np.hypot(x - 0.3, y - 0.4) < 0.2, 1 - 2e-8, 1e-8)
    ahe = np.where(np.hypot(x - 0.7, y - 0.6) < 0.15, 1 - 2e-8, 1e-8)
    u = 50 + 20 * np.sin(2 * np.pi * y)
    v = -30 + 10 * np.cos(2 * np.pi * x)
    p = 1e5 * (1 + 0.5 * (x < 0.5))
    T = 300 + 50 * rng.random(n * n)
    prim = np.array([aw, 1 - aw - ahe, u, v, p, T])
    W = orc.ic_from_prim(f, prim)
    g = orc.make_grid([n, n], [1.0 / n] * 2, [1, 1, 1, 1])
    return f, g, W


def test_conservation_periodic(orc):
    """Sec. 4.4: the partial densities, momentum and total energy are conserved
    by the quasi-conservative update and by the relaxation (periodic grid with
    material interfaces, a pressure jump and shear)."""
    f, g, W = _blobs_2d(orc)
    dt, _ = orc.dt(f, g, W, 0.4)
    W1 = orc.step(f, orc.make_params(), g, W, dt, 4)
    for m in range(3 + 2 + 1):  # alpha_k rho_k, rho u, rho v, E
        s0, s1 = W[m].sum(), W1[m].sum()
        scale = np.abs(W[m]).sum()
        assert abs(s1 - s0) <= 1e-13 * scale, (m, s0, s1)
    assert orc.admissibility(f, g, W1) == [0, 0, 0, 0]


def test_extreme_shock_tube_positivity(orc):
    """Sec. 5.5: the extreme gas/liquid shock tube (1e12 / 1e5 Pa) stays
    admissible with the limiters and fails with them off."""
    pr = P.shock_tube_1d_paper(200, extreme=True)
    f, g, W0 = orc.setup(pr)
    dt = 4.0e-8  # the paper's dt x dx ratio at 200 cells; CFL < 0.5
    assert orc.dt(f, g, W0, 0.5)[0] > dt
    W = W0.copy()
    for _ in range(40):
        W = orc.step(f, orc.make_params(), g, W, dt, 1)
        assert orc.admissibility(f, g, W) == [0, 0, 0, 0]
    W = W0.copy()
    failed = False
    for _ in range(40):
        W = orc.step(f, orc.make_params(limiters=0), g, W, dt, 1)
        if sum(orc.admissibility(f, g, W)) or not np.isfinite(W).all():
            failed = True
            break
    assert failed


def test_shock_tube_converges_to_exact(orc):
    """Sec. 5.4 gas/liquid shock tube at t = 3e-4 s: the L1 error of the
    mixture density against the exact two-material Riemann solution decreases
    under grid refinement, and the shock and interface sit where the exact
    solution puts them."""
    errs = []
    for n in (150, 300):
        pr = P.shock_tube_1d_paper(n)
        f, g, W = orc.setup(pr)
        dt = 5.0e-7 * 500.0 / n
        nsteps = int(round(3e-4 / dt))
        W = orc.step(f, orc.make_params(), g, W, dt, nsteps)
        x = (np.arange(n) + 0.5) * 1.5 / n
        L = ER.Side(1000.0, 0.0, 1e9, 3.0, 8.533e8)
        R = ER.Side(20.0, 0.0, 1e5, 1.4, 0.0)
        rho_e, u_e, p_e, _ = ER.solve(L, R, x, 0.8, 3e-4)
        rho = W[0] + W[1]
        errs.append(np.mean(np.abs(rho - rho_e)) * 1.5)
    assert errs[1] < 0.75 * errs[0], errs


def test_exact_riemann_textbook():
    """The exact solver reproduces textbook star states (Toro, Riemann solvers
    and numerical methods for fluid dynamics, Table 4.2, tests 1 and 3)."""
    p, u = ER.star_state(ER.Side(1.0, 0.0, 1.0, 1.4, 0.0), ER.Side(0.125, 0.0, 0.1, 1.4, 0.0))
    assert p == pytest.approx(0.30313, abs=5e-5) and u == pytest.approx(0.92745, abs=5e-5)
    p, u = ER.star_state(ER.Side(1.0, 0.0, 1000.0, 1.4, 0.0), ER.Side(1.0, 0.0, 0.01, 1.4, 0.0))
    assert p == pytest.approx(460.894, abs=5e-3) and u == pytest.approx(19.5975, abs=5e-4)


def test_material_interface_equilibrium(orc):
    """App. A: advecting material interfaces in p-T equilibrium keeps p, u and T
    uniform to relative errors of order 1e-5 (first tenth of the period; the
    paper reports 1e-5 to 1e-6 after a full period at 500 cells)."""
    pr = P.material_interface_1d(500)
    f, g, W = orc.setup(pr)
    W = orc.step(f, orc.make_params(), g, W, pr.dt, 1600)
    eu, ep = [], []
    for c in range(W.shape[1]):
        V, o = orc.prim_cell(f, W[:, c])
        eu.append(abs(V[2] / 100.0 - 1))
        ep.append(abs(V[3] / 101325.0 - 1))
    eT = [abs(orc.c4eq_cell(f, W[:, c])["T"] / 298.0 - 1) for c in range(W.shape[1])]
    assert max(eu) < 1e-4 and max(ep) < 1e-4 and max(eT) < 1e-4, (max(eu), max(ep), max(eT))


def test_limited_half_states_are_admissible(orc):
    """Sec. 4.3.2: at every face of the extreme shock tube (1e12 / 1e5 Pa,
    after a few steps, where the limiters do fire) the interpolation limiter
    leaves midpoint states with positive partial densities, bounded volume
    fractions and rho c^2 > 0, and after the flux limiter the half-cell states
    W_i - 2 lam (G^- - F_i) and W_{i+1} + 2 lam (G^+ - F_{i+1}) are in script-G."""
    pr = P.shock_tube_1d_paper(200, extreme=True)
    f, g, W = orc.setup(pr)
    dt = 4.0e-8
    p = orc.make_params()
    W = orc.step(f, p, g, W, dt, 9)
    lam = dt / g.dx[0]
    n = W.shape[1]
    limited = 0
    for fc in range(3, n - 2):
        W6 = np.ascontiguousarray(W[:, fc - 3:fc + 3].T)
        Gm, Gp, dg = orc.face(f, p, 0, lam, W6)
        limited += (dg["flux_flags"] != 0) + int(np.any(dg["VL"] != dg["VL_weno"]))
        limited += int(np.any(dg["VR"] != dg["VR_weno"]))
        for V in (dg["VL"], dg["VR"]):
            assert (V[:2] >= 0).all() and 0 <= V[4] <= 1
            Wc, o = orc.cons_cell(f, V)
            assert orc.prim_cell(f, Wc)[1]["rc2"] > 0
        for Wn, G, sgn in ((W6[2], Gm, -1.0), (W6[3], Gp, 1.0)):
            Vn, _ = orc.prim_cell(f, Wn)
            F = np.array([Wn[0] * Vn[2], Wn[1] * Vn[2], Wn[2] * Vn[2] + Vn[3],
                          (Wn[3] + Vn[3]) * Vn[2], 0.0])
            Wh = Wn + sgn * 2 * lam * (G - F)
            assert (Wh[:2] >= 0).all()
            assert 0.0 <= Wh[4] <= 1.0
            assert Wh[3] - 0.5 * Wh[2] ** 2 / Wh[:2].sum() - Wh[0] * f.q[0] > 0
    assert limited > 0  # these faces do exercise the limiters


def test_counting_build_matches_and_counts(orc):
    """The operation-counting build computes the same numbers."""
    pr = P.shock_bubble_2d(32, 16)
    f, g, W = orc.setup(pr)
    p = orc.make_params()
    a = orc.step(f, p, g, W, 1e-7, 1)
    b, counts = orc.step(f, p, g, W, 1e-7, 1, count=True)
    np.testing.assert_array_equal(a, b)
    per_cell = sum(counts.values()) / W.shape[1]
    assert 5e3 < per_cell < 1e5


def test_openmp_build_gives_identical_results(orc):
    """The multi-threaded oracle build shares the independent grid lines and
    cells among host threads; its states equal the serial build's exactly."""
    if not orc.has_omp():
        pytest.skip("no OpenMP in this compiler")
    pr = P.shock_bubble_2d(48, 24)
    f, g, W = orc.setup(pr)
    p = orc.make_params()
    dt, _ = orc.dt(f, g, W, pr.cfl)
    np.testing.assert_array_equal(orc.step(f, p, g, W, dt, 3), orc.step(f, p, g, W, dt, 3, omp=True))
    assert orc.threads(True) >= 1


def _golden_temporal():
    rows = {}
    path = os.path.join(os.path.dirname(__file__), "golden", "temporal_1d.txt")
    for line in open(path):
        if line.startswith("#") or not line.strip():
            continue
        name, steps, *vals = line.split()
        rows[(name, int(steps))] = [float(v) for v in vals]
    return rows


@pytest.mark.parametrize("integrator,name", [(1, "euler"), (2, "rk2"), (0, "rk3")])
def test_temporal_convergence_tables(orc, integrator, name):
    """Sec. 5.1, Tables 1D_errors_and_rate_of_temporal_convergence_advection_*:
    the 64-cell periodic advection with the exact spatial derivatives evaluated
    at each stage's time (t^n, t^n + dt, t^n + dt/2) and the thermal relaxation
    after every stage; the L2 and Linf errors of rho and alpha_1 at t = 0.1 s for
    10-80 steps of forward Euler, SSP-RK2 and SSP-RK3, as printed (4 digits)."""
    ref = _golden_temporal()
    pr = P.advection_1d_smooth(64)
    f, g, W = orc.setup(pr)
    r1 = W[0, 0] / pr.prim[0, 0]
    r2 = W[1, 0] / (1.0 - pr.prim[0, 0])
    adv = [0.5, 0.25, math.pi, 10.0, 101325.0, r1, r2, -1.0]
    x = -1.0 + (np.arange(64) + 0.5) * (2.0 / 64)
    a_ex = 0.5 + 0.25 * np.sin(math.pi * (x - 10.0 * 0.1))
    rho_ex = r1 * a_ex + r2 * (1.0 - a_ex)
    for ns in (10, 20, 40, 80):
        W1 = orc.step_exact(f, orc.make_params(integrator=integrator), g, W, 0.1 / ns, ns, 0.0, adv)
        rho, a1 = W1[0] + W1[1], W1[4]
        got = [np.sqrt(np.mean((rho - rho_ex) ** 2)), np.max(np.abs(rho - rho_ex)),
               np.sqrt(np.mean((a1 - a_ex) ** 2)), np.max(np.abs(a1 - a_ex))]
        for gv, rv in zip(got, ref[(name, ns)]):
            assert gv == pytest.approx(rv, rel=1e-3), (name, ns, got, ref[(name, ns)])
