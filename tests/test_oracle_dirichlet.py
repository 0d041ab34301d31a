"""Pins of the oracle's Dirichlet boundary (the prescribed inflow of the Sec. 5.9
jet) to an independent construction: the same grid widened by three cells on
every Dirichlet side, the new cells holding the boundary state of their line,
with transmissive sides. Every midpoint of an interior cell then sees the same
six nodes in both descriptions (a prescribed state fills all three ghost layers,
and the widened grid's own ghosts copy its outermost cell, which holds that
state), so the semi-discrete right-hand side of the interior cells must agree
bit for bit; the CFL maximum ranges over the same states, so dt and tau_d agree
bit for bit too (Sec. 4.1.2). A wrong side, a wrong transverse index or a ghost
layer left transmissive fails these comparisons.
"""
import itertools

import numpy as np
import pytest

from paper_2208_04488_gb300 import problems as P


def widened(pr, W, Wb):
    """W of the grid widened by 3 cells on every side (all sides Dirichlet);
    a cell outside the original grid takes the boundary state of the first
    direction in which it lies outside, at its other indices clamped to range."""
    n = list(pr.n)
    D = len(n)
    ne = [k + 6 for k in n]
    M = W.shape[0]
    Wi = W.reshape([M] + n[::-1])  # (M, [nz,] [ny,] nx)
    out = np.empty([M] + ne[::-1])
    for e in itertools.product(*[range(k) for k in ne]):
        o = [e[d] - 3 for d in range(D)]
        side = None
        for d in range(D):
            if o[d] < 0 or o[d] >= n[d]:
                side = (d, 0 if o[d] < 0 else 1)
                break
        if side is None:
            val = Wi[(slice(None),) + tuple(o[::-1])]
        else:
            d, s = side
            idx, stride = 0, 1
            for e2 in range(D):
                if e2 == d:
                    continue
                idx += min(max(o[e2], 0), n[e2] - 1) * stride
                stride *= n[e2]
            val = Wb[2 * d + s][:, idx]
        out[(slice(None),) + tuple(e[::-1])] = val
    return out.reshape(M, -1), ne


@pytest.mark.parametrize("n", [[11], [9, 7], [6, 5, 4]], ids=["1d", "2d", "3d"])
def test_dirichlet_matches_widened_grid(orc, n):
    pr = P.dirichlet_box(n)
    f, g, W = orc.setup(pr)
    Wb = {b: orc.ic_from_prim(f, prim) for b, prim in pr.boundary.items()}
    We, ne = widened(pr, W, Wb)
    ge = orc.make_grid(ne, pr.dx, [0] * (2 * len(n)))
    dt, tau = orc.dt(f, g, W, 0.45)
    dte, taue = orc.dt(f, ge, We, 0.45)
    assert dt == dte
    np.testing.assert_array_equal(tau, taue)
    lam = orc.lambdas(f, g, W, dt)
    np.testing.assert_array_equal(lam, orc.lambdas(f, ge, We, dt))
    p = orc.make_params()
    R = orc.rhs(f, p, g, W, lam)
    Re = orc.rhs(f, p, ge, We, lam).reshape([pr.M] + ne[::-1])
    inner = (slice(None),) + tuple(slice(3, 3 + k) for k in n[::-1])
    np.testing.assert_array_equal(R, Re[inner].reshape(pr.M, -1))
    # the boundary states matter: the same grid with transmissive sides differs
    gt = orc.make_grid(n, pr.dx, [0] * (2 * len(n)))
    assert np.abs(orc.rhs(f, p, gt, W, lam) - R).max() > 0.0


def test_jet_time_step_sees_the_inflow(orc):
    """The ambient air is at rest; the CFL step must still resolve the 1.5e5 m/s
    inflow (Sec. 4.1.2 over every state the stencils read)."""
    pr = P.mach100_jet_2d(64, 32)
    f, g, W = orc.setup(pr)
    dt, tau = orc.dt(f, g, W, pr.cfl)
    dx = pr.dx[0]
    assert tau[0] >= 1.5e5 / dx
    assert dt <= pr.cfl * dx / 1.5e5
    # and the water enters: one step adds partial density of water next to the
    # inlet; beyond the reach of three stages' stencils (9 cells) only the
    # relaxation's round-off changes it
    W1 = orc.step(f, orc.make_params(), g, W, dt, 1)
    gain = (W1[0] - W[0]).reshape(pr.n[1], pr.n[0])
    assert gain[:, :3].sum() > 1.0
    assert np.abs(gain[:, 10:]).max() <= 1e-14 * np.abs(W[0]).max()
    assert orc.admissibility(f, g, W1) == [0, 0, 0, 0]
