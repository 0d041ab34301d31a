"""Pins of the oracle pieces of the learned smoothness detector: the MLP's
back-propagated gradient, loss, Adam update and bfloat16 rounding; the
normalised stencil features and WENO-IS weight deviation; the gated scheme.

Expected values come from finite differences, closed forms, library routines
(torch's bfloat16 conversion) and invariants -- never from the oracle itself or
the CUDA path.
"""
import math

import numpy as np
import pytest

from oracle import mlp
from paper_2208_04488_gb300 import problems as P


# ---------------------------------------------------------------- MLP

def _theta(seed, scale=0.3):
    rng = np.random.default_rng(seed)
    return rng.normal(0.0, scale, mlp.NPARAM)


def test_mlp_grad_matches_central_differences():
    """Back-propagation (oracle.mlp.grad) against central differences of the
    loss in every parameter: catches a transposed weight, a dropped bias or a
    wrong ReLU mask."""
    rng = np.random.default_rng(1)
    theta = _theta(2)
    X = rng.uniform(-1.0, 1.0, (24, mlp.NIN))
    y = (rng.uniform(size=24) < 0.5).astype(np.float64)
    g = mlp.grad(theta, X, y)
    h = 1e-6
    fd = np.zeros_like(theta)
    for i in range(theta.size):
        e = np.zeros_like(theta)
        e[i] = h
        fd[i] = (mlp.loss(theta + e, X, y) - mlp.loss(theta - e, X, y)) / (2 * h)
    assert np.linalg.norm(g - fd) <= 1e-7 * np.linalg.norm(fd)
    # every parameter block receives gradient
    for lo, hi in ((0, 960), (960, 992), (992, 2016), (2016, 2048), (2048, 2080), (2080, 2081)):
        assert np.any(g[lo:hi] != 0.0)


def test_mlp_loss_closed_forms():
    """Zero weights give p = 1/2 and loss n log 2; one sample matches the
    cross-entropy -[y log p + (1 - y) log(1 - p)] with p = 1/(1 + e^-z)."""
    X = np.ones((7, mlp.NIN))
    y = np.array([0, 1, 1, 0, 1, 0, 0], dtype=np.float64)
    assert mlp.loss(np.zeros(mlp.NPARAM), X, y) == pytest.approx(7 * math.log(2.0), rel=1e-15)
    theta = _theta(5)
    x = np.linspace(-1, 1, mlp.NIN)[None, :]
    # logit by explicit loops (not the oracle's matrix products)
    W1, b1, W2, b2, w3, b3 = mlp.unpack(theta)
    h1 = [max(0.0, sum(x[0, k] * W1[k, n] for k in range(30)) + b1[n]) for n in range(32)]
    h2 = [max(0.0, sum(h1[k] * W2[k, n] for k in range(32)) + b2[n]) for n in range(32)]
    z = sum(h2[n] * w3[n] for n in range(32)) + b3
    p = 1.0 / (1.0 + math.exp(-z))
    for yy in (0.0, 1.0):
        ref = -(yy * math.log(p) + (1 - yy) * math.log(1 - p))
        assert mlp.loss(theta, x, np.array([yy])) == pytest.approx(ref, rel=1e-12)
    assert mlp.forward(theta, x)[0][0] == pytest.approx(p, rel=1e-13)


def test_adam_constant_gradient_steps():
    """With a constant gradient the bias-corrected moments equal g and g^2 at
    every step, so each Adam step moves theta by lr g / (|g| + eps)."""
    g = np.array([0.5, -2.0, 1e-3, 0.0])
    th = np.zeros(4)
    m = np.zeros(4)
    v = np.zeros(4)
    for t in range(1, 6):
        th_new, m, v = mlp.adam_step(th, m, v, g, t, lr=0.01)
        np.testing.assert_allclose(th_new - th, -0.01 * g / (np.abs(g) + 1e-8), rtol=1e-12, atol=0)
        th = th_new


def test_bf16_rounding_matches_torch():
    """Round-to-nearest-even to bfloat16 against torch's conversion (a library
    routine), including ties and values near powers of two."""
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(3)
    x = np.concatenate([rng.normal(0, 1, 4000), rng.normal(0, 1e-3, 1000),
                        np.array([1.0, 1.00390625, 1.01171875, -1.00390625, 0.0, 2.0 ** -20, 3.0])])
    x32 = x.astype(np.float32)
    ref = torch.from_numpy(x32).to(torch.bfloat16).to(torch.float64).numpy()
    np.testing.assert_array_equal(mlp.bf16_round(x32), ref)


def test_forward_bf16_exact_on_representable_values():
    """With weights, inputs and hidden values exactly representable in bfloat16
    the inference arithmetic equals the FP64 forward pass."""
    rng = np.random.default_rng(4)
    theta = rng.integers(-4, 5, mlp.NPARAM) / 16.0
    X = rng.integers(-2, 3, (16, mlp.NIN)) / 4.0
    # hidden values stay small integers / 64: exact in bfloat16 (8 significant bits)
    _, (_, _, h1, _, _, z_ref) = mlp.forward(theta, X)
    assert np.all(mlp.bf16_round(h1) == h1)
    np.testing.assert_array_equal(mlp.forward_bf16(theta, X), z_ref)


# ---------------------------------------------------------------- features and labels

def _line_state(orc, fl, V_cols, D=1):
    """W[M, n] from primitive columns V = (alpha_k rho_k, u_d, p, alpha_k)."""
    gamma, pinf, cv, q = P._species(fl)
    f = orc.make_fluid(gamma, pinf, cv, q, D=D)
    V = np.asarray(V_cols, dtype=np.float64)
    W = np.stack([orc.cons_cell(f, V[:, c])[0] for c in range(V.shape[1])], axis=1)
    return f, W


def test_features_normalisation_and_selection(orc):
    """Features of a 2D three-species state: zero mean and unit range per
    quantity, zero for a quantity that is uniform on the stencil, invariant
    under the affine maps they normalise away, and the velocity block reads the
    velocity of the midpoint's direction."""
    fl = [P.BENCH_WATER, P.BENCH_AIR, P.BENCH_HELIUM]
    nx, ny = 8, 8
    rng = np.random.default_rng(7)
    n = nx * ny
    a1 = rng.uniform(0.1, 0.4, n)
    a2 = rng.uniform(0.1, 0.4, n)
    a3 = 1 - a1 - a2
    rho = np.array([1000.0, 1.2, 0.17])
    V = np.stack([a1 * rho[0], a2 * rho[1], a3 * rho[2],
                  rng.uniform(-10, 10, n),           # u_x varies
                  np.zeros(n),                       # u_y uniform (exactly: rho v = 0)
                  rng.uniform(1e5, 2e5, n), a1, a2])
    f, W = _line_state(orc, fl, V, D=2)
    g = orc.make_grid([nx, ny], [0.1, 0.1], [0, 0, 1, 1])
    p = orc.make_params()
    for d in (0, 1):
        nf = (nx + (d == 0)) * (ny + (d == 1))
        feat, dev = orc.stencil_sample(f, p, g, W, d, np.arange(nf))
        F = feat.reshape(nf, 5, 6)
        np.testing.assert_allclose(F.mean(axis=2), 0.0, atol=1e-14)
        rng_ = F.max(axis=2) - F.min(axis=2)
        if d == 0:
            # interior faces: every quantity varies along x
            inner = [t for t in range(nf) if 3 <= t % (nx + 1) <= nx - 3]
            np.testing.assert_allclose(rng_[inner], 1.0, rtol=1e-13)
        else:
            # u_y is uniform: its block is exactly zero along y, others vary
            assert np.all(F[:, 3, :] == 0.0)
            inner = [t for t in range(nf) if 3 <= t // nx <= ny - 3]
            np.testing.assert_allclose(rng_[inner][:, [0, 1, 2, 4]], 1.0, rtol=1e-13)
        assert np.all(dev >= 0.0) and np.all(dev < 1.0)
    # invariance: the pressure block is unchanged when p -> 3 p + 1e4 (stencil-wise affine)
    V2 = V.copy()
    V2[5] = 3.0 * V[5] + 1e4
    f2, W2 = _line_state(orc, fl, V2, D=2)
    nf = (nx + 1) * ny
    F1 = orc.stencil_sample(f, p, g, W, 0, np.arange(nf))[0].reshape(nf, 5, 6)
    F2 = orc.stencil_sample(f2, p, g, W2, 0, np.arange(nf))[0].reshape(nf, 5, 6)
    np.testing.assert_allclose(F2[:, 4], F1[:, 4], atol=1e-12)
    np.testing.assert_allclose(F2[:, :4], F1[:, :4], atol=1e-12)


def test_features_two_species_and_boundaries(orc):
    """Two species: the alpha_2 block is zero. A step in p over the stencil
    gives the -1/2, +1/2 pattern; transmissive ends repeat the edge cell and
    periodic ends wrap."""
    fl = [P.BENCH_WATER, P.BENCH_AIR]
    n = 12
    a1 = np.full(n, 0.5)
    p_ = np.where(np.arange(n) < 6, 2e5, 1e5)
    V = np.stack([a1 * 1000.0, (1 - a1) * 1.2, np.zeros(n), p_, a1])
    f, W = _line_state(orc, fl, V)
    prm = orc.make_params()
    g = orc.make_grid([n], [0.1], [0, 0])
    feat, dev = orc.stencil_sample(f, prm, g, W, 0, np.arange(n + 1))
    F = feat.reshape(n + 1, 5, 6)
    assert np.all(F[:, 1, :] == 0.0)      # no alpha_2
    assert np.all(F[:, 0, :] == 0.0)      # uniform alpha_1
    # midpoint 6 lies at the jump: nodes 3..8 -> p = 2e5 x3, 1e5 x3
    np.testing.assert_allclose(F[6, 4], [0.5, 0.5, 0.5, -0.5, -0.5, -0.5], atol=1e-15)
    assert dev[6] > 0.3                   # a jump drives the weights far from d_k
    # transmissive: uniform ghost stencil; its weights are d_k up to the rounding of
    # the common factor the weights are scaled by (App. C normalisation)
    assert dev[0] <= 1e-15 and np.all(F[0] == 0.0)
    gp = orc.make_grid([n], [0.1], [1, 1])
    Fp = orc.stencil_sample(f, prm, gp, W, 0, np.array([0]))[0].reshape(5, 6)
    # periodic midpoint 0: nodes n-3, n-2, n-1, 0, 1, 2 -> p = 1e5 x3, 2e5 x3
    np.testing.assert_allclose(Fp[4], [-0.5, -0.5, -0.5, 0.5, 0.5, 0.5], atol=1e-15)


def test_deviation_zero_on_linear_fields(orc):
    """A state linear in x has linear characteristic fields on every stencil, so
    the WENO-IS weights equal d_k (tau_5 = 0) and the deviation vanishes up to
    rounding; a single-cell spike drives it up."""
    fl = [P.BENCH_WATER, P.BENCH_AIR]
    n = 16
    x = np.arange(n, dtype=np.float64)
    a1 = 0.3 + 0.01 * x
    V = np.stack([a1 * 1000.0, (1 - a1) * 1.2, 2.0 + 0.5 * x, 1e6 + 1e4 * x, a1])
    f, W = _line_state(orc, fl, V)
    prm = orc.make_params()
    g = orc.make_grid([n], [0.1], [0, 0])
    idx = np.arange(3, n - 2)
    # partial densities are linear but rho c^2 is not: the projection matrices are
    # frozen per midpoint, so the characteristic fields stay linear on each stencil
    dev = orc.stencil_sample(f, prm, g, W, 0, idx)[1]
    assert np.all(dev < 1e-9), dev
    V2 = V.copy()
    V2[3, 8] *= 1.5
    f2, W2 = _line_state(orc, fl, V2)
    dev2 = orc.stencil_sample(f2, prm, g, W2, 0, np.array([8]))[1]
    assert dev2[0] > 0.1


# ---------------------------------------------------------------- gated scheme

def test_linear_weights_interpolate_quartics_exactly(orc):
    """With the linear weights the five-point interpolation to x_{i+1/2} is the
    fourth-degree interpolant: exact for polynomials up to degree 4, and the
    coefficients (3, -20, 90, 60, -5)/128 follow."""
    xs = np.array([-2.0, -1.0, 0.0, 1.0, 2.0])
    for deg in range(5):
        u = xs ** deg
        assert orc.weno_lin(u) == pytest.approx(0.5 ** deg, abs=1e-15)
    for j, c in enumerate([3, -20, 90, 60, -5]):
        e = np.zeros(5)
        e[j] = 1.0
        assert orc.weno_lin(e) == pytest.approx(c / 128.0, abs=1e-16)
    # and it is the limit of WENO-IS on smooth data (all beta equal, tau_5 -> 0)
    u = np.array([1.0, 2.0, 3.0, 4.0, 5.0])
    assert orc.weno_left(u)[0] == pytest.approx(orc.weno_lin(u), rel=1e-15)


def test_gated_rhs_locality_and_identity(orc):
    """An all-zero gate reproduces the ungated RHS bit for bit; gating one
    midpoint changes only its two neighbour cells; on a discontinuous state the
    fully gated RHS differs."""
    pr = P.shock_tube_1d_baseline(64)
    f, g, W = orc.setup(pr)
    prm = orc.make_params()
    lam = [1e-3]
    R0 = orc.rhs(f, prm, g, W, lam)
    Rz = orc.rhs(f, prm, g, W, lam, gates=[np.zeros(65, np.uint8)])
    np.testing.assert_array_equal(Rz, R0)
    # midpoint 45 sits at the interface (x = 0.7 -> cell 44.8)
    one = np.zeros(65, np.uint8)
    one[45] = 1
    R1 = orc.rhs(f, prm, g, W, lam, gates=[one])
    changed = np.nonzero(np.any(R1 != R0, axis=0))[0]
    assert set(changed.tolist()) <= {44, 45} and len(changed) > 0
    Rall = orc.rhs(f, prm, g, W, lam, gates=[np.ones(65, np.uint8)])
    assert np.any(Rall != R0)


def test_gated_step_smooth_advection_keeps_design_order(orc):
    """On the smooth 2D advection problem (Sec. 5.2) every stencil is smooth:
    with every midpoint gated to the linear weights (the optimal fifth-order
    interpolation) the scheme keeps its design order between 16^2 and 32^2 and
    errors within 25 % of WENO-IS's -- and not identical ones: the gate acts."""
    err = {}
    for n in (16, 32):
        pr = P.advection_2d_smooth(n)
        f, g, W = orc.setup(pr)
        nsteps = int(round(pr.t_end / pr.dt))
        _, _, We = orc.setup(P.advection_2d_smooth(n, t=pr.t_end))
        prm = orc.make_params()
        ones = [np.ones((n + (d == 0)) * (n + (d == 1)), np.uint8) for d in range(2)]
        for gated in (False, True):
            W1 = orc.step(f, prm, g, W, pr.dt, nsteps, gates=ones if gated else None)
            err[n, gated] = np.sqrt(np.mean((W1[5] - We[5]) ** 2))
    for n in (16, 32):
        assert err[n, True] != err[n, False]
        assert 0.8 <= err[n, True] / err[n, False] <= 1.25, err
    assert math.log2(err[16, True] / err[32, True]) >= 4.7, err
