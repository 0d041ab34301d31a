"""The learned smoothness gate on the GPU, through the C ABI.

- The gated scheme (a fixed gate, the same bytes on both sides) against the
  oracle's gated scheme: bit for bit in FP64.
- The training-sample kernels (features and WENO-IS weight deviation of every
  midpoint) against the oracle's stencil sample.
- The training kernels: the FP32 back-propagated gradient and Adam steps
  against the oracle's FP64 ones; the bfloat16 tensor-core inference and the
  FP32 forward pass against the oracle's forward passes; the gate kernel's
  decisions against the oracle's features through the oracle's network.
- End to end: training on the method's own stencils, and the ablation (what
  the gate changes in speed and error on the shock-water-column workload).
"""
import math

import numpy as np
import pytest

from oracle import mlp
from paper_2208_04488_gb300 import problems as P
from paper_2208_04488_gb300.metrics import rel_l1_state

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def hrm():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2208_04488_gb300 import build
    build.build()
    from paper_2208_04488_gb300 import hrm as H
    return H


def face_counts(pr):
    return [int(np.prod([pr.n[e] + (e == d) for e in range(pr.D)])) for d in range(pr.D)]


def random_gates(pr, seed, p=0.5):
    rng = np.random.default_rng(seed)
    return [(rng.uniform(size=nf) < p).astype(np.uint8) for nf in face_counts(pr)]


def oracle_state(orc, pr, steps):
    """(fluid, grid, W) after `steps` automatic-dt oracle steps."""
    f, g, W = orc.setup(pr)
    prm = orc.make_params()
    for _ in range(steps):
        dt, _ = orc.dt(f, g, W, pr.cfl)
        W = orc.step(f, prm, g, W, dt, 1)
    return f, g, W


GATE_PROBLEMS = [P.shock_tube_1d_baseline(64), P.shock_bubble_2d(40, 21), P.shock_water_column_2d(48, 26),
                 P.interface_3d(12)]


@pytest.mark.parametrize("pr", GATE_PROBLEMS, ids=[p.name for p in GATE_PROBLEMS])
def test_fixed_gate_scheme_bit_exact(hrm, orc, pr):
    """A fixed random gate (half of the midpoints gated) on both sides: the
    gated RHS and three gated SSP-RK3 steps agree bit for bit."""
    import torch
    f, g, W = orc.setup(pr)
    gates = random_gates(pr, 11)
    prm = hrm.params_default(cfl=pr.cfl)
    s = hrm.Solver.from_problem(pr, prm)
    for d in range(pr.D):
        s.set_gate(d, gates[d])
    prm.learned = hrm.LEARNED_FIXED
    s.set_params(prm)
    op = orc.make_params()
    lam = [2e-4, 3e-4, 1e-4][:pr.D]
    R = torch.empty((pr.M, pr.ncells), dtype=torch.float64, device="cuda")
    s.rhs(lam, R)
    R_or = orc.rhs(f, op, g, W, lam, gates=gates)
    np.testing.assert_array_equal(R.cpu().numpy(), R_or)
    # the gate changed something
    assert np.any(orc.rhs(f, op, g, W, lam) != R_or)
    dt, _ = orc.dt(f, g, W, pr.cfl)
    W3 = orc.step(f, op, g, W, dt, 3, gates=gates)
    s.step(dt, 3)
    np.testing.assert_array_equal(s.get(hrm.FIELD_W), W3)


def _node_cells(pr, d, t):
    """Cell indices of the six stencil nodes of midpoints t of direction d
    (periodic or clamped; a Dirichlet node keeps the clamped cell here and is
    replaced by its boundary slice in _stencil_inputs)."""
    ext = list(pr.n) + [1] * (3 - pr.D)
    fe = [ext[e] + (e == d) for e in range(3)]
    q = [t % fe[0], (t // fe[0]) % fe[1], t // (fe[0] * fe[1])]
    out = []
    for j in range(6):
        r = [q[0].copy(), q[1].copy(), q[2].copy()]
        jj = q[d] - 3 + j
        nn = ext[d]
        per_lo, per_hi = pr.bc[2 * d] == 1, pr.bc[2 * d + 1] == 1
        jj = np.where(jj < 0, jj + nn if per_lo else 0, jj)
        jj = np.where(jj >= nn, jj - nn if per_hi else nn - 1, jj)
        r[d] = jj
        out.append((r[2] * ext[1] + r[1]) * ext[0] + r[0])
    return np.stack(out, axis=1)


def _stencil_inputs(orc, pr, f, W, d):
    """The gate's five inputs (alpha_1, alpha_2, rho, u_d, p) at the six nodes of
    every midpoint of direction d, (n_faces, 6) each (None for an absent volume
    fraction): interior cells, and for a node beyond a Dirichlet side the cell of
    that side's boundary slice continuing the line (oracle values only)."""
    def per_cell(Wc):
        V = np.stack([orc.prim_cell(f, Wc[:, c])[0] for c in range(Wc.shape[1])], axis=1)
        al = [V[pr.N + pr.D + 1 + k] if pr.N > 1 + k else None for k in range(2)]
        return al + [Wc[:pr.N].sum(axis=0), V[pr.N + d], V[pr.N + pr.D]]
    inner = per_cell(W)
    bnd = {b: per_cell(orc.ic_from_prim(f, prim)) for b, prim in getattr(pr, "boundary", {}).items()}
    t = np.arange(face_counts(pr)[d])
    cells = _node_cells(pr, d, t)
    ext = list(pr.n) + [1] * (3 - pr.D)
    fe = [ext[e] + (e == d) for e in range(3)]
    q = [t % fe[0], (t // fe[0]) % fe[1], t // (fe[0] * fe[1])]
    sl, stride = np.zeros_like(t), 1  # slice cell: the other indices, lowest fastest
    for e in range(pr.D):
        if e != d:
            sl, stride = sl + q[e] * stride, stride * ext[e]
    out = []
    for a, arr in enumerate(inner):
        if arr is None:
            out.append(None)
            continue
        v = arr[cells]
        for j in range(6):
            jj = q[d] - 3 + j
            for side, beyond in ((0, jj < 0), (1, jj >= ext[d])):
                if pr.bc[2 * d + side] == 2 and beyond.any():
                    v[beyond, j] = bnd[2 * d + side][a][sl[beyond]]
        out.append(v)
    return out


COLLECT_PROBLEMS = [P.shock_tube_1d_baseline(64), P.shock_bubble_2d(40, 21), P.interface_3d(12)]


@pytest.mark.parametrize("pr", COLLECT_PROBLEMS, ids=[p.name for p in COLLECT_PROBLEMS])
def test_collect_matches_oracle(hrm, orc, pr):
    """Every midpoint kept: the GPU samples (direction by direction, in index
    order) carry the oracle's weight deviation and label, and its features up
    to the FP32 rounding of the inputs the gate reads."""
    f, g, W = oracle_state(orc, pr, 3)
    s = hrm.Solver.from_problem(pr, hrm.params_default(cfl=pr.cfl, check=0), set_state=False)
    s.set(W)
    det = hrm.Detector(capacity=sum(face_counts(pr)), seed=5)
    added = det.collect(s, 0.01, 1.0, 1.0, 1.0)
    assert added == sum(face_counts(pr)) == det.size()
    X, y, dv = det.samples()
    op = orc.make_params()
    off = 0
    for d, nf in enumerate(face_counts(pr)):
        idx = np.arange(nf)
        F_or, dev_or = orc.stencil_sample(f, op, g, W, d, idx)
        sl = slice(off, off + nf)
        np.testing.assert_allclose(dv[sl], dev_or.astype(np.float32), rtol=1e-6, atol=1e-30)
        clear = np.abs(dev_or - 0.01) > 1e-9
        np.testing.assert_array_equal(y[sl][clear], (dev_or < 0.01)[clear].astype(np.float32))
        # node values of the gate's inputs (alpha_1, alpha_2, rho, u_d, p) for the tolerance
        qs = _stencil_inputs(orc, pr, f, W, d)
        for a in range(5):
            got = X[sl, 6 * a:6 * a + 6].astype(np.float64)
            ref = F_or[:, 6 * a:6 * a + 6]
            if qs[a] is None:
                assert np.all(got == 0.0)
                continue
            qv = qs[a]
            rng_ = qv.max(axis=1) - qv.min(axis=1)
            mag = np.abs(qv).max(axis=1)
            # every input carries its FP32 rounding residue: ~2^-48 of its magnitude
            tol = 2e-5 + 4e-13 * mag / np.maximum(rng_, 1e-300)
            bad = np.abs(got - ref) > tol[:, None]
            assert not bad.any(), (d, a, np.argwhere(bad)[:3], got[bad][:3], ref[bad][:3])
        off += nf


def fp32_sensitive(orc, pr, f, W, d):
    """Midpoints of direction d where a stencil input (alpha_1, alpha_2, rho,
    u_d, p) varies by less than 1e-10 of its magnitude: there even the
    residue-carrying FP32 inputs of the gate (2^-48 of the magnitude) visibly
    round the normalised features (oracle values only)."""
    sens = np.zeros(face_counts(pr)[d], dtype=bool)
    for qv in _stencil_inputs(orc, pr, f, W, d):
        if qv is None:
            continue
        r = qv.max(axis=1) - qv.min(axis=1)
        sens |= (r > 0) & (r < 1e-10 * np.abs(qv).max(axis=1))
    return sens


def fp32_level(orc, pr, f, W, d):
    """Midpoints of direction d where every stencil input (alpha_1, alpha_2,
    rho, u_d, p) varies by at most 2^-21 of its magnitude (a few FP32 units in
    the last place) or stays below the smallest normal float (a velocity of
    1e-51 rounds to 0): the stencils whose FP32 planes can all be equal, which
    the precision form's sweep takes as uniform (oracle values only)."""
    flat = np.ones(face_counts(pr)[d], dtype=bool)
    for qv in _stencil_inputs(orc, pr, f, W, d):
        if qv is None:
            continue
        mag = np.abs(qv).max(axis=1)
        flat &= ((qv.max(axis=1) - qv.min(axis=1)) <= 2.0 ** -21 * mag) | (mag < 2.0 ** -126)
    return flat


def _random_set(seed, n=1000):
    rng = np.random.default_rng(seed)
    theta = rng.normal(0.0, 0.3, mlp.NPARAM).astype(np.float32)
    X = rng.uniform(-1.0, 1.0, (n, mlp.NIN)).astype(np.float32)
    y = (rng.uniform(size=n) < 0.4).astype(np.float32)
    return theta, X, y


def test_gradient_matches_oracle(hrm):
    """FP32 forward + back-propagation kernels against the FP64 oracle gradient
    (sum over 1000 samples, parameter block by block)."""
    theta, X, y = _random_set(3)
    det = hrm.Detector(capacity=2000, seed=1)
    det.set_weights(theta)
    det.add_samples(X, y)
    g, loss = det.gradient(0, 1000)
    t64, X64, y64 = theta.astype(np.float64), X.astype(np.float64), y.astype(np.float64)
    g_ref = mlp.grad(t64, X64, y64)
    assert loss == pytest.approx(mlp.loss(t64, X64, y64), rel=1e-5)
    for lo, hi in ((0, 960), (960, 992), (992, 2016), (2016, 2048), (2048, 2080), (2080, 2081)):
        num = np.linalg.norm(g[lo:hi] - g_ref[lo:hi])
        assert num <= 2e-5 * np.linalg.norm(g_ref[lo:hi]) + 1e-6, (lo, hi)
    # a sub-range
    g2, _ = det.gradient(100, 300)
    g2_ref = mlp.grad(t64, X64[100:400], y64[100:400])
    assert np.linalg.norm(g2 - g2_ref) <= 2e-5 * np.linalg.norm(g2_ref)


def test_adam_full_batch_matches_oracle(hrm):
    """Three full-batch Adam steps: the batch-mean losses before each step and
    the weights after them, against the oracle's FP64 gradient and Adam update
    (parameters with a gradient below FP32 resolution only within one step)."""
    theta, X, y = _random_set(4, n=512)
    det = hrm.Detector(capacity=512, seed=1)
    det.set_weights(theta)
    det.add_samples(X, y)
    lr = 1e-3
    losses = det.train(3, batch=0, lr=lr)
    th = theta.astype(np.float64)
    m = np.zeros_like(th)
    v = np.zeros_like(th)
    X64, y64 = X.astype(np.float64), y.astype(np.float64)
    gmin = np.full_like(th, np.inf)
    for t in range(1, 4):
        assert losses[t - 1] == pytest.approx(mlp.loss(th, X64, y64) / 512, rel=1e-5)
        gr = mlp.grad(th, X64, y64) / 512
        gmin = np.minimum(gmin, np.abs(gr))
        th, m, v = mlp.adam_step(th, m, v, gr, t, lr)
    got = det.get_weights().astype(np.float64)
    firm = gmin > 1e-4
    assert firm.mean() > 0.5
    np.testing.assert_allclose(got[firm], th[firm], atol=2e-6, rtol=0)
    assert np.all(np.abs(got - th) <= 3 * 2 * lr)


def test_logits_match_oracle(hrm):
    """Inference on the tensor cores (bfloat16 operands, FP32 accumulation)
    against the oracle's bfloat16 arithmetic with exact accumulation; the FP32
    training forward pass against the FP64 one."""
    theta, X, y = _random_set(6, n=4099)
    det = hrm.Detector(capacity=4099, seed=1)
    det.set_weights(theta)
    det.add_samples(X, y)
    t64, X64 = theta.astype(np.float64), X.astype(np.float64)
    z32 = det.logits(bf16=False)
    np.testing.assert_allclose(z32, mlp.forward(t64, X64)[1][5], rtol=1e-5, atol=1e-5)
    z16 = det.logits(bf16=True)
    ref = mlp.forward_bf16(t64, X64)
    err = np.abs(z16 - ref)
    # a hidden value may round to the other neighbouring bfloat16 when FP32
    # accumulation puts it on the other side of a rounding boundary
    assert np.mean(err <= 1e-4 * (1 + np.abs(ref))) > 0.99
    assert np.all(err <= 3e-2 * (1 + np.abs(ref)))
    # a ragged sub-range (not a multiple of the 32-row tiles)
    np.testing.assert_array_equal(det.logits(17, 45, bf16=True), z16[17:62])


# 48 x 26 and the others: stencil planes staged by TMA (rows a multiple of 16
# bytes); 50 x 26: the direct-load path of the same kernel; the jet: two
# species in 2D with a Dirichlet side (boundary slices after the interior cells)
TC_GATE_PROBLEMS = [P.shock_tube_1d_baseline(64), P.shock_water_column_2d(48, 26), P.shock_water_column_2d(50, 26),
                    P.interface_3d(12), P.mach100_jet_2d(48, 24)]


@pytest.mark.parametrize("pr", TC_GATE_PROBLEMS, ids=[f"{p.name}_{p.n[0]}" for p in TC_GATE_PROBLEMS])
def test_gate_kernel_matches_oracle(hrm, orc, pr):
    """Gate bytes of the network against the oracle's features through the
    oracle's bfloat16 network, at a threshold that gates about half of the
    non-uniform midpoints: equal wherever the oracle's logit is not within
    rounding distance of the threshold and the stencil's variation is not at
    rounding level; and the learned RHS equals the RHS with those bytes as a
    fixed gate. FP64: the tensor-core gate kernel (1D with two species and one
    partial 128-midpoint tile, 2D, 3D; stencil planes staged by TMA and read
    directly). FP32: the network inside the screened sweep (warp-level MMA),
    whose uniform stencils (every FP32 plane equal at the six nodes) take byte 2
    (the exact node flux)."""
    import torch
    f, g, W = oracle_state(orc, pr, 2)
    theta, _, _ = _random_set(8)
    op = orc.make_params()
    feats = [orc.stencil_sample(f, op, g, W, d, np.arange(nf))[0] for d, nf in enumerate(face_counts(pr))]
    zs = [mlp.forward_bf16(theta.astype(np.float64), F) for F in feats]
    # a threshold at the median logit of the non-uniform stencils, kept away
    # from the logit every uniform stencil shares
    zall = np.concatenate(zs)
    flat = np.concatenate([np.all(F == 0.0, axis=1) for F in feats])
    zthr = float(np.median(zall[~flat]))
    if flat.any() and abs(zall[flat][0] - zthr) < 0.2:
        zthr = float(zall[flat][0]) + 0.2 * np.sign(zthr - zall[flat][0] + 1e-300)
    thr = 1.0 / (1.0 + math.exp(-zthr))
    det = hrm.Detector(capacity=16, seed=1)
    det.set_weights(theta)
    s = hrm.Solver.from_problem(pr, hrm.params_default(cfl=pr.cfl), set_state=False)
    s.set(W)
    s.set_detector(det)
    for precision in (hrm.FP64, hrm.FP32):
        s.set_params(hrm.params_default(cfl=pr.cfl, precision=precision, learned=hrm.LEARNED_GATE,
                                        learned_threshold=thr))
        lam = [2e-4, 3e-4, 2.5e-4][:pr.D]
        R1 = torch.empty((pr.M, pr.ncells), dtype=torch.float64, device="cuda")
        s.rhs(lam, R1)
        gates = []
        for d in range(pr.D):
            gg = s.get_gate(d)
            z = zs[d]
            flat = np.all(feats[d] == 0.0, axis=1)
            uni = gg == 2
            if precision == hrm.FP64:
                assert not uni.any()
            assert fp32_level(orc, pr, f, W, d)[uni].all()
            firm = (np.abs(z - zthr) > 0.05 * (1 + np.abs(z))) & ~fp32_sensitive(orc, pr, f, W, d) & ~uni
            # enough compared midpoints (FP32: among the non-uniform ones, many of
            # which lie at the threshold or vary at rounding level)
            if precision == hrm.FP64:
                assert firm.mean() > 0.4
            else:
                assert firm.sum() >= 0.1 * (~uni).sum(), (int(firm.sum()), int((~uni).sum()))
            np.testing.assert_array_equal(gg[firm], (z[firm] > zthr).astype(np.uint8))
            rough = ~flat
            if rough.sum() >= 20:
                assert 0.05 < (gg[rough] == 1).mean() < 0.95
            gates.append(gg)
        for d in range(pr.D):
            s.set_gate(d, gates[d])
        s.set_params(hrm.params_default(cfl=pr.cfl, precision=precision, learned=hrm.LEARNED_FIXED))
        R2 = torch.empty_like(R1)
        s.rhs(lam, R2)
        assert torch.equal(R1, R2)


def test_learned_params_validation(hrm):
    pr = P.shock_tube_1d_baseline(32)
    s = hrm.Solver.from_problem(pr)
    with pytest.raises(hrm.HrmError):
        s.set_params(hrm.params_default(learned=hrm.LEARNED_GATE))      # no detector
    with pytest.raises(hrm.HrmError):
        s.set_params(hrm.params_default(learned=hrm.LEARNED_FIXED))     # no gate
    det = hrm.Detector(capacity=0, seed=1)
    s.set_detector(det)
    with pytest.raises(hrm.HrmError):
        s.set_params(hrm.params_default(learned=hrm.LEARNED_GATE, learned_threshold=1.0))
    with pytest.raises(hrm.HrmError):
        s.set_params(hrm.params_default(learned=hrm.LEARNED_GATE, scheme=1))
    s.set_params(hrm.params_default(learned=hrm.LEARNED_GATE, learned_threshold=0.9))
    s.step(0.0, 2)
    assert s.admissibility() == [0, 0, 0, 0]
    with pytest.raises(hrm.HrmError):
        det.train(1, 16, 1e-3)  # no samples


@pytest.fixture(scope="module")
def trained(hrm):
    from paper_2208_04488_gb300 import learned
    det, rep = learned.build_detector(scale="small", steps=3000, capacity=1 << 21)
    return det, rep


def test_training_on_method_stencils(hrm, trained):
    """Trained on stencils of the method's own runs (shock tube, shock-bubble,
    3D interface, smooth periodic advection): the loss falls, the set holds both classes, and the
    tensor-core inference classifies the training midpoints with few
    smooth-predictions on rough stencils."""
    det, rep = trained
    assert rep.samples > 20000 and 0.05 < rep.rough / rep.samples < 0.95
    assert rep.losses[-200:].mean() < 0.5 * rep.losses[:20].mean()
    ev = det.evaluate(0.5, bf16=True)
    n = ev["tp"] + ev["fp"] + ev["tn"] + ev["fn"]
    assert n == rep.samples
    acc = (ev["tp"] + ev["tn"]) / n
    fpr = ev["fp"] / max(1, ev["fp"] + ev["tn"])
    print(f"\ntraining set: {n} samples, accuracy {acc:.4f}, rough-as-smooth rate {fpr:.4f}, "
          f"collect {rep.collect_s:.1f} s, train {rep.train_s:.2f} s ({rep.steps} Adam steps)")
    assert acc > 0.9 and fpr < 0.1


def _run(hrm, pr, precision, learned_mode, det, dt, steps, threshold=0.5):
    prm = hrm.params_default(cfl=pr.cfl, precision=precision, check=0)
    s = hrm.Solver.from_problem(pr, prm)
    if learned_mode:
        s.set_detector(det)
        s.set_params(hrm.params_default(cfl=pr.cfl, precision=precision, check=0, learned=hrm.LEARNED_GATE,
                                        learned_threshold=threshold))
    s.set_profiling(True)
    s.step(dt, steps)
    prof = s.profile_read()
    # the sweeps of a stage run concurrently: their common bracket (kind 7)
    face_ms = sum(ms for k, ms in prof if k == hrm.KERNEL_SWEEPS)
    gate_ms = sum(ms for k, ms in prof if k == 6)
    frac = None
    if learned_mode:  # gated: linear weights (1) or, in the precision form, a uniform stencil (2)
        frac = float(np.mean(np.concatenate([s.get_gate(d) for d in range(pr.D)]) != 0))
    W = s.get(hrm.FIELD_W)
    adm = s.admissibility()
    s.close()
    return W, face_ms, gate_ms, frac, adm


def _ablation(hrm, det, pr, steps, label):
    s0 = hrm.Solver.from_problem(pr, hrm.params_default(cfl=pr.cfl))
    dt, _ = s0.dt(pr.cfl)
    s0.close()
    ref, f64_ms, _, _, ref_adm = _run(hrm, pr, hrm.FP64, 0, det, dt, steps)
    rows = {}
    for name, prec, lm in (("fp32", hrm.FP32, 0), ("fp32+learned", hrm.FP32, 1), ("fp64+learned", hrm.FP64, 1)):
        W, fms, gms, frac, adm = _run(hrm, pr, prec, lm, det, dt, steps)
        err = float(np.max(rel_l1_state(W, ref, pr.N, pr.D)))
        rows[name] = (fms, gms, frac, err, adm)
    print(f"\nablation, {label}, {steps} steps, last-step midpoint kernels:")
    print(f"  fp64            face {f64_ms:.3f} ms  admissibility {ref_adm}")
    for k, (fms, gms, frac, err, adm) in rows.items():
        print(f"  {k:15s} face {fms:.3f} ms  gate {gms:.3f} ms  gated {frac if frac is not None else 0:.3f}  "
              f"rel L1 vs fp64 {err:.3e}  admissibility {adm}")
    assert ref_adm == [0, 0, 0, 0]
    for k, (fms, gms, frac, err, adm) in rows.items():
        assert adm == [0, 0, 0, 0], k
        assert err < 1e-3, k
    return f64_ms, rows


def test_ablation_shock_water_column(hrm, trained):
    """What the trained gate changes on the shock-water-column workload (a
    problem it was not trained on), 512 x 256, 20 equal steps: the share of
    gated midpoints, the midpoint-kernel time per step with and without it, and
    the state error against plain FP64 -- for the precision form and for FP64.
    Most of its midpoints are constant stencils, which every interpolation
    returns exactly without weights, so the gate saves little here; the
    timings are reported, not asserted."""
    det, _ = trained
    _, rows = _ablation(hrm, det, P.shock_water_column_2d(512, 256), 20, "shock-water column 512x256")
    assert rows["fp64+learned"][2] > 0.3


def test_ablation_smooth_advection(hrm, trained):
    """The gate where the flow is smooth but not constant: the periodic
    advection of Sec. 5.2 (a sine in alpha, constant u, v, p) at 512 x 512.
    The volume-fraction and partial-density fields vary at every midpoint, the
    detector gates most of them, and in FP64 -- where the WENO-IS weights are
    the dominant work -- the gated sweep with the gate kernel is faster than
    the plain one, at a small error against plain FP64."""
    det, _ = trained
    f64_ms, rows = _ablation(hrm, det, P.advection_2d_smooth(512), 20, "smooth advection 512x512")
    assert rows["fp64+learned"][2] > 0.5
    assert rows["fp64+learned"][0] + rows["fp64+learned"][1] < f64_ms


def test_bounded_tensor_core_wait_reports_timeout(hrm):
    """The bounded mbarrier wait of the tensor-core kernels, on a phase that
    nothing completes: every thread's wait runs out within its limit, the call
    returns HRM_E_TIMEOUT, and the device stays usable."""
    import time
    t0 = time.time()
    st, expired = hrm.probe_wait_timeout()
    assert st == hrm.HRM_E_TIMEOUT
    assert expired == 128
    assert time.time() - t0 < 30.0
    assert hrm.probe_fma_peak(hrm.FP32, iters=256) > 0.0
