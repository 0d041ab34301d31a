"""Batched form: many uneven 2D instances in one persistent launch per phase.

Each batched instance must reproduce the single-problem context of the same
problem: bit for bit in FP64 (same per-element arithmetic, same rounding),
whatever the launch shape, and to the precision form's rounding in FP32; the
autotuner must leave the states untouched."""
import numpy as np
import pytest

from paper_2208_04488_gb300 import problems as P

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


def _problems():
    ps = P.batch_instances(count=6, scale=16, seed=7)
    ps.append(P.shock_bubble_2d(48, 24))
    ps.append(P.advection_2d_smooth(16))
    return ps


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_batch_reproduces_single_contexts(hrm, precision):
    prec = hrm.FP64 if precision == "fp64" else hrm.FP32
    ps = _problems()
    assert {p.N for p in ps} == {2, 3}
    prm = hrm.params_default(cfl=0.4, check=0, precision=prec)
    b = hrm.BatchSolver(ps, params=prm)
    b.step(4)
    for i, pr in enumerate(ps):
        s = hrm.Solver.from_problem(pr, params=prm)
        s.step(0.0, 4)
        Wb, Ws = b.get(i), s.get(hrm.FIELD_W)
        if precision == "fp64":
            np.testing.assert_array_equal(Wb, Ws)
        else:
            # the batched precision form runs the same screened body in its own
            # kernels, whose FP32 contraction may differ: the two agree to the
            # precision form's rounding, and the batch is as close to FP64 as the
            # single context is
            from paper_2208_04488_gb300.metrics import rel_l1_state
            assert rel_l1_state(Wb, Ws, pr.N, pr.D).max() <= 1e-7
            s64 = hrm.Solver.from_problem(pr, params=hrm.params_default(cfl=0.4, check=0))
            for _ in range(4):
                dt, _ = s64.dt(0.4)
                s64.step(dt, 1)
            W64 = s64.get(hrm.FIELD_W)
            e_batch = rel_l1_state(Wb, W64, pr.N, pr.D).max()
            e_single = rel_l1_state(Ws, W64, pr.N, pr.D).max()
            assert e_batch <= 2.0 * e_single + 1e-9, (e_batch, e_single)
        if precision == "fp64":
            assert b.time(i) == s.time()
        else:
            (tb, nb), (ts, ns) = b.time(i), s.time()
            assert nb == ns and tb == pytest.approx(ts, rel=1e-6)
    assert b.admissibility() == [0, 0, 0, 0]


def test_batch_launch_shape_does_not_change_results(hrm):
    ps = _problems()
    prm = hrm.params_default(cfl=0.4, check=0)
    outs = []
    for shape in [(128, 128, 4096, 2), (64, 512, 256, 8), (256, 16384, 65536, 1)]:
        b = hrm.BatchSolver(ps, params=prm)
        b.set_launch(*shape)
        b.step(2)
        outs.append([b.get(i) for i in range(len(ps))])
    for o in outs[1:]:
        for a, c in zip(outs[0], o):
            np.testing.assert_array_equal(a, c)


def test_autotuner_restores_states_and_picks_a_candidate(hrm):
    ps = _problems()
    prm = hrm.params_default(cfl=0.4, check=0, precision=hrm.FP32)
    b = hrm.BatchSolver(ps, params=prm)
    b.step(1)
    before = [b.get(i) for i in range(len(ps))]
    t_before = [b.time(i) for i in range(len(ps))]
    best = b.tune(1)
    assert best["face_threads"] in (64, 128, 256) and best["blocks_per_sm"] in (1, 2, 4, 8)
    for i in range(len(ps)):
        np.testing.assert_array_equal(b.get(i), before[i])
        assert b.time(i) == t_before[i]


def test_batch_rejects_invalid_instances(hrm):
    with pytest.raises(hrm.HrmError):
        hrm.BatchSolver([P.shock_tube_1d_baseline(32)])  # 1D: the batched form is 2D
