"""Batched form: many uneven 2D instances, one persistent launch per RK stage.

Each batched instance must reproduce the single-problem context of the same
problem bit for bit, in FP64 and in the precision form (same per-element
arithmetic, same rounding), whatever the launch shape; a step is three
launches; the autotuner must leave the states untouched; the grid barrier's
bounded wait reports a barrier that cannot complete as HRM_E_TIMEOUT."""
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
    prm = hrm.params_default(cfl=0.4, check=1, precision=prec)
    b = hrm.BatchSolver(ps, params=prm)
    k0 = b.kernel_launches()
    b.step(4)
    # one persistent launch per stage, and with params.check one admissibility
    # kernel per instance after the steps
    assert b.kernel_launches() - k0 == 4 * 3 + len(ps)
    for i, pr in enumerate(ps):
        s = hrm.Solver.from_problem(pr, params=hrm.params_default(cfl=0.4, check=0, precision=prec))
        s.step(0.0, 4)
        np.testing.assert_array_equal(b.get(i), s.get(hrm.FIELD_W))
        assert b.time(i) == s.time()
        s.close()
    assert b.admissibility() == [0, 0, 0, 0]


def test_batch_state_written_between_steps(hrm):
    """The precision form leaves out the cells a stage returns unchanged only
    while W^n came out of its own relaxation; writing an instance's state
    (hrm_batch_set with a state that was not relaxed, hrm_batch_set_primitive)
    withdraws that for the instance. A batch and single contexts given the same
    writes between steps agree bit for bit."""
    ps = _problems()
    prm = hrm.params_default(cfl=0.4, check=0, precision=hrm.FP32)
    b = hrm.BatchSolver(ps, params=prm)
    ss = [hrm.Solver.from_problem(pr, params=prm) for pr in ps]
    b.step(2)
    for s in ss:
        s.step(0.0, 2)
    # instance 0: a set-up state of another time (not relaxed by the form);
    # instance 1: its primitives again
    W0 = hrm.Solver.from_problem(ps[0], params=prm)
    Wset = W0.get(hrm.FIELD_W)
    W0.close()
    b.set(0, Wset)
    ss[0].set(Wset)
    b.set_primitive(1, ps[1].prim)
    ss[1].set_primitive(ps[1].prim)
    b.step(3)
    for i, s in enumerate(ss):
        s.step(0.0, 3)
        np.testing.assert_array_equal(b.get(i), s.get(hrm.FIELD_W))
        s.close()


def test_batch_launch_shape_does_not_change_results(hrm):
    ps = _problems()
    prm = hrm.params_default(cfl=0.4, check=0)
    outs = []
    for shape in [(128, 128, 4096, 2), (128, 128, 256, 1), (128, 128, 65536, 0)]:
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
    assert best["cell_tile"] in (1024, 4096, 16384) and best["blocks_per_sm"] >= 1
    for i in range(len(ps)):
        np.testing.assert_array_equal(b.get(i), before[i])
        assert b.time(i) == t_before[i]


def test_bounded_grid_barrier_reports_timeout(hrm):
    """A grid barrier that nothing completes (it counts one block more than
    run) ends every wait within its limit; the probe returns HRM_E_TIMEOUT and
    the device keeps working."""
    st, expired = hrm.probe_barrier_timeout(50.0)
    assert st == hrm.HRM_E_TIMEOUT and expired == 4
    ps = _problems()[:2]
    b = hrm.BatchSolver(ps, params=hrm.params_default(cfl=0.4, check=1))
    b.step(1)
    assert b.admissibility() == [0, 0, 0, 0]


def test_batch_rejects_invalid_instances(hrm):
    with pytest.raises(hrm.HrmError):
        hrm.BatchSolver([P.shock_tube_1d_baseline(32)])  # 1D: the batched form is 2D
