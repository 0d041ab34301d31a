"""Host logic of bench.py (no GPU): the concurrent sweeps of a stage are timed
by their common bracket, shared among their launches, and the time shares leave
out the sweeps' own (overlapping) brackets; the method's flops per midpoint over
a run are counted on its first and last state."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


@pytest.fixture(scope="module")
def mods():
    import bench
    from paper_2208_04488_gb300 import hrm
    return bench, hrm


def test_sweeps_bracket_is_the_sweep_time(mods):
    bench, hrm = mods
    # 3 stages x 2 directions: each sweep's own bracket 2 ms (running beside the
    # other), the common bracket 3 ms per stage
    per = {hrm.KERNEL_PRIM: (3, 0.3e-3), hrm.KERNEL_FACE_X: (3, 6e-3), hrm.KERNEL_FACE_Y: (3, 6e-3),
           hrm.KERNEL_SWEEPS: (3, 9e-3), hrm.KERNEL_UPDATE: (3, 0.6e-3)}
    n, t = bench.sweep_time(hrm, per, 2)
    assert n == 6 and t == pytest.approx(9e-3)
    sh = bench.time_shares(hrm, per, 2)
    assert set(sh) == {"prim", "sweeps", "update"}
    assert sum(sh.values()) == pytest.approx(1.0, abs=1e-3)
    assert sh["sweeps"] == pytest.approx(9.0 / 9.9, abs=1e-4)


def test_without_a_sweeps_bracket_the_launches_add(mods):
    bench, hrm = mods
    per = {hrm.KERNEL_PRIM: (3, 0.3e-3), hrm.KERNEL_FACE_X: (3, 6e-3), hrm.KERNEL_UPDATE: (3, 0.6e-3)}
    n, t = bench.sweep_time(hrm, per, 1)
    assert n == 3 and t == pytest.approx(6e-3)
    sh = bench.time_shares(hrm, per, 1)
    assert set(sh) == {"prim", "face_x", "update"}
    assert sum(sh.values()) == pytest.approx(1.0, abs=1e-3)


def test_run_face_flops_means_the_first_and_last_state(mods):
    """The method's flops per midpoint over a run are the mean of the oracle's
    counts on the initial state and on the run's last state: a state with more
    non-uniform stencils costs more (uniform stencils cost only the node flux)."""
    bench, _ = mods
    import oracle
    from paper_2208_04488_gb300 import problems as P
    pr = P.shock_bubble_2d(64, 32)
    f, g, W0 = oracle.setup(pr)
    same = bench.run_face_flops(pr, pr.cfl, W0)
    first = bench.algorithmic_face_flops(pr, pr.cfl)
    for d in range(pr.D):
        assert same[d][0] == pytest.approx(first[d][0]) and same[d][1] == first[d][1]
    p = oracle.make_params()
    W = W0
    for _ in range(3):
        dt, _ = oracle.dt(f, g, W, pr.cfl)
        W = oracle.step(f, p, g, W, dt, 1)
    run = bench.run_face_flops(pr, pr.cfl, W)
    last = bench.algorithmic_face_flops(pr, pr.cfl, W)
    for d in range(pr.D):
        assert run[d][0] == pytest.approx(0.5 * (first[d][0] + last[d][0]))
        assert last[d][0] > first[d][0]
