"""The precision form's persistent step (hrm_set_step_path 1: three persistent
stage launches per step over one context) against the captured graph of
per-phase kernels (path 0): the same states bit for bit, with the CFL step and
with a fixed step, three launches per step, and phase times for profiling."""
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


def _run(H, pr, path, dt, nsteps, **kw):
    s = H.Solver.from_problem(pr, params=H.params_default(cfl=pr.cfl, check=1, precision=H.FP32, **kw))
    s.set_step_path(path)
    s.step(dt, nsteps)
    out = (s.get(H.FIELD_W), s.time(), s.step_launches())
    s.close()
    return out


@pytest.mark.parametrize("pr", [P.shock_bubble_2d(96, 48), P.shock_water_column_2d(160, 80)],
                         ids=["shock_bubble_96x48", "water_column_160x80"])
@pytest.mark.parametrize("fixed_dt", [False, True])
def test_persistent_step_equals_per_phase_graph(hrm, pr, fixed_dt):
    dt = 0.0
    if fixed_dt:
        s = hrm.Solver.from_problem(pr, params=hrm.params_default(cfl=pr.cfl, check=0, precision=hrm.FP32))
        dt = 0.8 * s.dt(pr.cfl)[0]
        s.close()
    W1, t1, k1 = _run(hrm, pr, 1, dt, 10)
    W0, t0, k0 = _run(hrm, pr, 0, dt, 10)
    assert k1 == 3 and k0 > 3
    np.testing.assert_array_equal(W1, W0)
    assert t1 == t0


def test_persistent_step_relax_modes_and_profile(hrm):
    pr = P.shock_bubble_2d(64, 32)
    for mode in (0, 2):
        W1, _, _ = _run(hrm, pr, 1, 0.0, 4, relax_mode=mode)
        W0, _, _ = _run(hrm, pr, 0, 0.0, 4, relax_mode=mode)
        np.testing.assert_array_equal(W1, W0)
    s = hrm.Solver.from_problem(pr, params=hrm.params_default(cfl=pr.cfl, check=0, precision=hrm.FP32))
    s.set_step_path(1)
    s.set_profiling(True)
    s.step(0.0, 2)
    assert s.step_launches() == 3
    prof = s.profile_read()
    kinds = [k for k, _ in prof]
    assert kinds.count(hrm.KERNEL_SWEEPS) == 3 and kinds.count(hrm.KERNEL_UPDATE) == 3
    assert all(ms >= 0.0 for _, ms in prof) and sum(ms for _, ms in prof) > 0.0
    s.close()
