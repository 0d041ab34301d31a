"""The bounds-check build (HRM_BOUNDS_CHECK=1): every midpoint's node indices
and every cell's midpoint indices are checked against their arrays while
problems covering every dimension, boundary type (Dirichlet slices included),
both forms, the learned gate's fixed path and the first-order scheme are
stepped; no index may fall outside. Runs in a child process, which builds and
loads the checked library."""
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r"""
import json, sys
import numpy as np
sys.path.insert(0, ROOT)
from paper_2208_04488_gb300 import build, hrm, problems as P
build.build()
out = {}
cases = [P.shock_tube_1d_baseline(37), P.shock_bubble_2d(41, 23), P.interface_3d(12), P.dirichlet_box([13]),
         P.dirichlet_box([11, 9]), P.dirichlet_box([7, 6, 5]), P.mach100_jet_2d(48, 24), P.undex_2d(30, 38)]
for pr in cases:
    for prec in (hrm.FP64, hrm.FP32):
        for extra in ({}, {"scheme": 1}):
            s = hrm.Solver.from_problem(pr, params=hrm.params_default(cfl=0.4, check=0, precision=prec, **extra))
            s.step(0.0, 3)
            if not extra:
                for d in range(pr.D):
                    s.set_gate(d, (np.arange(s.face_count(d)) % 3 == 0).astype(np.uint8))
                s.set_params(hrm.params_default(cfl=0.4, check=0, precision=prec, learned=hrm.LEARNED_FIXED))
                s.step(0.0, 2)
            for field in range(9):
                s.get(field)
            out[f"{pr.name}_{'x'.join(map(str, pr.n))}_{prec}_{'hllc' if extra else 'wcns'}"] = s.bounds_violations()
            s.close()
print(json.dumps(out))
"""


def test_bounds_check_build_meets_no_out_of_range_index():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    env = dict(os.environ, HRM_BOUNDS_CHECK="1")
    r = subprocess.run([sys.executable, "-c", f"ROOT = {ROOT!r}\n" + CHILD], env=env, capture_output=True, text=True,
                       timeout=900)
    assert r.returncode == 0, r.stderr[-3000:]
    counts = json.loads(r.stdout.strip().splitlines()[-1])
    assert counts and all(v == 0 for v in counts.values()), counts
