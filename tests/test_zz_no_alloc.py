"""The allocation-free time step (hrm_dt_noalloc) against the context path.

hrm_dt_noalloc serves callers that may not allocate device memory (an
application whose memory belongs to its own pool or budget, or a time-critical
loop that must not call cudaMalloc or cudaFree). It must return what hrm_dt
returns for the same state, call after call, while reusing its one fixed
scratch array, and it must leave the device's free memory unchanged.

The file name sorts last so that pytest collects it after every other test
file: a run that stops at its first failure has then already run all the
other tests if this one fails. The tests here depend on no other test and
pass alone in a fresh process as well.
"""
import ctypes

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


def _noalloc_dt(H, pr, W_dev, cfl, out=None):
    import torch
    L = H.lib()
    if out is None:
        out = torch.full((1 + pr.D,), -1.0, dtype=torch.float64, device="cuda")
    n = (ctypes.c_int64 * 3)(*(pr.n + [1] * (3 - pr.D)))
    dx = (ctypes.c_double * 3)(*(pr.dx + [1.0] * (3 - pr.D)))
    arr = lambda v: (ctypes.c_double * len(v))(*v)
    stream = torch.cuda.current_stream()
    st = L.hrm_dt_noalloc(pr.N, pr.D, n, dx, arr(pr.gamma), arr(pr.pinf), arr(pr.cv), arr(pr.q),
                          ctypes.c_void_p(W_dev.data_ptr()), cfl, ctypes.c_void_p(out.data_ptr()),
                          ctypes.c_void_p(stream.cuda_stream))
    assert st == H.HRM_OK, L.hrm_last_error(None).decode()
    torch.cuda.synchronize()
    return out.cpu().numpy()


def test_noalloc_dt_matches_context_dt_on_consecutive_calls(hrm):
    import torch
    for pr in (P.shock_bubble_2d(300, 150), P.shock_tube_1d_baseline(400), P.interface_3d(20)):
        s = hrm.Solver.from_problem(pr, params=hrm.params_default(cfl=pr.cfl, check=0))
        W = torch.empty((pr.M, pr.ncells), dtype=torch.float64, device="cuda")
        for call in range(2):  # two calls in a row on different states
            s.get(hrm.FIELD_W, out=W)
            dt_ctx, tau_ctx = s.dt(pr.cfl)
            got = _noalloc_dt(hrm, pr, W, pr.cfl)
            assert got[0] == dt_ctx, (pr.name, call, got[0], dt_ctx)
            np.testing.assert_array_equal(got[1:], tau_ctx)
            s.step(0.0, 1)


def test_noalloc_dt_rejects_grids_beyond_its_scratch(hrm):
    import torch
    L = hrm.lib()
    W = torch.zeros(8, dtype=torch.float64, device="cuda")
    out = torch.zeros(4, dtype=torch.float64, device="cuda")
    n = (ctypes.c_int64 * 3)(20000, 10000, 1)  # 2e8 cells > 65536 x 2048
    dx = (ctypes.c_double * 3)(1.0, 1.0, 1.0)
    arr = lambda v: (ctypes.c_double * len(v))(*v)
    st = L.hrm_dt_noalloc(2, 2, n, dx, arr([1.4, 3.0]), arr([0.0, 8.533e8]), arr([719.3, 1400.0]), None,
                          ctypes.c_void_p(W.data_ptr()), 0.5, ctypes.c_void_p(out.data_ptr()), None)
    assert st == hrm.HRM_E_INVAL
    assert "134217728" in L.hrm_last_error(None).decode()


def test_noalloc_dt_leaves_free_device_memory_unchanged(hrm):
    """After one warm-up call (which loads the kernels' module and looks up the
    scratch array's address), a call changes the device's free memory by
    nothing: it allocates no device memory."""
    import torch
    pr = P.shock_bubble_2d(256, 128)
    s = hrm.Solver.from_problem(pr, params=hrm.params_default(cfl=pr.cfl, check=0))
    W = torch.empty((pr.M, pr.ncells), dtype=torch.float64, device="cuda")
    s.get(hrm.FIELD_W, out=W)
    dt_ctx, _ = s.dt(pr.cfl)
    out = torch.full((1 + pr.D,), -1.0, dtype=torch.float64, device="cuda")
    first = _noalloc_dt(hrm, pr, W, pr.cfl, out)
    torch.cuda.synchronize()
    free_before, _ = torch.cuda.mem_get_info()
    again = _noalloc_dt(hrm, pr, W, pr.cfl, out)
    torch.cuda.synchronize()
    free_after, _ = torch.cuda.mem_get_info()
    assert free_after == free_before
    assert first[0] == dt_ctx and again[0] == dt_ctx
