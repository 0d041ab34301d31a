"""Host-side checks of the C ABI that need no GPU: the library loads, exports
every function include/hrm.h declares, fills the paper's constants, and
rejects invalid species tables before touching the device."""
import ctypes

import pytest


@pytest.fixture(scope="module")
def H():
    from paper_2208_04488_gb300 import build
    build.build()
    from paper_2208_04488_gb300 import hrm
    return hrm


def test_exports_every_declared_symbol(H):
    names = H.declared_functions()
    assert len(names) >= 15
    L = ctypes.CDLL(H.LIB_PATH)
    for n in names:
        assert hasattr(L, n), n


def test_params_default_are_the_papers_constants(H):
    p = H.params_default()
    assert (p.eps_ar, p.eps_a, p.eps_rhoe) == (1e-10, 1e-10, 1e-8)       # Sec. 4.3.2
    assert (p.hs_ar, p.hs_a, p.hs_rc2, p.hs_rhoe) == (1e-11, 1e-11, 1e-9, 1e-9)
    assert p.weno_eps == 1e-15                                          # App. C
    assert (p.Cs, p.q_sensor) == (1e12, 2.0)                            # Sec. 4.3.1
    assert p.cfl == 0.5 and p.limiters == 1 and p.blend == 1 and p.relax_mode == 1


@pytest.mark.parametrize("kw,msg", [
    (dict(gamma=[1.4, 0.9]), "gamma"),
    (dict(pinf=[1e9, 8e8]), "stiffened"),
    (dict(cv=[700.0, -1.0]), "c_v"),
    (dict(N=5), "nspecies"),
])
def test_create_rejects_invalid_tables(H, kw, msg):
    N = kw.get("N", 2)
    gamma = kw.get("gamma", [1.4, 3.0] + [1.5] * (N - 2))
    pinf = kw.get("pinf", [0.0, 8e8] + [0.0] * (N - 2))
    cv = kw.get("cv", [700.0, 1400.0] + [800.0] * (N - 2))
    L = H.lib()
    g = H.HrmGrid()
    g.ndim = 1
    g.n[0], g.n[1], g.n[2] = 10, 1, 1
    g.hi[0] = 1.0
    p = H.params_default()
    h = ctypes.c_void_p()
    arr = lambda v: (ctypes.c_double * len(v))(*v)
    st = L.hrm_create(ctypes.byref(h), ctypes.byref(g), N, arr(gamma), arr(pinf), arr(cv), None,
                      ctypes.byref(p), None)
    assert st == H.HRM_E_INVAL
    assert not h.value
    assert msg in L.hrm_last_error(None).decode()


def test_binding_raises_without_library(H, monkeypatch, tmp_path):
    """The product path has no CPU fallback: a missing library is an error."""
    monkeypatch.setattr(H, "_lib", None)
    monkeypatch.setattr(H, "LIB_PATH", str(tmp_path / "missing.so"))
    with pytest.raises(RuntimeError, match="no CPU fallback"):
        H.lib()
