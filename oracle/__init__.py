"""TEST INFRASTRUCTURE -- the serial FP64 CPU oracle of the PP-WCNS-IS fractional
algorithm (Wong, Angel & Kiris, arXiv 2208.04488).

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline leg
may import this package. It is independent of the CUDA library: it shares no
source, header, constant table or helper with ``paper_2208_04488_gb300``, and
the product path never calls it.

The arithmetic lives in ``hrm_oracle.cpp`` (plain C++17, serial, FP64,
``-O2 -ffp-contract=off``); this module only builds and loads it with ctypes.
A second build (``-DOR_COUNT``) counts the floating-point operations the
method performs, which the roofline figures use as algorithmic work.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "hrm_oracle.cpp")
_BUILD = os.path.join(_HERE, "_build")
_LOCK = threading.Lock()

MAXN = 4


def _lib_path(count) -> str:
    name = {False: "liboracle.so", True: "liboracle_count.so", "omp": "liboracle_omp.so"}[count]
    return os.path.join(_BUILD, name)


def build(force: bool = False) -> None:
    """Compile the oracle shared libraries with gcc (seconds): serial, counting,
    and (where the compiler has OpenMP) the multi-threaded build."""
    os.makedirs(_BUILD, exist_ok=True)
    for count in (False, True, "omp"):
        out = _lib_path(count)
        if not force and os.path.exists(out) and os.path.getmtime(out) >= os.path.getmtime(_SRC):
            continue
        cmd = ["g++", "-std=c++17", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
               "-shared", _SRC, "-o", out + ".tmp"]
        if count is True:
            cmd.insert(1, "-DOR_COUNT")
        if count == "omp":
            cmd[1:1] = ["-DOR_OMP", "-fopenmp"]
            if subprocess.run(cmd, capture_output=True).returncode != 0:
                continue  # no OpenMP: the serial build serves
        else:
            subprocess.run(cmd, check=True)
        os.replace(out + ".tmp", out)


def has_omp() -> bool:
    build()
    return os.path.exists(_lib_path("omp"))


class Fluid(ctypes.Structure):
    _fields_ = [("N", ctypes.c_int32), ("D", ctypes.c_int32), ("liq", ctypes.c_int32),
                ("pad", ctypes.c_int32),
                ("gamma", ctypes.c_double * MAXN), ("pinf", ctypes.c_double * MAXN),
                ("cv", ctypes.c_double * MAXN), ("q", ctypes.c_double * MAXN)]


class Params(ctypes.Structure):
    _fields_ = [("limiters", ctypes.c_int32), ("blend", ctypes.c_int32),
                ("relax_mode", ctypes.c_int32), ("scheme", ctypes.c_int32),
                ("integrator", ctypes.c_int32), ("cfl_sound", ctypes.c_int32),
                ("pad1", ctypes.c_int32), ("pad2", ctypes.c_int32),
                ("eps_ar", ctypes.c_double), ("eps_a", ctypes.c_double),
                ("eps_rhoe", ctypes.c_double), ("hs_ar", ctypes.c_double),
                ("hs_a", ctypes.c_double), ("hs_rc2", ctypes.c_double),
                ("hs_rhoe", ctypes.c_double), ("weno_eps", ctypes.c_double),
                ("Cs", ctypes.c_double), ("q_sensor", ctypes.c_double)]


class Grid(ctypes.Structure):
    _fields_ = [("D", ctypes.c_int32), ("pad", ctypes.c_int32),
                ("n", ctypes.c_int64 * 3), ("dx", ctypes.c_double * 3),
                ("bc", ctypes.c_int32 * 6), ("bnd", ctypes.c_void_p * 6)]


_DP = ctypes.POINTER(ctypes.c_double)
_libs: dict = {}


def lib(count: bool = False):
    with _LOCK:
        if count in _libs:
            return _libs[count]
        path = _lib_path(count)
        if not os.path.exists(path) or os.path.getmtime(path) < os.path.getmtime(_SRC):
            build()
        L = ctypes.CDLL(path)
        P = ctypes.POINTER
        L.or_params_default.argtypes = [P(Params)]
        L.or_prim_cell.argtypes = [P(Fluid), _DP, _DP, _DP]
        L.or_cons_cell.argtypes = [P(Fluid), _DP, _DP, _DP]
        L.or_weno_left.argtypes = [_DP, ctypes.c_double, _DP]
        L.or_weno_left.restype = ctypes.c_double
        L.or_weno_lin.argtypes = [_DP]
        L.or_weno_lin.restype = ctypes.c_double
        L.or_hllc.argtypes = [P(Fluid), ctypes.c_int, _DP, _DP, _DP]
        L.or_hllc.restype = ctypes.c_double
        L.or_sensor.argtypes = [_DP]
        L.or_sensor.restype = ctypes.c_double
        L.or_face.argtypes = [P(Fluid), P(Params), ctypes.c_int, ctypes.c_double, _DP, _DP, _DP, _DP]
        L.or_rhs.argtypes = [P(Fluid), P(Params), P(Grid), _DP, _DP, _DP]
        L.or_interp_limit.argtypes = [P(Fluid), P(Params), _DP, _DP]
        L.or_interp_limit.restype = ctypes.c_int
        L.or_flux_limit.argtypes = [P(Fluid), P(Params), ctypes.c_int, ctypes.c_double, _DP, _DP, _DP, _DP,
                                    _DP, _DP]
        L.or_flux_limit.restype = ctypes.c_int
        L.or_char_matrices.argtypes = [P(Fluid), ctypes.c_int, _DP, _DP, _DP, _DP, _DP]
        _U8 = ctypes.POINTER(ctypes.c_uint8)
        L.or_rhs_gated.argtypes = [P(Fluid), P(Params), P(Grid), _DP, _DP, _U8, _U8, _U8, _DP]
        L.or_step_gated.argtypes = [P(Fluid), P(Params), P(Grid), _DP, ctypes.c_double, ctypes.c_int,
                                    _U8, _U8, _U8]
        L.or_stencil_sample.argtypes = [P(Fluid), P(Params), P(Grid), _DP, ctypes.c_int, ctypes.c_int64,
                                        P(ctypes.c_int64), _DP, _DP]
        L.or_relax_cell.argtypes = [P(Fluid), _DP, _DP]
        L.or_relax.argtypes = [P(Fluid), P(Grid), _DP]
        L.or_dt.argtypes = [P(Fluid), P(Grid), _DP, ctypes.c_double, _DP]
        L.or_dt.restype = ctypes.c_double
        L.or_dt_sound.argtypes = [P(Fluid), P(Grid), _DP, ctypes.c_double, ctypes.c_int, _DP]
        L.or_dt_sound.restype = ctypes.c_double
        L.or_lambdas.argtypes = [P(Fluid), P(Grid), _DP, ctypes.c_double, _DP]
        L.or_step.argtypes = [P(Fluid), P(Params), P(Grid), _DP, ctypes.c_double, ctypes.c_int]
        L.or_admissibility.argtypes = [P(Fluid), P(Grid), _DP, P(ctypes.c_int64)]
        L.or_c4eq_cell.argtypes = [P(Fluid), _DP, _DP]
        L.or_ic_from_prim.argtypes = [P(Fluid), ctypes.c_int64, _DP, _DP]
        L.or_tanh.argtypes = [ctypes.c_double]
        L.or_tanh.restype = ctypes.c_double
        L.or_faces_flops.argtypes = [P(Fluid), P(Params), P(Grid), _DP, _DP, ctypes.c_int, _DP]
        L.or_faces_flops.restype = ctypes.c_int64
        L.or_faces_flops_gated.argtypes = [P(Fluid), P(Params), P(Grid), _DP, _DP, ctypes.c_int, ctypes.c_int,
                                           _DP]
        L.or_faces_flops_gated.restype = ctypes.c_int64
        if count is True:
            L.or_count_reset.argtypes = []
            L.or_count_get.argtypes = [P(ctypes.c_ulonglong)]
        L.or_step_exact.argtypes = [P(Fluid), P(Params), P(Grid), _DP, ctypes.c_double, ctypes.c_int,
                                    ctypes.c_double, _DP]
        L.or_threads.argtypes = []
        L.or_threads.restype = ctypes.c_int
        _libs[count] = L
        return L


def _ptr(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(_DP)


# ---------------------------------------------------------------- descriptions

def make_fluid(gamma, pinf, cv, q=None, D=1, liq=None) -> Fluid:
    n = len(gamma)
    assert 1 <= n <= MAXN
    f = Fluid()
    f.N, f.D = n, D
    if liq is None:
        liq = next((k for k in range(n) if pinf[k] > 0), 0)
    f.liq = liq
    for k in range(n):
        f.gamma[k] = gamma[k]
        f.pinf[k] = pinf[k]
        f.cv[k] = cv[k]
        f.q[k] = 0.0 if q is None else q[k]
    return f


def make_params(**kw) -> Params:
    p = Params()
    lib().or_params_default(ctypes.byref(p))
    for k, v in kw.items():
        setattr(p, k, v)
    return p


def make_grid(n, dx, bc=None, bnd=None) -> Grid:
    """bnd (optional): {side b = 2 d + s: W of the boundary slice, (M, cells of
    the side)} for the Dirichlet sides (bc 2)."""
    g = Grid()
    g.D = len(n)
    for d in range(3):
        g.n[d] = n[d] if d < len(n) else 1
        g.dx[d] = dx[d] if d < len(n) else 1.0
    bc = bc or [0] * (2 * len(n))
    for i in range(6):
        g.bc[i] = bc[i] if i < len(bc) else 0
    g._keep = {}
    for b, Wb in (bnd or {}).items():
        Wb = np.ascontiguousarray(Wb, dtype=np.float64)
        g._keep[b] = Wb
        g.bnd[b] = Wb.ctypes.data
    return g


def fluid_dict(f: Fluid) -> dict:
    return {"gamma": list(f.gamma)[:f.N], "pinf": list(f.pinf)[:f.N],
            "cv": list(f.cv)[:f.N], "q": list(f.q)[:f.N], "D": f.D, "liq": f.liq}


# ---------------------------------------------------------------- calls

def prim_cell(f: Fluid, W):
    W = np.ascontiguousarray(W, dtype=np.float64)
    M = 2 * f.N + f.D
    V = np.zeros(M)
    out = np.zeros(4)
    lib().or_prim_cell(ctypes.byref(f), _ptr(W), _ptr(V), _ptr(out))
    return V, {"rho": out[0], "c": out[1], "rc2": out[2], "rhoe": out[3]}


def cons_cell(f: Fluid, V):
    V = np.ascontiguousarray(V, dtype=np.float64)
    W = np.zeros_like(V)
    out = np.zeros(3)
    lib().or_cons_cell(ctypes.byref(f), _ptr(V), _ptr(W), _ptr(out))
    return W, {"rho": out[0], "c": out[1], "E": out[2]}


def weno_left(u, eps=1e-15):
    u = np.ascontiguousarray(u, dtype=np.float64)
    om = np.zeros(4)
    v = lib().or_weno_left(_ptr(u), eps, _ptr(om))
    return v, om


def weno_lin(u):
    """Left-biased interpolation with the linear weights d_k (the gated value)."""
    u = np.ascontiguousarray(u, dtype=np.float64)
    return lib().or_weno_lin(_ptr(u))


def hllc(f: Fluid, dir_, VL, VR):
    VL = np.ascontiguousarray(VL, dtype=np.float64)
    VR = np.ascontiguousarray(VR, dtype=np.float64)
    G = np.zeros_like(VL)
    s = lib().or_hllc(ctypes.byref(f), dir_, _ptr(VL), _ptr(VR), _ptr(G))
    return G, s


def sensor(u6):
    u6 = np.ascontiguousarray(u6, dtype=np.float64)
    return lib().or_sensor(_ptr(u6))


def face(f: Fluid, p: Params, dir_, lam, W6):
    W6 = np.ascontiguousarray(W6, dtype=np.float64)
    M = 2 * f.N + f.D
    assert W6.shape == (6, M)
    Gm = np.zeros(M)
    Gp = np.zeros(M)
    diag = np.zeros(8 * M + 8)
    lib().or_face(ctypes.byref(f), ctypes.byref(p), dir_, lam, _ptr(W6), _ptr(Gm), _ptr(Gp), _ptr(diag))
    names = ["VL_weno", "VR_weno", "VL", "VR", "Gt", "GH", "Ghcs"]
    d = {nm: diag[i * M:(i + 1) * M].copy() for i, nm in enumerate(names)}
    t = diag[7 * M:]
    d.update(ut=t[0], uH=t[1], uhcs=t[2], sig=t[3], hsL=int(t[4]), hsR=int(t[5]), flux_flags=int(t[6]))
    return Gm, Gp, d


def interp_limit(f: Fluid, p: Params, Vt, Wnode):
    """The interpolation limiter on one biased midpoint state: returns the
    limited primitive vector and whether the hard switch fired."""
    V = np.array(Vt, dtype=np.float64)
    Wn = np.ascontiguousarray(Wnode, dtype=np.float64)
    hs = lib().or_interp_limit(ctypes.byref(f), ctypes.byref(p), _ptr(V), _ptr(Wn))
    return V, hs


def flux_limit(f: Fluid, p: Params, dir_, lam, Wi, Wj, Gm, Gp, Hm, Hp):
    """The flux limiter of one midpoint: returns the limited G^-, G^+ and the
    flag mask (1 first stage, 2 energy stage, 4 hard switch)."""
    c = lambda a: np.ascontiguousarray(a, dtype=np.float64)
    Wi, Wj, Hm, Hp = c(Wi), c(Wj), c(Hm), c(Hp)
    gm, gp = np.array(Gm, dtype=np.float64), np.array(Gp, dtype=np.float64)
    flags = lib().or_flux_limit(ctypes.byref(f), ctypes.byref(p), dir_, lam, _ptr(Wi), _ptr(Wj), _ptr(gm),
                                _ptr(gp), _ptr(Hm), _ptr(Hp))
    return gm, gp, flags


def char_matrices(f: Fluid, dir_, Wi, Wj):
    """R^{-1} and R of a midpoint as the oracle applies them, and the averaged
    state (alpha_k rho_k, rho, c) they are built from."""
    M = 2 * f.N + f.D
    Wi = np.ascontiguousarray(Wi, dtype=np.float64)
    Wj = np.ascontiguousarray(Wj, dtype=np.float64)
    Rinv = np.zeros((M, M))
    R = np.zeros((M, M))
    avg = np.zeros(f.N + 2)
    lib().or_char_matrices(ctypes.byref(f), dir_, _ptr(Wi), _ptr(Wj), _ptr(Rinv), _ptr(R), _ptr(avg))
    return Rinv, R, avg


def _gate_ptrs(g: Grid, gates):
    """Per-direction byte arrays over each direction's midpoint grid (or None)."""
    keep, ptrs = [], []
    for d in range(3):
        a = None if gates is None or d >= len(gates) else gates[d]
        if a is None:
            ptrs.append(None)
            continue
        nf = 1
        for e in range(g.D):
            nf *= g.n[e] + (e == d)
        a = np.ascontiguousarray(a, dtype=np.uint8).reshape(-1)
        assert a.size == nf, (a.size, nf)
        keep.append(a)
        ptrs.append(a.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)))
    return keep, ptrs


def rhs(f: Fluid, p: Params, g: Grid, W, lam, gates=None):
    """L(W) with the given lambdas; `gates` (optional): per direction, a byte
    per midpoint (nonzero = linear WENO weights there)."""
    W = np.ascontiguousarray(W, dtype=np.float64)
    R = np.zeros_like(W)
    lam = np.ascontiguousarray(np.resize(np.asarray(lam, dtype=np.float64), 3))
    keep, gp = _gate_ptrs(g, gates)
    lib().or_rhs_gated(ctypes.byref(f), ctypes.byref(p), ctypes.byref(g), _ptr(W), _ptr(lam),
                       gp[0], gp[1], gp[2], _ptr(R))
    return R


def stencil_sample(f: Fluid, p: Params, g: Grid, W, dir_, idx):
    """Learned-detector data of midpoints `idx` of direction `dir_`: the 30
    normalised stencil features (n, 30) and the WENO-IS weight deviation (n,)."""
    W = np.ascontiguousarray(W, dtype=np.float64)
    idx = np.ascontiguousarray(idx, dtype=np.int64)
    feat = np.zeros((idx.size, 30))
    dev = np.zeros(idx.size)
    lib().or_stencil_sample(ctypes.byref(f), ctypes.byref(p), ctypes.byref(g), _ptr(W), dir_, idx.size,
                            idx.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), _ptr(feat), _ptr(dev))
    return feat, dev


def relax_cell(f: Fluid, W):
    W = np.array(W, dtype=np.float64)
    pT = np.zeros(2)
    lib().or_relax_cell(ctypes.byref(f), _ptr(W), _ptr(pT))
    return W, pT[0], pT[1]


def relax(f: Fluid, g: Grid, W):
    W = np.array(W, dtype=np.float64, order="C")
    lib().or_relax(ctypes.byref(f), ctypes.byref(g), _ptr(W))
    return W


def dt(f: Fluid, g: Grid, W, cfl, sound=0):
    """CFL step and tau_d; sound 1: the four-equation HRM sound speed in the
    wave speeds (Eq. 4_eqn_sos) instead of the five-equation one."""
    W = np.ascontiguousarray(W, dtype=np.float64)
    tau = np.zeros(3)
    d = lib().or_dt_sound(ctypes.byref(f), ctypes.byref(g), _ptr(W), cfl, int(sound), _ptr(tau))
    return d, tau[:g.D].copy()


def lambdas(f: Fluid, g: Grid, W, dt_):
    W = np.ascontiguousarray(W, dtype=np.float64)
    lam = np.zeros(3)
    lib().or_lambdas(ctypes.byref(f), ctypes.byref(g), _ptr(W), dt_, _ptr(lam))
    return lam


def threads(omp: bool = False) -> int:
    """Host threads the oracle's sweeps use (the OpenMP build: all available)."""
    return int(lib("omp" if omp and has_omp() else False).or_threads())


def step(f: Fluid, p: Params, g: Grid, W, dt_, nsteps=1, count=False, gates=None, omp=False):
    """nsteps steps of size dt_. omp: the multi-threaded build (same results)."""
    W = np.array(W, dtype=np.float64, order="C")
    L = lib("omp" if omp and not count and has_omp() else count)
    if count:
        L.or_count_reset()
    if gates is not None:
        keep, gp = _gate_ptrs(g, gates)
        L.or_step_gated(ctypes.byref(f), ctypes.byref(p), ctypes.byref(g), _ptr(W), dt_, nsteps,
                        gp[0], gp[1], gp[2])
    else:
        L.or_step(ctypes.byref(f), ctypes.byref(p), ctypes.byref(g), _ptr(W), dt_, nsteps)
    if count:
        out = (ctypes.c_ulonglong * 5)()
        L.or_count_get(out)
        return W, {"add": out[0], "mul": out[1], "div": out[2], "sqrt": out[3], "tanh": out[4]}
    return W


def step_exact(f: Fluid, p: Params, g: Grid, W, dt_, nsteps, t0, adv):
    """Steps with the exact-derivative right-hand side of the Sec. 5.1 temporal
    test; adv = (a0, a1, k, u, p, rho_1, rho_2, x0)."""
    W = np.array(W, dtype=np.float64, order="C")
    a = np.ascontiguousarray(adv, dtype=np.float64)
    lib().or_step_exact(ctypes.byref(f), ctypes.byref(p), ctypes.byref(g), _ptr(W), dt_, nsteps, t0, _ptr(a))
    return W


def admissibility(f: Fluid, g: Grid, W):
    W = np.ascontiguousarray(W, dtype=np.float64)
    c = (ctypes.c_int64 * 4)()
    lib().or_admissibility(ctypes.byref(f), ctypes.byref(g), _ptr(W), c)
    return [int(x) for x in c]


def c4eq_cell(f: Fluid, W):
    W = np.ascontiguousarray(W, dtype=np.float64)
    out = np.zeros(4 + MAXN)
    lib().or_c4eq_cell(ctypes.byref(f), _ptr(W), _ptr(out))
    return {"c4": out[0], "p": out[1], "T": out[2], "Gamma": out[3], "Psi": out[4:4 + f.N].copy()}


def ic_from_prim(f: Fluid, prim):
    """Conservative initial state W[M, ncells] from primitive planes
    (alpha_1..alpha_{N-1}, u_d, p, T) in p-T equilibrium."""
    prim = np.ascontiguousarray(prim, dtype=np.float64)
    nc = prim.shape[1]
    W = np.zeros((2 * f.N + f.D, nc))
    lib().or_ic_from_prim(ctypes.byref(f), nc, _ptr(prim), _ptr(W))
    return W


def setup(problem):
    """Oracle descriptions (fluid, grid) and the initial W of a problem from
    paper_2208_04488_gb300.problems."""
    f = make_fluid(problem.gamma, problem.pinf, problem.cv, problem.q, D=problem.D, liq=problem.liq)
    bnd = {b: ic_from_prim(f, prim) for b, prim in getattr(problem, "boundary", {}).items()}
    g = make_grid(problem.n, problem.dx, problem.bc, bnd)
    return f, g, ic_from_prim(f, problem.prim)


def faces_flops(f: Fluid, p: Params, g: Grid, W, lam, dir_, gated=False):
    """Algorithmic operation counts of the midpoint computations of one
    direction (counting build): (counts dict, number of faces). gated: every
    midpoint with the linear WENO weights."""
    W = np.ascontiguousarray(W, dtype=np.float64)
    lam = np.ascontiguousarray(np.resize(np.asarray(lam, dtype=np.float64), 3))
    out = np.zeros(5)
    nf = lib(True).or_faces_flops_gated(ctypes.byref(f), ctypes.byref(p), ctypes.byref(g), _ptr(W), _ptr(lam),
                                        dir_, 1 if gated else 0, _ptr(out))
    return dict(zip(["add", "mul", "div", "sqrt", "tanh"], out.tolist())), nf


def tanh(x: float) -> float:
    """The oracle's explicit tanh (Cody-Waite reduction and Taylor series)."""
    return lib().or_tanh(float(x))
