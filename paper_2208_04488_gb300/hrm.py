"""Python binding of the C ABI in include/hrm.h (ctypes, argument marshalling
only). Every step of the method runs in the CUDA library; there is no CPU
path: a missing library raises.

Device buffers are passed as torch CUDA tensors (their data pointers), host
buffers as numpy arrays; the CUDA stream is torch's current stream unless one
is given.
"""
from __future__ import annotations

import ctypes
import os
import sys
import re
from typing import Optional

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build_check" if os.environ.get("HRM_BOUNDS_CHECK", "0") == "1" else "_build",
                        "libhrm.so")
HEADER = os.path.join(HERE, "..", "include", "hrm.h")

HRM_OK, HRM_E_INVAL, HRM_E_CUDA, HRM_E_ADMISSIBILITY, HRM_E_TIMEOUT, HRM_E_NOMEM = 0, -1, -2, -3, -4, -5
FIELD_W, FIELD_V, FIELD_C5, FIELD_PT, FIELD_C4, FIELD_PSI_GAMMA, FIELD_ALPHA, FIELD_Y = 0, 1, 2, 3, 4, 5, 6, 7
FIELD_SCHLIEREN = 8
FP64, FP32 = 0, 1
RK3, EULER, RK2 = 0, 1, 2
RELAX_OFF, RELAX_STAGE, RELAX_STEP = 0, 1, 2
KERNEL_PRIM, KERNEL_FINALIZE, KERNEL_FACE_X, KERNEL_FACE_Y, KERNEL_FACE_Z, KERNEL_UPDATE = 0, 1, 2, 3, 4, 5
KERNEL_GATE = 6
KERNEL_NAMES = {0: "prim", 1: "finalize", 2: "face_x", 3: "face_y", 4: "face_z", 5: "update", 6: "gate",
                7: "sweeps"}
KERNEL_SWEEPS = 7
LEARNED_OFF, LEARNED_GATE, LEARNED_FIXED = 0, 1, 2
BC_TRANSMISSIVE, BC_PERIODIC, BC_DIRICHLET = 0, 1, 2
DETECTOR_PARAMS, DETECTOR_INPUTS = 2081, 30


class HrmGrid(ctypes.Structure):
    _fields_ = [("ndim", ctypes.c_int32), ("pad", ctypes.c_int32), ("n", ctypes.c_int64 * 3),
                ("lo", ctypes.c_double * 3), ("hi", ctypes.c_double * 3), ("bc", ctypes.c_int32 * 6)]


class HrmParams(ctypes.Structure):
    _fields_ = [("cfl", ctypes.c_double),
                ("limiters", ctypes.c_int32), ("blend", ctypes.c_int32), ("relax_mode", ctypes.c_int32),
                ("scheme", ctypes.c_int32), ("integrator", ctypes.c_int32), ("precision", ctypes.c_int32),
                ("learned", ctypes.c_int32), ("check", ctypes.c_int32),
                ("eps_ar", ctypes.c_double), ("eps_a", ctypes.c_double), ("eps_rhoe", ctypes.c_double),
                ("hs_ar", ctypes.c_double), ("hs_a", ctypes.c_double), ("hs_rc2", ctypes.c_double),
                ("hs_rhoe", ctypes.c_double), ("weno_eps", ctypes.c_double), ("Cs", ctypes.c_double),
                ("q_sensor", ctypes.c_double), ("learned_threshold", ctypes.c_double),
                ("screen", ctypes.c_int32), ("cfl_sound", ctypes.c_int32)]


class HrmInstance(ctypes.Structure):
    _fields_ = [("grid", HrmGrid), ("nspecies", ctypes.c_int32), ("pad", ctypes.c_int32),
                ("gamma", ctypes.c_double * 4), ("p_inf", ctypes.c_double * 4), ("c_v", ctypes.c_double * 4),
                ("q", ctypes.c_double * 4)]


class HrmError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"hrm status {status}: {message}")
        self.status = status


_lib = None
_VP = ctypes.c_void_p
_DP = ctypes.POINTER(ctypes.c_double)


def declared_functions(header: str = HEADER):
    """Names of the functions declared in include/hrm.h."""
    txt = open(header).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(hrm_[a-z0-9_]+)\s*\(", txt)))


def lib():
    """The loaded library; raises if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"CUDA library not built ({LIB_PATH}); run "
                           "paper_2208_04488_gb300.build.build() -- there is no CPU fallback")
    L = ctypes.CDLL(LIB_PATH)
    P = ctypes.POINTER
    L.hrm_params_default.argtypes = [P(HrmParams)]
    L.hrm_params_default.restype = None
    L.hrm_create.argtypes = [P(_VP), P(HrmGrid), ctypes.c_int32, _DP, _DP, _DP, _DP, P(HrmParams), _VP]
    L.hrm_destroy.argtypes = [_VP]
    L.hrm_destroy.restype = None
    L.hrm_last_error.argtypes = [_VP]
    L.hrm_last_error.restype = ctypes.c_char_p
    L.hrm_set_params.argtypes = [_VP, P(HrmParams)]
    L.hrm_set.argtypes = [_VP, _VP, ctypes.c_int32]
    L.hrm_set_primitive.argtypes = [_VP, _VP, ctypes.c_int32]
    L.hrm_set_allocator.argtypes = [_VP, _VP, _VP]
    L.hrm_set_boundary.argtypes = [_VP, ctypes.c_int32, _VP, ctypes.c_int32, ctypes.c_int32]
    L.hrm_dt.argtypes = [_VP, ctypes.c_double, _DP, _DP]
    L.hrm_step.argtypes = [_VP, ctypes.c_double, ctypes.c_int32]
    L.hrm_relax.argtypes = [_VP]
    L.hrm_rhs.argtypes = [_VP, _DP, _VP]
    L.hrm_get.argtypes = [_VP, ctypes.c_int32, _VP, ctypes.c_int32]
    L.hrm_time.argtypes = [_VP, _DP, P(ctypes.c_int64)]
    L.hrm_bounds_violations.argtypes = [_VP]
    L.hrm_bounds_violations.restype = ctypes.c_int64
    L.hrm_set_time.argtypes = [_VP, ctypes.c_double, ctypes.c_int64]
    L.hrm_admissibility.argtypes = [_VP, P(ctypes.c_int64)]
    L.hrm_kernel_launches.argtypes = [_VP]
    L.hrm_kernel_launches.restype = ctypes.c_int64
    L.hrm_set_profiling.argtypes = [_VP, ctypes.c_int32]
    L.hrm_set_profiling.restype = ctypes.c_int
    L.hrm_profile_read.argtypes = [_VP, ctypes.c_int32, ctypes.POINTER(ctypes.c_float),
                                   ctypes.POINTER(ctypes.c_int32)]
    L.hrm_profile_read.restype = ctypes.c_int32
    L.hrm_dt_noalloc.argtypes = [ctypes.c_int32, ctypes.c_int32, ctypes.POINTER(ctypes.c_int64), _DP, _DP, _DP,
                                 _DP, _DP, _VP, ctypes.c_double, _VP, _VP]
    L.hrm_dt_noalloc.restype = ctypes.c_int
    L.hrm_batch_create.argtypes = [P(_VP), ctypes.c_int32, P(HrmInstance), P(HrmParams), _VP]
    L.hrm_batch_destroy.argtypes = [_VP]
    L.hrm_batch_destroy.restype = None
    L.hrm_batch_last_error.argtypes = [_VP]
    L.hrm_batch_last_error.restype = ctypes.c_char_p
    L.hrm_batch_set_primitive.argtypes = [_VP, ctypes.c_int32, _VP, ctypes.c_int32]
    L.hrm_batch_set.argtypes = [_VP, ctypes.c_int32, _VP, ctypes.c_int32]
    L.hrm_batch_get.argtypes = [_VP, ctypes.c_int32, _VP, ctypes.c_int32]
    L.hrm_batch_step.argtypes = [_VP, ctypes.c_int32]
    L.hrm_batch_time.argtypes = [_VP, ctypes.c_int32, _DP, P(ctypes.c_int64)]
    L.hrm_batch_admissibility.argtypes = [_VP, P(ctypes.c_int64)]
    L.hrm_batch_set_launch.argtypes = [_VP, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32]
    L.hrm_batch_tune.argtypes = [_VP, ctypes.c_int32, P(ctypes.c_int32)]
    L.hrm_batch_kernel_launches.argtypes = [_VP]
    L.hrm_batch_kernel_launches.restype = ctypes.c_int64
    L.hrm_batch_total_cells.argtypes = [_VP]
    L.hrm_batch_total_cells.restype = ctypes.c_int64
    for name in ("hrm_batch_create", "hrm_batch_set_primitive", "hrm_batch_set", "hrm_batch_get",
                 "hrm_batch_step", "hrm_batch_time", "hrm_batch_admissibility", "hrm_batch_set_launch",
                 "hrm_batch_tune"):
        getattr(L, name).restype = ctypes.c_int
    _FP = ctypes.POINTER(ctypes.c_float)
    _U8 = ctypes.POINTER(ctypes.c_uint8)
    _I64 = ctypes.POINTER(ctypes.c_int64)
    L.hrm_detector_create.argtypes = [P(_VP), ctypes.c_int64, ctypes.c_uint64, _VP]
    L.hrm_detector_destroy.argtypes = [_VP]
    L.hrm_detector_destroy.restype = None
    L.hrm_detector_last_error.argtypes = [_VP]
    L.hrm_detector_last_error.restype = ctypes.c_char_p
    L.hrm_detector_set_weights.argtypes = [_VP, _FP]
    L.hrm_detector_get_weights.argtypes = [_VP, _FP]
    L.hrm_detector_size.argtypes = [_VP]
    L.hrm_detector_size.restype = ctypes.c_int64
    L.hrm_detector_clear.argtypes = [_VP]
    L.hrm_detector_add_samples.argtypes = [_VP, _FP, _FP, ctypes.c_int64]
    L.hrm_detector_samples.argtypes = [_VP, ctypes.c_int64, ctypes.c_int64, _FP, _FP, _FP]
    L.hrm_detector_collect.argtypes = [_VP, _VP, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                       ctypes.c_double, _I64]
    L.hrm_detector_gradient.argtypes = [_VP, ctypes.c_int64, ctypes.c_int64, _FP, _DP]
    L.hrm_detector_train.argtypes = [_VP, ctypes.c_int32, ctypes.c_int32, ctypes.c_double, _FP]
    L.hrm_detector_logits.argtypes = [_VP, ctypes.c_int64, ctypes.c_int64, ctypes.c_int32, _FP]
    L.hrm_detector_evaluate.argtypes = [_VP, ctypes.c_double, ctypes.c_int32, _I64, _DP]
    L.hrm_set_detector.argtypes = [_VP, _VP]
    L.hrm_set_gate.argtypes = [_VP, ctypes.c_int32, _U8]
    L.hrm_get_gate.argtypes = [_VP, ctypes.c_int32, _U8]
    for name in ("hrm_detector_create", "hrm_detector_set_weights", "hrm_detector_get_weights",
                 "hrm_detector_clear", "hrm_detector_add_samples", "hrm_detector_samples", "hrm_detector_collect",
                 "hrm_detector_gradient", "hrm_detector_train", "hrm_detector_logits", "hrm_detector_evaluate",
                 "hrm_set_detector", "hrm_set_gate", "hrm_get_gate"):
        getattr(L, name).restype = ctypes.c_int
    L.hrm_probe_fma_peak.argtypes = [ctypes.c_int32, ctypes.c_int32, _VP, _DP]
    L.hrm_probe_fma_peak.restype = ctypes.c_int
    L.hrm_probe_wait_timeout.argtypes = [_VP, ctypes.POINTER(ctypes.c_int64)]
    L.hrm_probe_wait_timeout.restype = ctypes.c_int
    L.hrm_probe_convert.argtypes = [_VP, _VP, ctypes.c_int64, _VP, _VP, _VP]
    L.hrm_probe_convert.restype = ctypes.c_int
    L.hrm_probe_barrier_timeout.argtypes = [_VP, ctypes.c_double, ctypes.POINTER(ctypes.c_int64)]
    L.hrm_probe_barrier_timeout.restype = ctypes.c_int
    L.hrm_step_tau.argtypes = [_VP, _DP]
    L.hrm_begin_step.argtypes = [_VP, _DP, ctypes.c_double]
    L.hrm_stages.argtypes = [_VP]
    L.hrm_stages.restype = ctypes.c_int32
    L.hrm_stage.argtypes = [_VP, ctypes.c_int32]
    L.hrm_layers.argtypes = [_VP, ctypes.c_int32, ctypes.c_int32, ctypes.c_int64, ctypes.c_int64, _VP,
                             ctypes.c_int32]
    L.hrm_set_step_path.argtypes = [_VP, ctypes.c_int32]
    L.hrm_step_launches.argtypes = [_VP]
    L.hrm_step_launches.restype = ctypes.c_int32
    for name in ("hrm_step_tau", "hrm_begin_step", "hrm_stage", "hrm_layers", "hrm_set_step_path"):
        getattr(L, name).restype = ctypes.c_int
    for name in ("hrm_create", "hrm_set_params", "hrm_set", "hrm_set_primitive", "hrm_dt", "hrm_step",
                 "hrm_relax", "hrm_rhs", "hrm_get", "hrm_time", "hrm_admissibility"):
        getattr(L, name).restype = ctypes.c_int
    _lib = L
    return L


def probe_fma_peak(precision=FP64, iters=4096, stream=None) -> float:
    """Measured FMA-pipe throughput (flop/s) of the current device."""
    v = ctypes.c_double()
    st = lib().hrm_probe_fma_peak(precision, iters, _VP(_stream_handle(stream)), ctypes.byref(v))
    if st != HRM_OK:
        raise HrmError(st, "fma probe failed")
    return v.value


def probe_wait_timeout(stream=None):
    """(status, expired) of the bounded-wait probe: HRM_E_TIMEOUT and 128."""
    n = ctypes.c_int64()
    st = lib().hrm_probe_wait_timeout(_VP(_stream_handle(stream)), ctypes.byref(n))
    return st, n.value


def probe_barrier_timeout(limit_ms=50.0, stream=None):
    """(status, expired) of the grid-barrier probe: HRM_E_TIMEOUT and 4."""
    n = ctypes.c_int64()
    st = lib().hrm_probe_barrier_timeout(_VP(_stream_handle(stream)), float(limit_ms), ctypes.byref(n))
    return st, n.value


def probe_convert(in_d, in_f, stream=None):
    """The library's integer-pipe FP64 -> FP32 (nearest) and FP32 -> FP64
    conversions of two device tensors of equal length: (narrowed, widened)."""
    import torch
    assert in_d.dtype == torch.float64 and in_f.dtype == torch.float32 and in_d.numel() == in_f.numel()
    in_d, in_f = in_d.contiguous(), in_f.contiguous()
    narrowed = torch.empty_like(in_f)
    widened = torch.empty_like(in_d)
    st = lib().hrm_probe_convert(_VP(in_d.data_ptr()), _VP(in_f.data_ptr()), in_d.numel(),
                                 _VP(narrowed.data_ptr()), _VP(widened.data_ptr()), _VP(_stream_handle(stream)))
    if st != HRM_OK:
        raise HrmError(st, "conversion probe failed")
    return narrowed, widened


def params_default(**overrides) -> HrmParams:
    p = HrmParams()
    lib().hrm_params_default(ctypes.byref(p))
    for k, v in overrides.items():
        if not hasattr(p, k):
            raise AttributeError(k)
        setattr(p, k, v)
    return p


def _darr(values, n):
    a = (ctypes.c_double * n)()
    for i, v in enumerate(values):
        a[i] = float(v)
    return a


def _stream_handle(stream):
    if stream is not None:
        return int(stream) if isinstance(stream, int) else int(stream.cuda_stream)
    import torch
    return int(torch.cuda.current_stream().cuda_stream)


_ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)
_FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p)
_allocator_keep = None


def use_torch_allocator(on: bool = True):
    """Solvers created after this call take their device memory from PyTorch's
    caching allocator (on the solver's stream) instead of cudaMalloc; False
    restores cudaMalloc. Solvers keep the allocator they were created with."""
    global _allocator_keep
    if not on:
        lib().hrm_set_allocator(None, None, None)
        _allocator_keep = None
        return
    import torch

    def _alloc(nbytes, stream, user):
        try:
            return int(torch.cuda.caching_allocator_alloc(int(nbytes), stream=int(stream or 0)))
        except Exception:
            return None

    def _free(ptr, stream, user):
        torch.cuda.caching_allocator_delete(int(ptr))

    a, f = _ALLOC_FN(_alloc), _FREE_FN(_free)
    _allocator_keep = (a, f)
    st = lib().hrm_set_allocator(ctypes.cast(a, _VP), ctypes.cast(f, _VP), None)
    if st != HRM_OK:
        raise HrmError(st, "hrm_set_allocator")


class Solver:
    """One hrm_ctx: a problem's grid and species table on the GPU."""

    def __init__(self, n, lo, hi, bc, gamma, pinf, cv, q=None, params: Optional[HrmParams] = None,
                 stream=None):
        L = lib()
        self.N = len(gamma)
        self.D = len(n)
        self.M = 2 * self.N + self.D
        self.n = list(n)
        self.ncells = int(np.prod(n))
        g = HrmGrid()
        g.ndim = self.D
        for d in range(3):
            g.n[d] = n[d] if d < self.D else 1
            g.lo[d] = lo[d] if d < self.D else 0.0
            g.hi[d] = hi[d] if d < self.D else 1.0
        for i in range(6):
            g.bc[i] = bc[i] if i < len(bc) else 0
        self.grid = g
        self.params = params if params is not None else params_default()
        self.stream = _stream_handle(stream)
        h = _VP()
        st = L.hrm_create(ctypes.byref(h), ctypes.byref(g), self.N, _darr(gamma, self.N), _darr(pinf, self.N),
                          _darr(cv, self.N), None if q is None else _darr(q, self.N), ctypes.byref(self.params),
                          _VP(self.stream))
        if st != HRM_OK:
            raise HrmError(st, L.hrm_last_error(None).decode())
        self.h = h
        # the allocator callbacks this context returns its memory through
        self._allocator = _allocator_keep

    @classmethod
    def from_problem(cls, problem, params: Optional[HrmParams] = None, stream=None, set_state=True):
        s = cls(problem.n, problem.lo, problem.hi, problem.bc, problem.gamma, problem.pinf, problem.cv,
                problem.q, params=params, stream=stream)
        for b, prim in getattr(problem, "boundary", {}).items():
            s.set_boundary(b, prim, primitive=True)
        if set_state:
            s.set_primitive(problem.prim)
        return s

    # -- lifetime
    def close(self):
        if getattr(self, "h", None):
            lib().hrm_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            # at interpreter exit, memory from PyTorch's allocator is left to the
            # process teardown (the allocator may already be gone)
            if getattr(self, "_allocator", None) is not None and sys.is_finalizing():
                return
            self.close()
        except Exception:
            pass

    def _check(self, st):
        if st != HRM_OK:
            raise HrmError(st, lib().hrm_last_error(self.h).decode())
        return st

    # -- state
    @staticmethod
    def _ptr(a):
        """(pointer, on_device) of a numpy array or a torch tensor."""
        if isinstance(a, np.ndarray):
            assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
            return a.ctypes.data, 0
        assert a.dtype.__str__() == "torch.float64" and a.is_contiguous()
        return a.data_ptr(), 1 if a.is_cuda else 0

    def set(self, W):
        ptr, dev = self._ptr(W)
        self._check(lib().hrm_set(self.h, _VP(ptr), dev))

    def set_primitive(self, prim):
        ptr, dev = self._ptr(np.ascontiguousarray(prim, dtype=np.float64) if isinstance(prim, np.ndarray) else prim)
        self._check(lib().hrm_set_primitive(self.h, _VP(ptr), dev))

    def set_boundary(self, side, values, primitive=True):
        """State of Dirichlet side `side` (2 d + 0 low, 2 d + 1 high): primitive
        planes (N + D + 1, slice cells) or, with primitive=False, W planes (M, slice cells)."""
        ptr, dev = self._ptr(np.ascontiguousarray(values, dtype=np.float64)
                             if isinstance(values, np.ndarray) else values)
        self._check(lib().hrm_set_boundary(self.h, int(side), _VP(ptr), 1 if primitive else 0, dev))

    def set_params(self, params: HrmParams):
        self._check(lib().hrm_set_params(self.h, ctypes.byref(params)))
        self.params = params

    def get(self, field=FIELD_W, out=None):
        planes = {FIELD_W: self.M, FIELD_V: self.M, FIELD_C5: 1, FIELD_PT: 2, FIELD_C4: 1,
                  FIELD_PSI_GAMMA: self.N + 1, FIELD_ALPHA: self.N, FIELD_Y: self.N, FIELD_SCHLIEREN: 1}[field]
        if out is None:
            out = np.empty((planes, self.ncells))
        ptr, dev = self._ptr(out)
        self._check(lib().hrm_get(self.h, field, _VP(ptr), dev))
        return out

    # -- method
    def dt(self, cfl):
        dt = ctypes.c_double()
        tau = (ctypes.c_double * 3)()
        self._check(lib().hrm_dt(self.h, cfl, ctypes.byref(dt), tau))
        return dt.value, np.array(tau[:self.D])

    def bounds_violations(self) -> int:
        """Out-of-range indices the kernels met (bounds-check builds; -1 otherwise)."""
        return int(lib().hrm_bounds_violations(self.h))

    def set_time(self, t, steps):
        """Restore the simulated time and step count (checkpoint / restart)."""
        self._check(lib().hrm_set_time(self.h, float(t), int(steps)))

    def step(self, dt=0.0, nsteps=1):
        return self._check(lib().hrm_step(self.h, float(dt), int(nsteps)))

    def set_step_path(self, path):
        """1: persistent stage launches where eligible (default); 0: per-phase kernels."""
        self._check(lib().hrm_set_step_path(self.h, int(path)))

    def step_launches(self) -> int:
        return int(lib().hrm_step_launches(self.h))

    # -- one stage at a time (domain decomposition)
    def step_tau(self):
        """tau_d of the step state as a step computes them (D values)."""
        tau = (ctypes.c_double * 3)()
        self._check(lib().hrm_step_tau(self.h, tau))
        return np.array(tau[:self.D])

    def begin_step(self, tau, dt=0.0):
        t3 = (ctypes.c_double * 3)(*[float(v) for v in tau])
        self._check(lib().hrm_begin_step(self.h, t3, float(dt)))

    def stages(self) -> int:
        return int(lib().hrm_stages(self.h))

    def stage(self, k):
        self._check(lib().hrm_stage(self.h, int(k)))

    def layer_cells(self) -> int:
        """Cells of one layer along the slowest direction."""
        return int(np.prod(self.n[:-1])) if self.D > 1 else 1

    def get_layers(self, stage, first, count, out=None):
        """Layers first..first+count-1 (slowest direction) of the state stage
        `stage` reads: (M, count x layer) numpy array or the given tensor."""
        if out is None:
            out = np.empty((self.M, count * self.layer_cells()))
        ptr, dev = self._ptr(out)
        self._check(lib().hrm_layers(self.h, int(stage), 0, int(first), int(count), _VP(ptr), dev))
        return out

    def set_layers(self, stage, first, count, buf):
        ptr, dev = self._ptr(buf)
        self._check(lib().hrm_layers(self.h, int(stage), 1, int(first), int(count), _VP(ptr), dev))

    def try_step(self, dt=0.0, nsteps=1):
        """hrm_step returning the status instead of raising."""
        return lib().hrm_step(self.h, float(dt), int(nsteps))

    def relax(self):
        self._check(lib().hrm_relax(self.h))

    def rhs(self, lam, out):
        ptr, dev = self._ptr(out)
        assert dev == 1
        self._check(lib().hrm_rhs(self.h, _darr(lam, 3), _VP(ptr)))
        return out

    def time(self):
        t = ctypes.c_double()
        n = ctypes.c_int64()
        self._check(lib().hrm_time(self.h, ctypes.byref(t), ctypes.byref(n)))
        return t.value, n.value

    def admissibility(self):
        c = (ctypes.c_int64 * 4)()
        self._check(lib().hrm_admissibility(self.h, c))
        return [int(x) for x in c]

    def set_profiling(self, on=True):
        self._check(lib().hrm_set_profiling(self.h, 1 if on else 0))

    def profile_read(self, maxn=32):
        """[(kind, ms)] of the kernels of the last traced step."""
        ms = (ctypes.c_float * maxn)()
        kd = (ctypes.c_int32 * maxn)()
        n = lib().hrm_profile_read(self.h, maxn, ms, kd)
        return [(int(kd[i]), float(ms[i])) for i in range(n)]

    def kernel_launches(self) -> int:
        return int(lib().hrm_kernel_launches(self.h))

    # -- learned smoothness gate
    def face_count(self, d):
        n = 1
        for e in range(self.D):
            n *= self.n[e] + (e == d)
        return n

    def set_detector(self, det: "Detector"):
        """Snapshot of the detector's inference weights; params.learned = 1 then allowed."""
        self._check(lib().hrm_set_detector(self.h, det.h))

    def set_gate(self, d, gate):
        g = np.ascontiguousarray(gate, dtype=np.uint8).reshape(-1)
        assert g.size == self.face_count(d)
        self._check(lib().hrm_set_gate(self.h, d, g.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8))))

    def get_gate(self, d):
        g = np.empty(self.face_count(d), dtype=np.uint8)
        self._check(lib().hrm_get_gate(self.h, d, g.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8))))
        return g


def _fptr(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_float))


class Detector:
    """One hrm_detector: the learned smoothness gate's weights, Adam state and
    training samples, all on the GPU."""

    def __init__(self, capacity=1 << 20, seed=0, stream=None):
        L = lib()
        self.stream = _stream_handle(stream)
        h = _VP()
        st = L.hrm_detector_create(ctypes.byref(h), int(capacity), int(seed), _VP(self.stream))
        if st != HRM_OK:
            raise HrmError(st, "hrm_detector_create failed")
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            lib().hrm_detector_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, st):
        if st != HRM_OK:
            raise HrmError(st, lib().hrm_detector_last_error(self.h).decode())
        return st

    def set_weights(self, theta):
        t = np.ascontiguousarray(theta, dtype=np.float32)
        assert t.size == DETECTOR_PARAMS
        self._check(lib().hrm_detector_set_weights(self.h, _fptr(t)))

    def get_weights(self):
        t = np.empty(DETECTOR_PARAMS, dtype=np.float32)
        self._check(lib().hrm_detector_get_weights(self.h, _fptr(t)))
        return t

    def size(self) -> int:
        return int(lib().hrm_detector_size(self.h))

    def clear(self):
        self._check(lib().hrm_detector_clear(self.h))

    def add_samples(self, X, y):
        X = np.ascontiguousarray(X, dtype=np.float32)
        y = np.ascontiguousarray(y, dtype=np.float32)
        assert X.shape == (y.size, DETECTOR_INPUTS)
        self._check(lib().hrm_detector_add_samples(self.h, _fptr(X), _fptr(y), y.size))

    def samples(self, first=0, n=None):
        n = self.size() - first if n is None else n
        X = np.empty((n, DETECTOR_INPUTS), dtype=np.float32)
        y = np.empty(n, dtype=np.float32)
        dv = np.empty(n, dtype=np.float32)
        self._check(lib().hrm_detector_samples(self.h, first, n, _fptr(X), _fptr(y), _fptr(dv)))
        return X, y, dv

    def collect(self, solver: Solver, delta=0.01, keep_rough=1.0, keep_smooth=0.1, keep_flat=0.01) -> int:
        added = ctypes.c_int64()
        self._check(lib().hrm_detector_collect(self.h, solver.h, delta, keep_rough, keep_smooth, keep_flat,
                                               ctypes.byref(added)))
        return added.value

    def gradient(self, first=0, n=None):
        n = self.size() - first if n is None else n
        g = np.empty(DETECTOR_PARAMS, dtype=np.float32)
        loss = ctypes.c_double()
        self._check(lib().hrm_detector_gradient(self.h, first, n, _fptr(g), ctypes.byref(loss)))
        return g, loss.value

    def train(self, steps, batch=4096, lr=1e-3):
        losses = np.empty(max(steps, 1), dtype=np.float32)
        self._check(lib().hrm_detector_train(self.h, int(steps), int(batch), float(lr), _fptr(losses)))
        return losses[:steps]

    def logits(self, first=0, n=None, bf16=True):
        n = self.size() - first if n is None else n
        z = np.empty(n, dtype=np.float32)
        self._check(lib().hrm_detector_logits(self.h, first, n, 1 if bf16 else 0, _fptr(z)))
        return z

    def evaluate(self, threshold=0.5, bf16=True):
        """{'tp','fp','tn','fn','loss'}: positive = gated (predicted smooth)."""
        c = (ctypes.c_int64 * 4)()
        loss = ctypes.c_double()
        self._check(lib().hrm_detector_evaluate(self.h, float(threshold), 1 if bf16 else 0, c, ctypes.byref(loss)))
        return {"tp": c[0], "fp": c[1], "tn": c[2], "fn": c[3], "loss": loss.value}


class BatchSolver:
    """One hrm_batch: many 2D problems (paper_2208_04488_gb300.problems.Problem)
    advanced together."""

    def __init__(self, problems, params: Optional[HrmParams] = None, stream=None, set_state=True):
        L = lib()
        self.problems = list(problems)
        arr = (HrmInstance * len(self.problems))()
        for i, pr in enumerate(self.problems):
            it = arr[i]
            it.grid.ndim = pr.D
            for d in range(3):
                it.grid.n[d] = pr.n[d] if d < pr.D else 1
                it.grid.lo[d] = pr.lo[d] if d < pr.D else 0.0
                it.grid.hi[d] = pr.hi[d] if d < pr.D else 1.0
            for j in range(6):
                it.grid.bc[j] = pr.bc[j] if j < len(pr.bc) else 0
            it.nspecies = pr.N
            for k in range(pr.N):
                it.gamma[k], it.p_inf[k], it.c_v[k], it.q[k] = pr.gamma[k], pr.pinf[k], pr.cv[k], pr.q[k]
        self.params = params if params is not None else params_default()
        self.stream = _stream_handle(stream)
        h = _VP()
        st = L.hrm_batch_create(ctypes.byref(h), len(self.problems), arr, ctypes.byref(self.params),
                                _VP(self.stream))
        if st != HRM_OK:
            raise HrmError(st, L.hrm_batch_last_error(None).decode())
        self.h = h
        if set_state:
            for i, pr in enumerate(self.problems):
                self._check(L.hrm_batch_set_primitive(self.h, i, _VP(np.ascontiguousarray(pr.prim).ctypes.data), 0))

    def close(self):
        if getattr(self, "h", None):
            lib().hrm_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, st):
        if st != HRM_OK:
            raise HrmError(st, lib().hrm_batch_last_error(self.h).decode())
        return st

    def step(self, nsteps=1):
        return self._check(lib().hrm_batch_step(self.h, int(nsteps)))

    def set(self, i, W):
        """Instance i's conservative state, (M, cells) FP64 host array."""
        self._check(lib().hrm_batch_set(self.h, int(i), _VP(np.ascontiguousarray(W, dtype=np.float64).ctypes.data), 0))

    def set_primitive(self, i, prim):
        """Instance i's state from primitives, (N + D + 1, cells) FP64 host array."""
        self._check(lib().hrm_batch_set_primitive(self.h, int(i),
                                                  _VP(np.ascontiguousarray(prim, dtype=np.float64).ctypes.data), 0))

    def get(self, i):
        pr = self.problems[i]
        out = np.empty((pr.M, pr.ncells))
        self._check(lib().hrm_batch_get(self.h, i, _VP(out.ctypes.data), 0))
        return out

    def time(self, i):
        t = ctypes.c_double()
        n = ctypes.c_int64()
        self._check(lib().hrm_batch_time(self.h, i, ctypes.byref(t), ctypes.byref(n)))
        return t.value, n.value

    def admissibility(self):
        c = (ctypes.c_int64 * 4)()
        self._check(lib().hrm_batch_admissibility(self.h, c))
        return [int(x) for x in c]

    def set_launch(self, face_threads, face_tile, cell_tile, blocks_per_sm):
        self._check(lib().hrm_batch_set_launch(self.h, face_threads, face_tile, cell_tile, blocks_per_sm))

    def tune(self, steps_per_trial=1):
        best = (ctypes.c_int32 * 4)()
        self._check(lib().hrm_batch_tune(self.h, steps_per_trial, best))
        return dict(zip(["face_threads", "face_tile", "cell_tile", "blocks_per_sm"], list(best)))

    def kernel_launches(self) -> int:
        return int(lib().hrm_batch_kernel_launches(self.h))

    def total_cells(self) -> int:
        return int(lib().hrm_batch_total_cells(self.h))
