"""ctypes binding of the plain FP64 CPU oracle (``hj_oracle.c``).

TEST INFRASTRUCTURE. Only the test-suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` import this module. It shares no code with
the CUDA library and never imports it.

Arrays are numpy float64 arrays of shape ``(n0, n1, ..., n_{D-1})`` in
Fortran order, so that dimension 0 is contiguous (the paper's column-major
layout, Sec. 2.1). A grid is any object with attributes ``n``, ``lo``, ``hi``
(sequences) and ``periodic`` (sequence of dimension indices).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "hj_oracle.c")
HDR = os.path.join(HERE, "hj_oracle.h")
LIB = os.path.join(HERE, "liboracle.so")
# The same source compiled with floating-point contraction: every a*b + c the
# compiler fuses rounds once instead of twice (on Arm; on targets without a
# fused multiply-add instruction it is the same code). The distance between
# the two builds is the oracle's own sensitivity to rounding order, the yard
# stick of the parity tests on ill-conditioned solves.
LIB_FMA = os.path.join(HERE, "liboracle_fma.so")

ENO1, ENO2, ENO3, WENO5 = 1, 2, 3, 5
DYN_DOUBLE_INTEGRATOR, DYN_AIR3D, DYN_DUBINS4D, DYN_NORM, DYN_ADVECT, DYN_ROTATE, DYN_ROCKETS = 1, 2, 3, 4, 5, 6, 7
BRT_NONE, BRT_MIN0, BRT_MINV = 0, 1, 2
EXTRAP_AWAY_FROM_ZERO, EXTRAP_LINEAR = 0, 1

_lock = threading.Lock()
_lib = None


def build(force: bool = False, fma: bool = False) -> str:
    """Compile the oracle with gcc (plain C99, no FMA contraction, no
    fast-math); fma=True compiles the contracted variant (LIB_FMA)."""
    path = LIB_FMA if fma else LIB
    stale = (not os.path.exists(path)
             or os.path.getmtime(path) < max(os.path.getmtime(SRC), os.path.getmtime(HDR)))
    if force or stale:
        tmp = path + ".%d.tmp" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-std=c99", "-fPIC", "-shared",
                               "-ffp-contract=fast" if fma else "-ffp-contract=off",
                               "-fno-fast-math", "-o", tmp, SRC, "-lm"])
        os.replace(tmp, path)
    return path


class _Grid(ctypes.Structure):
    _fields_ = [("ndim", ctypes.c_int), ("n", ctypes.c_int64 * 4), ("lo", ctypes.c_double * 4),
                ("hi", ctypes.c_double * 4), ("periodic_mask", ctypes.c_uint32)]


class _Method(ctypes.Structure):
    _fields_ = [("scheme", ctypes.c_int), ("dynamics", ctypes.c_int), ("params", ctypes.c_double * 8),
                ("brt", ctypes.c_int), ("extrap", ctypes.c_int), ("weno_ideal", ctypes.c_int),
                ("cfl", ctypes.c_double), ("max_step", ctypes.c_double), ("order", ctypes.c_int),
                ("alpha_global", ctypes.c_int), ("alpha_box", ctypes.c_int)]


_DP = ctypes.POINTER(ctypes.c_double)


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = ctypes.CDLL(LIB)
            P = ctypes.POINTER
            L.orc_spacing.restype = ctypes.c_double
            L.orc_spacing.argtypes = [P(_Grid), ctypes.c_int]
            L.orc_pad_line.argtypes = [_DP, ctypes.c_int64, ctypes.c_int, ctypes.c_int, _DP]
            L.orc_upwind_line.argtypes = [ctypes.c_int, ctypes.c_int, _DP, ctypes.c_int64, ctypes.c_double, _DP, _DP]
            L.orc_upwind.argtypes = [P(_Grid), P(_Method), _DP, ctypes.c_int, _DP, _DP]
            L.orc_weno5.restype = ctypes.c_double
            L.orc_weno5.argtypes = [_DP, ctypes.c_int]
            L.orc_hamiltonian.argtypes = [P(_Method), ctypes.c_int, _DP, _DP, _DP]
            L.orc_alpha.argtypes = [P(_Method), ctypes.c_int, _DP, _DP]
            L.orc_alpha_box.argtypes = [P(_Method), ctypes.c_int, _DP, _DP, _DP, _DP]
            L.orc_term.argtypes = [P(_Grid), P(_Method), _DP, _DP]
            L.orc_step_bound_inv.argtypes = [P(_Grid), P(_Method), _DP]
            L.orc_rk3_step.argtypes = [P(_Grid), P(_Method), ctypes.c_double, _DP]
            L.orc_rk_step.argtypes = [P(_Grid), P(_Method), ctypes.c_double, _DP]
            L.orc_alpha_max.argtypes = [P(_Grid), P(_Method), _DP]
            L.orc_solve.argtypes = [P(_Grid), P(_Method), _DP, ctypes.c_int, _DP, _DP,
                                    P(ctypes.c_int64), _DP]
            L.orc_time_eps.restype = ctypes.c_double
            _lib = L
    return _lib


def _grid(g) -> _Grid:
    G = _Grid()
    G.ndim = len(g.n)
    mask = 0
    for d in range(G.ndim):
        G.n[d] = int(g.n[d])
        G.lo[d] = float(g.lo[d])
        G.hi[d] = float(g.hi[d])
    for d in g.periodic:
        mask |= 1 << int(d)
    G.periodic_mask = mask
    return G


def method(scheme=WENO5, dynamics=DYN_DOUBLE_INTEGRATOR, params=(), brt=BRT_MIN0,
           extrap=EXTRAP_AWAY_FROM_ZERO, weno_ideal=False, cfl=0.8, max_step=float("inf"), order=3,
           alpha_global=False, alpha_box=False) -> _Method:
    M = _Method()
    M.scheme = scheme
    M.dynamics = dynamics
    for i, p in enumerate(params):
        M.params[i] = float(p)
    M.brt = brt
    M.extrap = extrap
    M.weno_ideal = 1 if weno_ideal else 0
    M.cfl = float(cfl)
    M.max_step = float(max_step)
    M.order = int(order)
    M.alpha_global = 1 if alpha_global else 0
    M.alpha_box = 1 if alpha_box else 0
    return M


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(_DP)


def _f64(V, shape=None) -> np.ndarray:
    A = np.asfortranarray(np.asarray(V, dtype=np.float64))
    if shape is not None and A.shape != tuple(shape):
        raise ValueError("array shape %s does not match grid %s" % (A.shape, tuple(shape)))
    return A


def _check(rc: int, what: str):
    if rc != 0:
        raise ValueError("oracle %s failed with code %d" % (what, rc))


def spacing(g, d: int) -> float:
    return lib().orc_spacing(ctypes.byref(_grid(g)), d)


def time_eps() -> float:
    return lib().orc_time_eps()


def pad_line(line, periodic: bool, extrap=EXTRAP_AWAY_FROM_ZERO) -> np.ndarray:
    line = np.ascontiguousarray(line, dtype=np.float64)
    out = np.empty(line.size + 6)
    _check(lib().orc_pad_line(_ptr(line), line.size, int(periodic), extrap, _ptr(out)), "pad_line")
    return out


def upwind_line(padded, dx: float, scheme=WENO5, weno_ideal=False):
    padded = np.ascontiguousarray(padded, dtype=np.float64)
    n = padded.size - 6
    pm, pp = np.empty(n), np.empty(n)
    _check(lib().orc_upwind_line(scheme, int(weno_ideal), _ptr(padded), n, float(dx), _ptr(pm), _ptr(pp)),
           "upwind_line")
    return pm, pp


def weno5(v, ideal=False) -> float:
    v = np.ascontiguousarray(v, dtype=np.float64)
    return lib().orc_weno5(_ptr(v), int(ideal))


def hamiltonian(m: _Method, x, p) -> float:
    x = np.ascontiguousarray(x, dtype=np.float64)
    p = np.ascontiguousarray(p, dtype=np.float64)
    out = np.zeros(1)
    _check(lib().orc_hamiltonian(ctypes.byref(m), x.size, _ptr(x), _ptr(p), _ptr(out)), "hamiltonian")
    return float(out[0])


def alpha(m: _Method, x) -> np.ndarray:
    x = np.ascontiguousarray(x, dtype=np.float64)
    out = np.zeros(x.size)
    _check(lib().orc_alpha(ctypes.byref(m), x.size, _ptr(x), _ptr(out)), "alpha")
    return out


def alpha_box(m: _Method, x, lo, hi) -> np.ndarray:
    """max of |dHg/dp_d| over the box lo <= p <= hi at coordinates x (R12)."""
    x = np.ascontiguousarray(x, dtype=np.float64)
    lo = np.ascontiguousarray(lo, dtype=np.float64)
    hi = np.ascontiguousarray(hi, dtype=np.float64)
    out = np.zeros(x.size)
    _check(lib().orc_alpha_box(ctypes.byref(m), x.size, _ptr(x), _ptr(lo), _ptr(hi), _ptr(out)), "alpha_box")
    return out


def upwind(g, m: _Method, V, dim: int):
    V = _f64(V, g.n)
    pm = np.empty(V.shape, order="F")
    pp = np.empty(V.shape, order="F")
    _check(lib().orc_upwind(ctypes.byref(_grid(g)), ctypes.byref(m), _ptr(V), dim, _ptr(pm), _ptr(pp)),
           "upwind")
    return pm, pp


def term(g, m: _Method, V) -> np.ndarray:
    V = _f64(V, g.n)
    out = np.empty(V.shape, order="F")
    _check(lib().orc_term(ctypes.byref(_grid(g)), ctypes.byref(m), _ptr(V), _ptr(out)), "term")
    return out


def step_bound_inv(g, m: _Method) -> float:
    out = np.zeros(1)
    _check(lib().orc_step_bound_inv(ctypes.byref(_grid(g)), ctypes.byref(m), _ptr(out)), "step_bound_inv")
    return float(out[0])


def rk3_step(g, m: _Method, V, dt: float) -> np.ndarray:
    W = np.array(_f64(V, g.n), order="F", copy=True)
    _check(lib().orc_rk3_step(ctypes.byref(_grid(g)), ctypes.byref(m), float(dt), _ptr(W)), "rk3_step")
    return W


def rk_step(g, m: _Method, V, dt: float) -> np.ndarray:
    """One TVD-RK step of the method's order (1, 2 or 3)."""
    W = np.array(_f64(V, g.n), order="F", copy=True)
    _check(lib().orc_rk_step(ctypes.byref(_grid(g)), ctypes.byref(m), float(dt), _ptr(W)), "rk_step")
    return W


def alpha_max(g, m: _Method) -> np.ndarray:
    out = np.zeros(4)
    _check(lib().orc_alpha_max(ctypes.byref(_grid(g)), ctypes.byref(m), _ptr(out)), "alpha_max")
    return out[:len(g.n)]


_lib_fma = None


def _solve_lib(fma: bool):
    global _lib_fma
    if not fma:
        return lib()
    with _lock:
        if _lib_fma is None:
            L = ctypes.CDLL(build(fma=True))
            L.orc_solve.argtypes = [ctypes.POINTER(_Grid), ctypes.POINTER(_Method), _DP, ctypes.c_int, _DP, _DP,
                                    ctypes.POINTER(ctypes.c_int64), _DP]
            _lib_fma = L
    return _lib_fma


def solve(g, m: _Method, V0, slice_times, fma: bool = False):
    """Returns (slices[n_slices, *n] , steps, times_reached); fma=True runs the
    contracted build (LIB_FMA)."""
    V0 = _f64(V0, g.n)
    ts = np.ascontiguousarray(slice_times, dtype=np.float64)
    total = int(np.prod(g.n))
    out = np.empty(ts.size * total)
    steps = ctypes.c_int64(0)
    times = np.empty(ts.size)
    _check(_solve_lib(fma).orc_solve(ctypes.byref(_grid(g)), ctypes.byref(m), _ptr(V0), ts.size, _ptr(ts),
                                     _ptr(out), ctypes.byref(steps), _ptr(times)), "solve")
    slices = [out[k * total:(k + 1) * total].reshape(tuple(g.n), order="F") for k in range(ts.size)]
    return np.stack(slices), int(steps.value), times
