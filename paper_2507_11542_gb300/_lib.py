"""Thin ctypes binding of libhj.so (include/hj.h), with the same names.

Argument marshalling only: every step of the level-set update runs in the
CUDA kernels of libhj.so. There is no fallback; loading fails loudly when the
library has not been built (``python -m paper_2507_11542_gb300.build``).

Grid arrays cross the boundary as flat, contiguous torch tensors (or host
numpy arrays for host-side inputs/outputs) of prod(n) elements with
dimension 0 fastest. ``to_flat`` / ``from_flat`` convert from/to numpy arrays
of shape (n0, ..., n_{D-1}) in Fortran order.
"""
from __future__ import annotations

import ctypes
import math
import os
import threading

import numpy as np

PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(PKG, "libhj.so")

HJ_OK, HJ_EINVAL, HJ_ENOMEM, HJ_ECUDA, HJ_ENONFINITE, HJ_ETIMEOUT, HJ_ECANCELLED, HJ_EBUSY = range(8)
HJ_ENO1, HJ_ENO2, HJ_ENO3, HJ_WENO5 = 1, 2, 3, 5
(HJ_DYN_DOUBLE_INTEGRATOR, HJ_DYN_AIR3D, HJ_DYN_DUBINS4D, HJ_DYN_NORM, HJ_DYN_ADVECT,
 HJ_DYN_ROTATE, HJ_DYN_ROCKETS) = 1, 2, 3, 4, 5, 6, 7
HJ_BRT_NONE, HJ_BRT_MIN0, HJ_BRT_MINV = 0, 1, 2
HJ_F32, HJ_F64 = 1, 2
HJ_EXTRAP_AWAY_FROM_ZERO, HJ_EXTRAP_LINEAR = 0, 1
HJ_ALPHA_NODE, HJ_ALPHA_GLOBAL, HJ_ALPHA_BOX = 0, 1, 2
HJ_KERNEL_AUTO, HJ_KERNEL_ROWS, HJ_KERNEL_NODE = 0, 1, 2

# every function include/hj.h declares (checked by the test-suite against the .so)
EXPORTS = ["hj_ctx_create", "hj_ctx_destroy", "hj_status_str", "hj_ctx_last_error", "hj_version",
           "hj_upwind", "hj_term", "hj_step_bound", "hj_rk3_step", "hj_rk3_stage", "hj_solve",
           "hj_rk3_step_static", "hj_solve_batch", "hj_server_create", "hj_server_submit", "hj_server_wait",
           "hj_server_cancel", "hj_server_counters", "hj_server_destroy", "hj_implicit_surface"]
HJ_SHAPE_SPHERE, HJ_SHAPE_ELLIPSOID, HJ_SHAPE_RECTANGLE = 1, 2, 3
HJ_SHAPE_UNION, HJ_SHAPE_INTERSECT, HJ_SHAPE_SUBTRACT = 1, 2, 3
HJ_MAX_SHAPES = 32
HJ_STATIC_MAX_NODES = 1 << 20
HJ_STATIC_MAX_ANGLES = 4096


class hj_grid(ctypes.Structure):
    _fields_ = [("ndim", ctypes.c_int32), ("n", ctypes.c_int64 * 4), ("lo", ctypes.c_double * 4),
                ("hi", ctypes.c_double * 4), ("periodic_mask", ctypes.c_uint32)]


class hj_method(ctypes.Structure):
    _fields_ = [("scheme", ctypes.c_int32), ("dynamics", ctypes.c_int32), ("params", ctypes.c_double * 8),
                ("brt", ctypes.c_int32), ("extrap", ctypes.c_int32), ("cfl", ctypes.c_double),
                ("max_step", ctypes.c_double), ("order", ctypes.c_int32), ("alpha_mode", ctypes.c_int32),
                ("kernel", ctypes.c_int32), ("tile_override", ctypes.c_int32 * 4)]


class hj_problem(ctypes.Structure):
    _fields_ = [("grid", hj_grid), ("method", hj_method), ("dtype", ctypes.c_int32), ("v0", ctypes.c_void_p),
                ("v0_on_device", ctypes.c_int32), ("n_slices", ctypes.c_int32),
                ("slice_times", ctypes.POINTER(ctypes.c_double)), ("t0", ctypes.c_double)]


class hj_stats(ctypes.Structure):
    _fields_ = [("steps", ctypes.c_int64), ("cell_updates", ctypes.c_int64), ("kernel_launches", ctypes.c_int64),
                ("step_bound_inv", ctypes.c_double), ("t_final", ctypes.c_double), ("elapsed_ms", ctypes.c_double),
                ("queued_ms", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class hj_server_info(ctypes.Structure):
    _fields_ = [("queued", ctypes.c_int64), ("running", ctypes.c_int64), ("completed", ctypes.c_int64),
                ("bytes_in_use", ctypes.c_int64), ("budget", ctypes.c_int64), ("kernel_launches", ctypes.c_int64)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class hj_shape(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("op", ctypes.c_int32), ("dims_mask", ctypes.c_uint32),
                ("center", ctypes.c_double * 4), ("axes", ctypes.c_double * 4), ("radius", ctypes.c_double)]


class HJError(RuntimeError):
    def __init__(self, status, message):
        super().__init__("%s (%d): %s" % (_STATUS.get(status, "?"), status, message))
        self.status = status


_STATUS = {HJ_OK: "HJ_OK", HJ_EINVAL: "HJ_EINVAL", HJ_ENOMEM: "HJ_ENOMEM", HJ_ECUDA: "HJ_ECUDA",
           HJ_ENONFINITE: "HJ_ENONFINITE", HJ_ETIMEOUT: "HJ_ETIMEOUT", HJ_ECANCELLED: "HJ_ECANCELLED",
           HJ_EBUSY: "HJ_EBUSY"}

_lock = threading.Lock()
_lib = None
_P = ctypes.POINTER
_vp = ctypes.c_void_p


def load():
    """Load libhj.so; raises if it is missing (no CPU or eager fallback exists)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError("libhj.so is not built at %s; run paper_2507_11542_gb300.build.build()" % LIB_PATH)
            L = ctypes.CDLL(LIB_PATH)
            L.hj_ctx_create.argtypes = [ctypes.c_int32, _vp, _P(_vp)]
            L.hj_ctx_destroy.argtypes = [_vp]
            L.hj_ctx_destroy.restype = None
            L.hj_status_str.argtypes = [ctypes.c_int]
            L.hj_status_str.restype = ctypes.c_char_p
            L.hj_ctx_last_error.argtypes = [_vp]
            L.hj_ctx_last_error.restype = ctypes.c_char_p
            L.hj_version.restype = ctypes.c_char_p
            L.hj_upwind.argtypes = [_vp, _P(hj_grid), _P(hj_method), ctypes.c_int32, _vp, ctypes.c_int32, _vp, _vp]
            L.hj_term.argtypes = [_vp, _P(hj_grid), _P(hj_method), ctypes.c_int32, _vp, _vp]
            L.hj_step_bound.argtypes = [_vp, _P(hj_grid), _P(hj_method), _P(ctypes.c_double)]
            L.hj_rk3_step.argtypes = [_vp, _P(hj_grid), _P(hj_method), ctypes.c_int32, _vp, ctypes.c_double]
            L.hj_rk3_stage.argtypes = [_vp, _P(hj_grid), _P(hj_method), ctypes.c_int32, ctypes.c_int32, _vp, _vp, _vp,
                                       ctypes.c_double]
            L.hj_solve.argtypes = [_vp, _P(hj_problem), _vp, ctypes.c_int32, _P(ctypes.c_double), _P(hj_stats)]
            L.hj_solve_batch.argtypes = [_vp, ctypes.c_int32, _P(hj_problem), _P(_vp), _P(ctypes.c_int32),
                                         _P(_P(ctypes.c_double)), _P(hj_stats)]
            L.hj_server_create.argtypes = [_vp, ctypes.c_size_t, ctypes.c_int32, _P(_vp)]
            L.hj_server_submit.argtypes = [_vp, _P(hj_problem), _vp, ctypes.c_int32, _P(ctypes.c_double),
                                           _P(ctypes.c_uint64)]
            L.hj_server_wait.argtypes = [_vp, ctypes.c_uint64, ctypes.c_int32, _P(hj_stats)]
            L.hj_server_cancel.argtypes = [_vp, ctypes.c_uint64]
            L.hj_server_counters.argtypes = [_vp, _P(hj_server_info)]
            L.hj_server_destroy.argtypes = [_vp]
            L.hj_server_destroy.restype = None
            L.hj_rk3_step_static.argtypes = [_vp, ctypes.c_int32, _P(hj_grid), _P(hj_method), ctypes.c_int32, _vp,
                                             ctypes.c_double]
            L.hj_implicit_surface.argtypes = [_vp, _P(hj_grid), ctypes.c_int32, _P(hj_shape), ctypes.c_int32, _vp,
                                              ctypes.c_int32]
            _lib = L
    return _lib


def _check(ctx, status):
    if status != HJ_OK:
        msg = load().hj_ctx_last_error(ctx).decode() if ctx else ""
        raise HJError(status, msg)


# ---------------------------------------------------------------------------
# struct builders
# ---------------------------------------------------------------------------

def make_grid(spec) -> hj_grid:
    """spec: any object with n, lo, hi (sequences) and periodic (dimension indices)."""
    g = hj_grid()
    g.ndim = len(spec.n)
    for d in range(g.ndim):
        g.n[d] = int(spec.n[d])
        g.lo[d] = float(spec.lo[d])
        g.hi[d] = float(spec.hi[d])
    mask = 0
    for d in spec.periodic:
        mask |= 1 << int(d)
    g.periodic_mask = mask
    return g


def make_method(scheme=HJ_WENO5, dynamics=HJ_DYN_DOUBLE_INTEGRATOR, params=(), brt=HJ_BRT_MIN0,
                extrap=HJ_EXTRAP_AWAY_FROM_ZERO, cfl=0.8, max_step=math.inf, order=3,
                alpha_mode=HJ_ALPHA_NODE, kernel=HJ_KERNEL_AUTO, tile_override=(0, 0, 0, 0)) -> hj_method:
    m = hj_method()
    m.scheme = scheme
    m.dynamics = dynamics
    for i, p in enumerate(params):
        m.params[i] = float(p)
    m.brt = brt
    m.extrap = extrap
    m.cfl = float(cfl)
    m.max_step = float(max_step)
    m.order = int(order)
    m.alpha_mode = int(alpha_mode)
    m.kernel = int(kernel)
    for i, t in enumerate(tile_override):
        m.tile_override[i] = int(t)
    return m


def dtype_code(torch_dtype) -> int:
    import torch
    if torch_dtype == torch.float64:
        return HJ_F64
    if torch_dtype == torch.float32:
        return HJ_F32
    raise ValueError("grid arrays must be float32 or float64")


def to_flat(V: np.ndarray) -> np.ndarray:
    """(n0, ..., n_{D-1}) array -> flat array with dimension 0 fastest."""
    return np.asarray(V).ravel(order="F")


def from_flat(flat, n) -> np.ndarray:
    return np.asarray(flat).reshape(tuple(n), order="F")


# ---------------------------------------------------------------------------
# entry points (same names as the C ABI)
# ---------------------------------------------------------------------------

def hj_version() -> str:
    return load().hj_version().decode()


def hj_status_str(status: int) -> str:
    return load().hj_status_str(status).decode()


def hj_ctx_create(device: int = 0, stream: int | None = None) -> int:
    """stream: a raw cudaStream_t (e.g. torch.cuda.current_stream().cuda_stream)."""
    out = _vp()
    st = load().hj_ctx_create(int(device), _vp(stream or 0), ctypes.byref(out))
    if st != HJ_OK:
        raise HJError(st, "hj_ctx_create(device=%d)" % device)
    return out.value


def hj_ctx_destroy(ctx: int) -> None:
    load().hj_ctx_destroy(_vp(ctx))


def hj_ctx_last_error(ctx: int) -> str:
    return load().hj_ctx_last_error(_vp(ctx)).decode()


def _ptr(t) -> int:
    return 0 if t is None else int(t.data_ptr())


def hj_upwind(ctx, grid: hj_grid, method: hj_method, dtype: int, v, dim: int, pm, pp) -> None:
    _check(ctx, load().hj_upwind(_vp(ctx), ctypes.byref(grid), ctypes.byref(method), dtype, _vp(_ptr(v)), dim,
                                 _vp(_ptr(pm)), _vp(_ptr(pp))))


def hj_term(ctx, grid: hj_grid, method: hj_method, dtype: int, v, ydot) -> None:
    _check(ctx, load().hj_term(_vp(ctx), ctypes.byref(grid), ctypes.byref(method), dtype, _vp(_ptr(v)),
                               _vp(_ptr(ydot))))


def hj_step_bound(ctx, grid: hj_grid, method: hj_method) -> float:
    out = ctypes.c_double(0.0)
    _check(ctx, load().hj_step_bound(_vp(ctx), ctypes.byref(grid), ctypes.byref(method), ctypes.byref(out)))
    return out.value


def hj_rk3_step(ctx, grid: hj_grid, method: hj_method, dtype: int, v, dt: float) -> None:
    _check(ctx, load().hj_rk3_step(_vp(ctx), ctypes.byref(grid), ctypes.byref(method), dtype, _vp(_ptr(v)),
                                   float(dt)))


def hj_rk3_stage(ctx, grid: hj_grid, method: hj_method, dtype: int, stage: int, u, vn, out, dt: float) -> None:
    _check(ctx, load().hj_rk3_stage(_vp(ctx), ctypes.byref(grid), ctypes.byref(method), dtype, int(stage),
                                    _vp(_ptr(u)), _vp(_ptr(vn)), _vp(_ptr(out)), float(dt)))


def hj_rk3_step_static(stream: int, device: int, grid: hj_grid, method: hj_method, dtype: int, v, dt: float) -> int:
    """No-allocation RK3 step; returns the raw hj_status (there is no context for a message)."""
    return load().hj_rk3_step_static(_vp(stream or 0), int(device), ctypes.byref(grid), ctypes.byref(method), dtype,
                                     _vp(_ptr(v)), float(dt))


def hj_solve(ctx, problem: hj_problem, out_slices_ptr: int, out_on_device: bool, out_times: np.ndarray | None):
    stats = hj_stats()
    tp = None if out_times is None else out_times.ctypes.data_as(_P(ctypes.c_double))
    _check(ctx, load().hj_solve(_vp(ctx), ctypes.byref(problem), _vp(out_slices_ptr), int(bool(out_on_device)), tp,
                                ctypes.byref(stats)))
    return stats


def hj_solve_batch(ctx, problems, out_ptrs, out_on_device, out_times):
    """problems: list of hj_problem; out_ptrs: list of int addresses; out_on_device: list of bools;
    out_times: list of float64 numpy arrays (or None). Returns a list of hj_stats."""
    n = len(problems)
    P = (hj_problem * n)(*problems)
    O = (_vp * n)(*[_vp(p) for p in out_ptrs])
    F = (ctypes.c_int32 * n)(*[int(bool(f)) for f in out_on_device])
    T = (_P(ctypes.c_double) * n)(*[(t.ctypes.data_as(_P(ctypes.c_double)) if t is not None else None)
                                   for t in out_times])
    S = (hj_stats * n)()
    _check(ctx, load().hj_solve_batch(_vp(ctx), n, P, O, F, T, S))
    return [S[i] for i in range(n)]


def hj_server_create(ctx, hbm_budget: int, max_slots: int) -> int:
    out = _vp()
    _check(ctx, load().hj_server_create(_vp(ctx), int(hbm_budget), int(max_slots), ctypes.byref(out)))
    return out.value


def hj_server_submit(srv, problem: hj_problem, out_ptr: int, out_on_device: bool, out_times) -> int:
    """Returns the ticket; raises HJError with the status on refusal."""
    t = ctypes.c_uint64(0)
    tp = None if out_times is None else out_times.ctypes.data_as(_P(ctypes.c_double))
    st = load().hj_server_submit(_vp(srv), ctypes.byref(problem), _vp(out_ptr), int(bool(out_on_device)), tp,
                                 ctypes.byref(t))
    if st != HJ_OK:
        raise HJError(st, "hj_server_submit")
    return t.value


def hj_server_wait(srv, ticket: int, timeout_ms: int = -1):
    """Returns (status, stats)."""
    s = hj_stats()
    st = load().hj_server_wait(_vp(srv), ctypes.c_uint64(ticket), int(timeout_ms), ctypes.byref(s))
    return st, s


def hj_server_cancel(srv, ticket: int) -> int:
    return load().hj_server_cancel(_vp(srv), ctypes.c_uint64(ticket))


def hj_server_counters(srv) -> dict:
    info = hj_server_info()
    st = load().hj_server_counters(_vp(srv), ctypes.byref(info))
    d = info.as_dict()
    d["status"] = st
    return d


def hj_server_destroy(srv) -> None:
    load().hj_server_destroy(_vp(srv))


def make_problem(spec, method: hj_method, dtype: int, v0_ptr: int, v0_on_device: bool, slice_times: np.ndarray,
                 t0: float = 0.0):
    """Returns (problem, keepalive) -- keep the second value alive while the problem is in use."""
    ts = np.ascontiguousarray(slice_times, dtype=np.float64)
    p = hj_problem()
    p.grid = make_grid(spec)
    p.method = method
    p.dtype = dtype
    p.v0 = v0_ptr
    p.v0_on_device = int(bool(v0_on_device))
    p.n_slices = ts.size
    p.slice_times = ts.ctypes.data_as(_P(ctypes.c_double))
    p.t0 = float(t0)
    return p, ts


def make_shapes(shapes):
    """shapes: sequence of dicts {kind, op, dims, center, axes, radius}; dims is
    a sequence of dimension indices (default: all four bits up to the center's
    length), center/axes sequences of up to 4 numbers."""
    arr = (hj_shape * len(shapes))()
    for k, sh in enumerate(shapes):
        a = arr[k]
        a.kind = int(sh["kind"])
        a.op = int(sh.get("op", HJ_SHAPE_UNION))
        dims = sh.get("dims", range(len(sh.get("center", ()))))
        a.dims_mask = sum(1 << int(d) for d in dims)
        for d, v in enumerate(sh.get("center", ())):
            a.center[d] = float(v)
        for d, v in enumerate(sh.get("axes", ())):
            a.axes[d] = float(v)
        a.radius = float(sh.get("radius", 0.0))
    return arr


def hj_implicit_surface(ctx, grid: hj_grid, shapes, dtype: int, out, out_on_device: bool = True) -> None:
    """out: a CUDA tensor (out_on_device) or a host numpy array / tensor of prod(n) elements."""
    arr = make_shapes(shapes)
    if out_on_device:
        ptr = _ptr(out)
    else:
        ptr = out.ctypes.data if isinstance(out, np.ndarray) else int(out.data_ptr())
    _check(ctx, load().hj_implicit_surface(_vp(ctx), ctypes.byref(grid), len(shapes), arr, dtype, _vp(ptr),
                                           1 if out_on_device else 0))
