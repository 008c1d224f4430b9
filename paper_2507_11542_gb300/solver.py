"""Torch-tensor convenience layer over the C ABI (argument marshalling only).

Grid arrays are flat contiguous tensors of prod(n) elements, dimension 0
fastest. Every call runs in libhj.so on the context's stream.
"""
from __future__ import annotations

import math

import numpy as np

from . import _lib as L


class Context:
    """An hj_ctx bound to one device and a torch stream (default: the current one)."""

    def __init__(self, device: int = 0, stream=None):
        import torch
        self.device = int(device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        self.handle = L.hj_ctx_create(self.device, self.stream.cuda_stream)

    def close(self):
        if getattr(self, "handle", None):
            L.hj_ctx_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def method(scheme=L.HJ_WENO5, dynamics=L.HJ_DYN_DOUBLE_INTEGRATOR, params=(), brt=L.HJ_BRT_MIN0,
           extrap=L.HJ_EXTRAP_AWAY_FROM_ZERO, cfl=0.8, max_step=math.inf, order=3,
           alpha_mode=L.HJ_ALPHA_NODE, kernel=L.HJ_KERNEL_AUTO, tile_override=(0, 0, 0, 0)) -> L.hj_method:
    """An hj_method; kernel and tile_override choose the stage kernel and pin
    the row kernel's launch shape {ty, tz, occ, flags} (all 0: tuned; see include/hj.h)."""
    return L.make_method(scheme, dynamics, params, brt, extrap, cfl, max_step, order, alpha_mode, kernel,
                         tile_override)


def _check_tensor(t, spec, name):
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda or not t.is_contiguous():
        raise ValueError("%s must be a contiguous CUDA tensor" % name)
    if t.numel() != int(np.prod(spec.n)):
        raise ValueError("%s has %d elements, the grid %d" % (name, t.numel(), int(np.prod(spec.n))))


def upwind(ctx: Context, spec, m: L.hj_method, V, dim: int):
    import torch
    _check_tensor(V, spec, "V")
    pm, pp = torch.empty_like(V), torch.empty_like(V)
    L.hj_upwind(ctx.handle, L.make_grid(spec), m, L.dtype_code(V.dtype), V, dim, pm, pp)
    return pm, pp


def term(ctx: Context, spec, m: L.hj_method, V):
    import torch
    _check_tensor(V, spec, "V")
    y = torch.empty_like(V)
    L.hj_term(ctx.handle, L.make_grid(spec), m, L.dtype_code(V.dtype), V, y)
    return y


def step_bound(ctx: Context, spec, m: L.hj_method) -> float:
    return L.hj_step_bound(ctx.handle, L.make_grid(spec), m)


def rk3_step(ctx: Context, spec, m: L.hj_method, V, dt: float):
    """One TVD-RK3 step in place on V."""
    _check_tensor(V, spec, "V")
    L.hj_rk3_step(ctx.handle, L.make_grid(spec), m, L.dtype_code(V.dtype), V, dt)
    return V


def rk3_stage(ctx: Context, spec, m: L.hj_method, stage: int, u, vn, out, dt: float):
    """One fused RK3 stage: out = cv*vn + cu*(u + dt*L(u)) (stage 1: out = u + dt*L(u))."""
    _check_tensor(u, spec, "u")
    _check_tensor(out, spec, "out")
    L.hj_rk3_stage(ctx.handle, L.make_grid(spec), m, L.dtype_code(u.dtype), stage, u, vn, out, dt)
    return out


def solve(ctx: Context, spec, m: L.hj_method, V0, slice_times, out=None, t0: float = 0.0):
    """Integrate V0 through the slice times.

    V0: flat CUDA tensor, or a host tensor (pinned memory recommended).
    out: optional tensor [n_slices, prod(n)] of V0's dtype (device or host).
    t0: the time of V0; to resume from a slice of an earlier solve, pass that
    slice and its reported time (the continuation equals the uninterrupted solve).
    Returns (out, times_reached, stats_dict).
    """
    import torch
    ts = np.ascontiguousarray(slice_times, dtype=np.float64)
    N = int(np.prod(spec.n))
    if V0.numel() != N or not V0.is_contiguous():
        raise ValueError("V0 must be contiguous with prod(n) elements")
    if out is None:
        out = torch.empty((ts.size, N), dtype=V0.dtype, device=V0.device)
    if out.dtype != V0.dtype or out.numel() != ts.size * N or not out.is_contiguous():
        raise ValueError("out must be a contiguous [n_slices, prod(n)] tensor of V0's dtype")
    prob, keep = L.make_problem(spec, m, L.dtype_code(V0.dtype), int(V0.data_ptr()), V0.is_cuda, ts, t0)
    times = np.zeros(ts.size)
    stats = L.hj_solve(ctx.handle, prob, int(out.data_ptr()), out.is_cuda, times)
    del keep
    return out, times, stats.as_dict()


def solve_batch(ctx: Context, specs, methods, V0s, slice_times, outs=None, t0s=None):
    """Many independent solves in one call (hj_solve_batch).

    specs, methods, V0s (flat tensors, device or host), slice_times: one entry
    per problem. outs: optional list of [n_slices, prod(n)] tensors. t0s:
    optional list of the times of the V0s (see solve).
    Returns (outs, times_list, stats_list)."""
    import torch
    n = len(specs)
    if not (len(methods) == len(V0s) == len(slice_times) == n):
        raise ValueError("one method, V0 and slice-time list per grid")
    probs, keep, times = [], [], []
    if outs is None:
        outs = [torch.empty((len(ts), V0.numel()), dtype=V0.dtype, device=V0.device)
                for V0, ts in zip(V0s, slice_times)]
    t0s = [0.0] * n if t0s is None else list(t0s)
    for spec, m, V0, ts, out, t0 in zip(specs, methods, V0s, slice_times, outs, t0s):
        N = int(np.prod(spec.n))
        if V0.numel() != N or not V0.is_contiguous() or out.numel() != len(ts) * N or out.dtype != V0.dtype:
            raise ValueError("V0/out do not match the grid")
        p, k = L.make_problem(spec, m, L.dtype_code(V0.dtype), int(V0.data_ptr()), V0.is_cuda, ts, t0)
        probs.append(p)
        keep.append(k)
        times.append(np.zeros(len(ts)))
    stats = L.hj_solve_batch(ctx.handle, probs, [int(o.data_ptr()) for o in outs], [o.is_cuda for o in outs], times)
    del keep
    return outs, times, [s.as_dict() for s in stats]


class Server:
    """A continuous-batching server (hj_server_*). Keeps every submitted
    request's buffers alive until its result has been collected."""

    def __init__(self, ctx: Context, hbm_budget: int, max_slots: int = 64):
        self.ctx = ctx
        self.handle = L.hj_server_create(ctx.handle, hbm_budget, max_slots)
        self._live = {}

    def submit(self, spec, m: L.hj_method, V0, slice_times, out=None, t0: float = 0.0):
        import torch
        ts = np.ascontiguousarray(slice_times, dtype=np.float64)
        if out is None:
            out = torch.empty((ts.size, V0.numel()), dtype=V0.dtype, device=V0.device)
        prob, keep = L.make_problem(spec, m, L.dtype_code(V0.dtype), int(V0.data_ptr()), V0.is_cuda, ts, t0)
        times = np.zeros(ts.size)
        ticket = L.hj_server_submit(self.handle, prob, int(out.data_ptr()), out.is_cuda, times)
        self._live[ticket] = (V0, out, times, keep)
        return ticket

    def wait(self, ticket: int, timeout_ms: int = -1):
        """Returns (status, out, times, stats) or raises on an unknown ticket; status
        HJ_ETIMEOUT leaves the request running."""
        st, stats = L.hj_server_wait(self.handle, ticket, timeout_ms)
        if st == L.HJ_ETIMEOUT:
            return st, None, None, None
        if st == L.HJ_EINVAL and ticket not in self._live:
            raise KeyError(ticket)
        V0, out, times, keep = self._live.pop(ticket)
        return st, out, times, stats.as_dict()

    def cancel(self, ticket: int) -> int:
        return L.hj_server_cancel(self.handle, ticket)

    def counters(self) -> dict:
        return L.hj_server_counters(self.handle)

    def close(self):
        if getattr(self, "handle", None):
            L.hj_server_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def implicit_surface(ctx: Context, spec, shapes, dtype="float32", out=None):
    """V0 from implicit primitives (Sec. 2.2), built on the device: a flat CUDA
    tensor of prod(n) elements. shapes: dicts {kind, op, dims, center, axes,
    radius} (see include/hj.h, hj_shape)."""
    import torch
    tdt = getattr(torch, dtype) if isinstance(dtype, str) else dtype
    n = int(np.prod(spec.n))
    if out is None:
        out = torch.empty(n, dtype=tdt, device="cuda:%d" % ctx.device)
    _check_tensor(out, spec, "out")
    L.hj_implicit_surface(ctx.handle, L.make_grid(spec), shapes, L.dtype_code(out.dtype), out)
    return out
