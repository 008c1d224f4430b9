"""Shared test helpers: conversions between the oracle's numpy arrays and the
library's flat device tensors, error metrics, and oracle windows for sampled
parity checks on grids too large for the oracle."""
from __future__ import annotations

import math

import numpy as np

from oracle import oracle as O
from paper_2507_11542_gb300 import workloads as W

# The oracle and the library number schemes, dynamics and BRT modes alike;
# both sides are always built from these neutral settings.
DI, AIR3D, DUBINS, NORM, ADVECT, ROTATE, ROCKETS = 1, 2, 3, 4, 5, 6, 7
PARAMS = {DI: (1.0,), AIR3D: (5.0, 5.0, 1.0, 1.0), DUBINS: (1.0, 0.5), NORM: (1.0,),
          ADVECT: (0.7, -1.3, 0.4), ROTATE: (1.3,), ROCKETS: (1.0, 32.0, 1.0, 1.0)}


def oracle_method(scheme=5, dynamics=DI, params=None, brt=1, extrap=0, cfl=0.8, max_step=math.inf, order=3,
                  alpha_global=False, alpha_box=False):
    return O.method(scheme=scheme, dynamics=dynamics, params=PARAMS[dynamics] if params is None else params,
                    brt=brt, extrap=extrap, cfl=cfl, max_step=max_step, order=order, alpha_global=alpha_global,
                    alpha_box=alpha_box)


def lib_method(scheme=5, dynamics=DI, params=None, brt=1, extrap=0, cfl=0.8, max_step=math.inf, order=3,
               alpha_global=False, alpha_box=False, kernel=0, tile=(0, 0, 0, 0)):
    """kernel: 0 automatic, 1 the row kernel, 2 the one-node-per-thread
    kernel; tile: the row kernel's pinned shape (ty, tz, occ, flags)."""
    from paper_2507_11542_gb300 import solver
    return solver.method(scheme=scheme, dynamics=dynamics, params=PARAMS[dynamics] if params is None else params,
                         brt=brt, extrap=extrap, cfl=cfl, max_step=max_step, order=order,
                         alpha_mode=2 if alpha_box else (1 if alpha_global else 0), kernel=kernel,
                         tile_override=tuple(tile))


def to_dev(V, dtype="float64"):
    import torch
    flat = np.ascontiguousarray(np.asarray(V).ravel(order="F"))
    return torch.from_numpy(flat).to(device="cuda", dtype=getattr(torch, dtype)).contiguous()


def to_host(t, n):
    return t.detach().double().cpu().numpy().reshape(tuple(n), order="F")


def rel_err(a, ref):
    scale = max(float(np.max(np.abs(ref))), 1e-300)
    return float(np.max(np.abs(np.asarray(a) - np.asarray(ref)))) / scale


def zero_set_displacement(V, Vref, spec, margin=0):
    """Zero-level-set displacement of V against Vref, in grid cells: over nodes
    within two cells of Vref's zero set, |V - Vref| / (|grad_h Vref| dx).
    margin > 0 leaves out nodes closer than that many cells to a non-periodic
    edge, where the away-from-zero ghost rule flips with the sign of V."""
    dxs = [(spec.hi[d] - spec.lo[d]) / (spec.n[d] if d in spec.periodic else spec.n[d] - 1)
           for d in range(len(spec.n))]
    grads = np.gradient(Vref, *dxs)
    if len(spec.n) == 1:
        grads = [grads]
    gnorm = np.sqrt(sum(g * g for g in grads))
    h = min(dxs)
    near = np.abs(Vref) < 2.0 * h * np.maximum(gnorm, 1e-12)
    if margin > 0:
        inner = np.ones(Vref.shape, dtype=bool)
        for d in range(len(spec.n)):
            if d in spec.periodic:
                continue
            sl = [slice(None)] * len(spec.n)
            sl[d] = slice(0, margin)
            inner[tuple(sl)] = False
            sl[d] = slice(spec.n[d] - margin, None)
            inner[tuple(sl)] = False
        near &= inner
    if not near.any():
        return 0.0
    return float(np.max(np.abs(V - Vref)[near] / (np.maximum(gnorm[near], 1e-12) * h)))


def window_spec(spec, center, half=10):
    """A sub-grid around `center` whose output at the center after one RK3
    step equals the full grid's (each stage reads 3 nodes per side, so 9
    nodes suffice). Returns (window GridSpec, index arrays, center in window).
    Real grid edges are kept (so the true ghost rule applies); periodic
    dimensions longer than the window are unwrapped into a plain line."""
    idx, lo, hi, n, periodic, cw = [], [], [], [], [], []
    for d in range(len(spec.n)):
        N = spec.n[d]
        per = d in spec.periodic
        dx = (spec.hi[d] - spec.lo[d]) / (N if per else N - 1)
        c = center[d]
        if per and N > 2 * half + 1:
            ii = np.arange(c - half, c + half + 1)
            idx.append(ii % N)
            lo.append(spec.lo[d] + (c - half) * dx)
            hi.append(spec.lo[d] + (c + half) * dx)
            n.append(2 * half + 1)
            cw.append(half)
        elif per:
            idx.append(np.arange(N))
            lo.append(spec.lo[d])
            hi.append(spec.hi[d])
            n.append(N)
            periodic.append(d)
            cw.append(c)
        else:
            a, b = max(0, c - half), min(N - 1, c + half)
            idx.append(np.arange(a, b + 1))
            lo.append(spec.lo[d] + a * dx)
            hi.append(spec.lo[d] + b * dx)
            n.append(b - a + 1)
            cw.append(c - a)
    return W.GridSpec(tuple(n), tuple(lo), tuple(hi), tuple(periodic)), idx, tuple(cw)


def oracle_window_step(spec, V, center, m, dt, half=10):
    ws, idx, cw = window_spec(spec, center, half)
    sub = V[np.ix_(*idx)]
    out = O.rk3_step(ws, m, np.asfortranarray(sub), dt)
    return out[cw]


def crossing_displacement(V, Vref, spec):
    """Zero-level-set displacement in cells measured on grid edges: where both
    fields change sign along an edge, |s - s_ref| of the interpolated crossing
    points; where only one does, the distance from that crossing to the
    nearer end of the edge (a lower bound of the move). Max over all edges."""
    worst = 0.0
    pos, pos_r = V > 0, Vref > 0
    for d in range(len(spec.n)):
        a = [slice(None)] * len(spec.n)
        b = [slice(None)] * len(spec.n)
        a[d] = slice(0, spec.n[d] - 1)
        b[d] = slice(1, spec.n[d])
        a, b = tuple(a), tuple(b)
        c = pos[a] != pos[b]
        cr = pos_r[a] != pos_r[b]
        with np.errstate(divide="ignore", invalid="ignore"):
            s = np.nan_to_num(V[a] / (V[a] - V[b]))
            sr = np.nan_to_num(Vref[a] / (Vref[a] - Vref[b]))
        both = c & cr
        if both.any():
            worst = max(worst, float(np.max(np.abs(s - sr)[both])))
        only = c ^ cr
        if only.any():
            t = np.where(c, s, sr)[only]
            worst = max(worst, float(np.max(np.minimum(t, 1.0 - t))))
    return worst


def zero_set_meets_extrapolated_edge(Vref, spec):
    """Whether the zero level set of Vref reaches a non-periodic boundary face."""
    for d in range(len(spec.n)):
        if d in spec.periodic:
            continue
        for idx in (0, spec.n[d] - 1):
            face = np.take(Vref, idx, axis=d)
            if (face > 0).any() and (face <= 0).any():
                return True
    return False
