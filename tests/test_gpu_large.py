"""Full-size solves of the large configurations: the expanding sphere on a
512^3 grid in FP32 against its Hopf-Lax closed form over the whole horizon,
and the Dubins car on an 81^4 grid in FP32 against the same solve in FP64
(whose single steps the sampled full-size tests check against the oracle)."""
from __future__ import annotations

import math

import numpy as np
import pytest

from paper_2507_11542_gb300 import workloads as W
from helpers import DUBINS, NORM, lib_method, oracle_method, window_spec

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_2507_11542_gb300 import solver
    c = solver.Context(0)
    yield c
    c.close()


def _axis_tensor(spec, d, device):
    import torch
    dx = (spec.hi[d] - spec.lo[d]) / (spec.n[d] if d in spec.periodic else spec.n[d] - 1)
    shape = [1] * len(spec.n)
    shape[d] = spec.n[d]
    return (spec.lo[d] + dx * torch.arange(spec.n[d], device=device, dtype=torch.float64)).reshape(shape), dx


def test_expanding_sphere_512_fp32_matches_hopf_lax():
    # H = -|p| (the front moves outward at unit speed), no BRT: the viscosity
    # solution is V(x, tau) = max(|x| - tau, 0) - r0 (Hopf-Lax), so the zero
    # set is the sphere of radius r0 + tau and |grad V| = 1 outside radius tau.
    import torch
    from paper_2507_11542_gb300 import solver
    c = solver.Context(0)
    try:
        spec, _ = W.expanding_sphere(512)
        r0, tau = 0.25, 0.5
        # V0 built on the device (the grid is 512^3): signed distance to the sphere
        axes = [_axis_tensor(spec, d, "cuda") for d in range(3)]
        h = axes[0][1]
        R = torch.sqrt(axes[0][0] ** 2 + axes[1][0] ** 2 + axes[2][0] ** 2)  # (n0, n1, n2), dimension 0 first
        v0 = (R - r0).to(torch.float32).permute(2, 1, 0).contiguous().reshape(-1)  # dimension 0 fastest
        m = lib_method(dynamics=NORM, brt=0)
        out, times, stats = solver.solve(c, spec, m, v0, [tau])
        assert times[-1] == tau and stats["steps"] > 400
        V = out[-1].reshape(spec.n[2], spec.n[1], spec.n[0]).permute(2, 1, 0).double()
        exact = torch.clamp(R - tau, min=0.0) - r0
        band = (exact.abs() < 2.0 * h)
        disp = float(((V - exact).abs()[band]).max()) / h  # |grad V| = 1 in the band
        print("512^3 FP32 sphere, tau = %.2f: %d steps, zero-set displacement %.3g cells" % (tau, stats["steps"], disp))
        assert disp < 0.1
        # |grad V| = 1 outside radius tau (central differences, away from the front's kink and the box edge)
        g = [(V[2:, 1:-1, 1:-1] - V[:-2, 1:-1, 1:-1]) / (2 * h), (V[1:-1, 2:, 1:-1] - V[1:-1, :-2, 1:-1]) / (2 * h),
             (V[1:-1, 1:-1, 2:] - V[1:-1, 1:-1, :-2]) / (2 * h)]
        gn = torch.sqrt(g[0] ** 2 + g[1] ** 2 + g[2] ** 2)
        Ri = R[1:-1, 1:-1, 1:-1]
        sel = (Ri > tau + 8 * h) & (Ri < 0.95)
        err = float((gn[sel] - 1.0).abs().max())
        print("|grad V| - 1 outside radius tau: max %.3g" % err)
        assert err < 1e-2
    finally:
        c.close()


def _crossings(V, Vref, margin_dims, margin):
    """Edge-crossing zero-set displacement (cells) over grid edges whose nodes
    are at least `margin` nodes from both ends of each dimension in margin_dims."""
    import torch
    worst = 0.0
    D = V.dim()
    inner = torch.ones_like(V, dtype=torch.bool)
    for d in margin_dims:
        idx = torch.arange(V.shape[d], device=V.device)
        keep = (idx >= margin) & (idx < V.shape[d] - margin)
        shape = [1] * D
        shape[d] = V.shape[d]
        inner &= keep.reshape(shape)
    for d in range(D):
        a = [slice(None)] * D
        b = [slice(None)] * D
        a[d] = slice(0, V.shape[d] - 1)
        b[d] = slice(1, V.shape[d])
        va, vb, ra, rb = V[tuple(a)], V[tuple(b)], Vref[tuple(a)], Vref[tuple(b)]
        ok = inner[tuple(a)] & inner[tuple(b)]
        c = ((va > 0) != (vb > 0)) & ok
        cr = ((ra > 0) != (rb > 0)) & ok
        s = va / (va - vb)
        sr = ra / (ra - rb)
        both = c & cr
        if both.any():
            worst = max(worst, float((s - sr).abs()[both].max()))
        only = c ^ cr
        if only.any():
            t = torch.where(c, s, sr)[only]
            worst = max(worst, float(torch.minimum(t, 1 - t).max()))
    return worst


def test_dubins_81_fp32_zero_set_matches_fp64(ctx):
    # The 81^4 Dubins car over the whole horizon (tau = 2, 11 slices), FP32
    # against FP64. The bar (0.1 cell) is checked on edges at least 4 nodes
    # from the speed boundaries v = 0 and v = 2, where the away-from-zero
    # ghost rule switches with the sign of V and FP32 rounding can flip it.
    import torch
    from paper_2507_11542_gb300 import solver
    spec, V0 = W.dubins4d(81)
    ts = W.slice_times(2.0)
    m = lib_method(dynamics=DUBINS, brt=1)
    v0 = torch.from_numpy(np.ascontiguousarray(V0.ravel(order="F")))
    o64, t64, s64 = solver.solve(ctx, spec, m, v0.to("cuda", torch.float64), ts)
    o32, t32, s32 = solver.solve(ctx, spec, m, v0.to("cuda", torch.float32), ts)
    assert s64["steps"] == s32["steps"] and np.array_equal(t64, t32)
    shape = tuple(reversed(spec.n))
    for k in (5, 10):
        V64 = o64[k].reshape(shape)
        V32 = o32[k].reshape(shape).double()
        # tensor dims are (v, theta, y, x): the speed is tensor dimension 0
        disp = _crossings(V32, V64, margin_dims=(0,), margin=4)
        dv = float((V32 - V64).abs().max()) / float(V64.abs().max())
        print("Dubins 81^4 slice %d: FP32 zero-set displacement %.3g cells, max|dV|/max|V| %.3g" % (k, disp, dv))
        assert disp < 0.1
        # FP32 rounding over ~140 steps, largest next to the speed boundaries (measured 3e-3 at tau = 2)
        assert dv < 1e-2


def test_grid_beyond_32_bit_indices_sampled(ctx):
    # 1000 x 1000 x 2148 nodes (more than 2^31): beyond the row kernel's 32-bit
    # flat indices, so the step runs on the one-node-per-thread kernel with
    # 64-bit indices. V0 is built on the device (8.6 GB per FP32 array); after
    # one RK3 step, sampled nodes (corners, faces, interior) are compared with
    # the oracle's step on the window around each.
    import torch
    from oracle import oracle as O
    from paper_2507_11542_gb300 import _lib as L, solver
    spec = W.GridSpec((1000, 1000, 2148), (-1.0,) * 3, (1.0,) * 3)
    n0, n1, n2 = spec.n
    assert n0 * n1 * n2 > 2 ** 31
    shapes = [dict(kind=L.HJ_SHAPE_SPHERE, op=L.HJ_SHAPE_UNION, dims=(0, 1, 2), center=(0.1, -0.05, 0.0),
                   radius=0.5)]
    V = solver.implicit_surface(ctx, spec, shapes, "float32")
    m_l = lib_method(dynamics=NORM, brt=0)
    m_o = oracle_method(dynamics=NORM, brt=0)
    dt = 0.8 / solver.step_bound(ctx, spec, m_l)
    rng = np.random.default_rng(11)
    nodes = [(0, 0, 0), (n0 - 1, n1 - 1, n2 - 1), (n0 // 2, n1 // 2, n2 // 2), (1, n1 - 2, n2 - 2),
             (450, 500, 1074), (0, 517, 2147)]
    nodes += [tuple(int(rng.integers(0, m)) for m in spec.n) for _ in range(4)]

    def gather(ws_idx):
        flat = (ws_idx[0][:, None, None] + n0 * (ws_idx[1][None, :, None] + n1 * ws_idx[2][None, None, :]))
        return torch.take(V, torch.from_numpy(flat.astype(np.int64)).to(V.device)).cpu().numpy()

    windows = []
    for node in nodes:
        ws, idx, cw = window_spec(spec, node)
        windows.append((ws, cw, np.asfortranarray(gather(idx).astype(np.float64))))
    solver.rk3_step(ctx, spec, m_l, V, dt)
    flat_nodes = torch.tensor([i + n0 * (j + n1 * k) for i, j, k in nodes], dtype=torch.int64, device=V.device)
    got = torch.take(V, flat_nodes).cpu().numpy()
    scale = max(float(np.max(np.abs(w[2]))) for w in windows)
    for (ws, cw, w0), g_val, node in zip(windows, got, nodes):
        want = O.rk3_step(ws, m_o, w0, dt)[cw]
        assert abs(float(g_val) - want) <= 2e-6 * scale, (node, float(g_val), want)
    del V
    torch.cuda.empty_cache()
