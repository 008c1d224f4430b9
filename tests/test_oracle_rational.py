"""One full TVD-RK3 step of the oracle against the same step computed with 80
significant digits (Python's decimal module) on tiny grids.

The rational step is written here from the textbook definitions, not from the
oracle's code:
- ghost nodes by the rule of Sec. 2.1 (reading: the outermost slope continued
  away from the zero level set) or by periodic wrap;
- per-node two-sided WENO5 from divided differences (Sec. 3.3; Jiang & Peng
  2000, Osher & Fedkiw Sec. 3.4), eps = 1e-6 max(v_k^2) + 1e-99;
- the Lax-Friedrichs term with each dynamics' alpha (Sec. 4);
- the BRT clamp min(0, H) (Sec. 6.1);
- the Shu-Osher TVD-RK3 combination (Sec. 5).

Every operation is rational once the grid spacing, coordinates, dt, and the
cos/sin of the heading angles are taken as the doubles the oracle uses. So
the 80-digit evaluation equals the exact step to about 1e-75, and the FP64
oracle must match it to rounding: 1e-14 of max|V|. (Exact fractions would
give the same answer, but their denominators grow past practical size within
the three stages.)
"""
import math
from decimal import Decimal, localcontext

import numpy as np

from oracle import oracle as O
from paper_2507_11542_gb300 import workloads as W

DIGITS = 80
TOL = 1e-14


def Q(a, b=1):
    """a/b, or the exact value of a double a, in the current 80-digit context."""
    return Decimal(a) / Decimal(b) if b != 1 else Decimal(a)


def _sign(v):
    return (v > 0) - (v < 0)


def _padded_line(line, periodic):
    """The line with three ghost nodes on each side."""
    n = len(line)
    out = []
    for i in range(-3, n + 3):
        if 0 <= i < n:
            out.append(line[i])
        elif periodic:
            out.append(line[i % n])
        else:
            edge, inner, m = (line[0], line[1], -i) if i < 0 else (line[n - 1], line[n - 2], i - (n - 1))
            out.append(edge + m * abs(edge - inner) * _sign(edge))
    return out


def _weno5(v1, v2, v3, v4, v5):
    """WENO5 from five divided differences (Jiang & Peng weights)."""
    phi1 = v1 / 3 - Q(7, 6) * v2 + Q(11, 6) * v3
    phi2 = -v2 / 6 + Q(5, 6) * v3 + v4 / 3
    phi3 = v3 / 3 + Q(5, 6) * v4 - v5 / 6
    s1 = Q(13, 12) * (v1 - 2 * v2 + v3) ** 2 + Q(1, 4) * (v1 - 4 * v2 + 3 * v3) ** 2
    s2 = Q(13, 12) * (v2 - 2 * v3 + v4) ** 2 + Q(1, 4) * (v2 - v4) ** 2
    s3 = Q(13, 12) * (v3 - 2 * v4 + v5) ** 2 + Q(1, 4) * (3 * v3 - 4 * v4 + v5) ** 2
    eps = Q(1, 10 ** 6) * max(v * v for v in (v1, v2, v3, v4, v5)) + Q(1, 10 ** 99)
    a1, a2, a3 = Q(1, 10) / (s1 + eps) ** 2, Q(6, 10) / (s2 + eps) ** 2, Q(3, 10) / (s3 + eps) ** 2
    return (a1 * phi1 + a2 * phi2 + a3 * phi3) / (a1 + a2 + a3)


def _one_sided(line, dx, periodic):
    """p- and p+ at every node of a grid line."""
    p = _padded_line(line, periodic)
    d = [(p[j + 1] - p[j]) / dx for j in range(len(p) - 1)]  # d[j]: between padded nodes j and j+1
    pm, pp = [], []
    for i in range(len(line)):
        k = i + 3  # padded index of node i; d[k-1] is the backward difference at i
        pm.append(_weno5(d[k - 3], d[k - 2], d[k - 1], d[k], d[k + 1]))
        pp.append(_weno5(d[k + 2], d[k + 1], d[k], d[k - 1], d[k - 2]))
    return pm, pp


def _spacing(g, d):
    periodic = d in g.periodic
    return (g.hi[d] - g.lo[d]) / (g.n[d] if periodic else g.n[d] - 1)


def _coord(g, d, i):
    return g.lo[d] + float(i) * _spacing(g, d)  # the double the oracle uses


def _term(g, dyn, params, V):
    """ydot = min(0, Hg(x, pbar) + sum_d alpha_d(x) (p+ - p-)/2) at every node."""
    D = len(g.n)
    pm = np.empty((D,) + V.shape, dtype=object)
    pp = np.empty((D,) + V.shape, dtype=object)
    for d in range(D):
        dx = Q(_spacing(g, d))
        other = [range(g.n[e]) for e in range(D) if e != d]
        for rest in np.ndindex(*[len(r) for r in other]):
            idx = list(rest)
            idx.insert(d, slice(None))
            m_, p_ = _one_sided(list(V[tuple(idx)]), dx, d in g.periodic)
            pm[(d,) + tuple(idx)] = m_
            pp[(d,) + tuple(idx)] = p_
    out = np.empty(V.shape, dtype=object)
    for node in np.ndindex(*V.shape):
        x = [Q(_coord(g, d, node[d])) for d in range(D)]
        pb = [(pm[(d,) + node] + pp[(d,) + node]) / 2 for d in range(D)]
        dd = [(pp[(d,) + node] - pm[(d,) + node]) / 2 for d in range(D)]
        if dyn == O.DYN_DOUBLE_INTEGRATOR:  # x' = (x2, u), |u| <= umax, u minimises
            umax = Q(params[0])
            hg = pb[0] * x[1] - umax * abs(pb[1])
            alpha = [abs(x[1]), umax]
        else:  # air3D: a maximises, b minimises
            va, vb, amax, bmax = (Q(p) for p in params)
            psi = _coord(g, 2, node[2])
            c, s = Q(math.cos(psi)), Q(math.sin(psi))
            f0, f1 = -va + vb * c, vb * s
            hg = pb[0] * f0 + pb[1] * f1 + amax * abs(pb[0] * x[1] - pb[1] * x[0] - pb[2]) - bmax * abs(pb[2])
            alpha = [abs(f0) + amax * abs(x[1]), abs(f1) + amax * abs(x[0]), amax + bmax]
        y = hg + sum(alpha[d] * dd[d] for d in range(D))
        out[node] = min(y, Q(0))
    return out


def _rk3_step(g, dyn, params, V0, dt):
    """Shu-Osher TVD-RK3: V1 = V + dt L(V); V2 = 3/4 V + 1/4 (V1 + dt L(V1));
    V3 = 1/3 V + 2/3 (V2 + dt L(V2))."""
    V1 = V0 + dt * _term(g, dyn, params, V0)
    V2 = Q(3, 4) * V0 + Q(1, 4) * (V1 + dt * _term(g, dyn, params, V1))
    return Q(1, 3) * V0 + Q(2, 3) * (V2 + dt * _term(g, dyn, params, V2))


def _compare(g, dyn, params, V0):
    m = O.method(scheme=O.WENO5, dynamics=dyn, params=params, brt=O.BRT_MIN0)
    dt = 0.8 / O.step_bound_inv(g, m)
    got = O.rk3_step(g, m, V0, dt)
    with localcontext() as c:
        c.prec = DIGITS
        exact = _rk3_step(g, dyn, params, np.vectorize(Q, otypes=[object])(V0), Q(dt))
        err = max(abs(Q(float(got[node])) - exact[node]) for node in np.ndindex(*V0.shape))
    scale = float(np.max(np.abs(V0)))
    return float(err) / scale


def test_double_integrator_step_equals_exact_rational_step():
    # 7 x 7 grid, extrapolated edges; V0 a disk's signed distance plus a smooth seeded bump
    g = W.GridSpec((7, 7), (-1.0, -1.0), (1.0, 1.0))
    V0 = W.sphere(g, (0.1, -0.05), 0.5) + 0.05 * W.random_field(g, 3)
    assert _compare(g, O.DYN_DOUBLE_INTEGRATOR, (1.0,), np.asfortranarray(V0)) <= TOL


def test_air3d_step_equals_exact_rational_step():
    # 5 x 5 x 5 grid, psi periodic; the cos and sin of the five headings enter as the doubles
    g = W.GridSpec((5, 5, 5), (-6.0, -10.0, 0.0), (20.0, 10.0, 2.0 * math.pi), (2,))
    V0 = W.sphere(g, (0.0, 0.0), 5.0, dims=(0, 1)) + 0.5 * W.random_field(g, 4)
    assert _compare(g, O.DYN_AIR3D, (5.0, 5.0, 1.0, 1.0), np.asfortranarray(V0)) <= TOL
