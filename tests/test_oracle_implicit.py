"""Pins of the oracle's initial surfaces (Sec. 2.2: implicit primitives and
Boolean operations): library distance routines, hand-worked values of the
rectangle and the ellipsoid listing, and set semantics of the operations."""
from __future__ import annotations

import numpy as np

from oracle import implicit as I
from paper_2507_11542_gb300 import workloads as W


def _grid(n, lo, hi, periodic=()):
    return W.GridSpec(tuple(n), tuple(lo), tuple(hi), tuple(periodic))


def test_sphere_is_the_euclidean_distance_minus_radius():
    g = _grid((17, 13, 11), (-1.0, -2.0, -0.5), (1.5, 1.0, 2.0))
    c, r = (0.3, -0.4, 0.7), 0.6
    V = I.implicit_surface(g, [{"kind": I.SPHERE, "center": c, "radius": r}])
    X = np.stack(np.meshgrid(*[g.axis(d) for d in range(3)], indexing="ij"))
    ref = np.linalg.norm(X - np.array(c).reshape(3, 1, 1, 1), axis=0) - r
    np.testing.assert_allclose(V, ref, rtol=0, atol=1e-15)


def test_cylinder_ignores_the_other_dimensions():
    g = _grid((9, 7, 8), (-1.0, -1.0, 0.0), (1.0, 1.0, 2 * np.pi), periodic=(2,))
    V = I.implicit_surface(g, [{"kind": I.SPHERE, "dims": (0, 1), "center": (0.2, -0.1), "radius": 0.5}])
    for k in range(1, 8):
        np.testing.assert_array_equal(V[:, :, k], V[:, :, 0])
    # and it matches the workload generator's cylinder (an independent construction)
    ref = W.sphere(g, (0.2, -0.1), 0.5, dims=(0, 1))
    np.testing.assert_allclose(V, ref, rtol=0, atol=1e-15)


def test_rectangle_worked_values():
    # box centred at (0, 0) with half-widths (1, 0.5); grid spacing 0.25 on [-2, 2]^2
    g = _grid((17, 17), (-2.0, -2.0), (2.0, 2.0))
    V = I.implicit_surface(g, [{"kind": I.RECTANGLE, "center": (0.0, 0.0), "axes": (1.0, 0.5)}])
    idx = lambda x, y: (int(round((x + 2) / 0.25)), int(round((y + 2) / 0.25)))
    assert V[idx(0, 0)] == -0.5          # centre: nearest face y = +-0.5
    assert V[idx(0.5, 0)] == -0.5        # max(-0.5, -0.5)
    assert V[idx(1, 0)] == 0.0           # on the face x = 1
    assert V[idx(0, 0.5)] == 0.0         # on the face y = 0.5
    assert V[idx(2, 0)] == 1.0           # one unit outside along the x normal
    assert V[idx(0, -1.5)] == 1.0        # one unit outside along the y normal
    assert V[idx(1.5, 1.0)] == 0.5       # max(0.5, 0.5) beyond a corner


def test_ellipsoid_listing_values():
    # the listing's quadratic x^2 + 4 y^2 - r (2-D), r = 1, spacing 0.5 on [-2, 2]^2
    g = _grid((9, 9), (-2.0, -2.0), (2.0, 2.0))
    V = I.implicit_surface(g, [{"kind": I.ELLIPSOID, "center": (0.0, 0.0), "axes": (1.0, 4.0), "radius": 1.0}])
    idx = lambda x, y: (int(round((x + 2) / 0.5)), int(round((y + 2) / 0.5)))
    assert V[idx(1, 0)] == 0.0 and V[idx(-1, 0)] == 0.0 and V[idx(0, 0.5)] == 0.0 and V[idx(0, -0.5)] == 0.0
    assert V[idx(0.5, 0.5)] == 0.25 and V[idx(0, 0)] == -1.0 and V[idx(2, 1)] == 7.0
    # 3-D: x^2 + 4 y^2 + 9 z^2 - r
    g3 = _grid((5, 5, 5), (-1.0, -1.0, -1.0), (1.0, 1.0, 1.0))
    V3 = I.implicit_surface(g3, [{"kind": I.ELLIPSOID, "center": (0, 0, 0), "axes": (1.0, 4.0, 9.0), "radius": 2.0}])
    assert V3[4, 2, 2] == -1.0 and V3[2, 4, 2] == 2.0 and V3[2, 2, 3] == 0.25


def test_boolean_operations_follow_set_semantics():
    g = _grid((41, 41), (-2.0, -2.0), (2.0, 2.0))
    A = {"kind": I.SPHERE, "center": (-0.4, 0.0), "radius": 0.8}
    B = {"kind": I.RECTANGLE, "center": (0.5, 0.2), "axes": (0.6, 0.9)}
    a = I.implicit_surface(g, [A]) < 0
    b = I.implicit_surface(g, [B]) < 0
    for op, want in ((I.UNION, a | b), (I.INTERSECT, a & b), (I.SUBTRACT, a & ~b)):
        V = I.implicit_surface(g, [A, dict(B, op=op)])
        # strict interiors agree; nodes exactly on a boundary (V == 0) are left out
        on = np.isclose(I.implicit_surface(g, [A]), 0) | np.isclose(I.implicit_surface(g, [B]), 0)
        np.testing.assert_array_equal((V < 0)[~on], want[~on])
    assert (a & ~b).any() and (a & b).any()
