"""Oracle of the initial surfaces (test infrastructure: only the tests, the
smoke check and the benchmark's CPU baseline use this package).

Implicit primitives on the grid container and their Boolean combinations
(Sec. 2.2 and its ellipsoid listing), in plain FP64 numpy, written from the
definitions:
  sphere     sqrt(sum_d (x_d - c_d)^2) - r        over the dimensions listed
  ellipsoid  sum_d a_d (x_d - c_d)^2 - r          (the listing's quadratic)
  rectangle  max_d (|x_d - c_d| - h_d)
  union min, intersection max, subtraction max(v, -s), applied in order.
Node coordinates are lo_d + i dx_d with dx_d = (hi - lo)/n for a periodic
dimension, (hi - lo)/(n - 1) otherwise (Sec. 2.1).
"""
from __future__ import annotations

import numpy as np

SPHERE, ELLIPSOID, RECTANGLE = 1, 2, 3
UNION, INTERSECT, SUBTRACT = 1, 2, 3


def node_coordinates(grid):
    """Broadcastable coordinate arrays, one per dimension, of the grid's nodes."""
    D = len(grid.n)
    out = []
    for d in range(D):
        n = int(grid.n[d])
        dx = (grid.hi[d] - grid.lo[d]) / (n if d in grid.periodic else n - 1)
        shape = [1] * D
        shape[d] = n
        out.append((grid.lo[d] + np.arange(n, dtype=np.float64) * dx).reshape(shape))
    return out


def primitive(grid, shape):
    X = node_coordinates(grid)
    D = len(grid.n)
    dims = list(shape.get("dims", range(len(shape.get("center", ())))))
    c = list(shape.get("center", ())) + [0.0] * 4
    a = list(shape.get("axes", ())) + [0.0] * 4
    kind = shape["kind"]
    if kind == RECTANGLE:
        v = None
        for d in dims:
            q = np.abs(X[d] - c[d]) - a[d]
            v = q if v is None else np.maximum(v, q)
        return np.broadcast_to(v, tuple(grid.n))
    acc = np.zeros([1] * D)
    for d in dims:
        q = X[d] - c[d]
        acc = acc + (a[d] * (q * q) if kind == ELLIPSOID else q * q)
    if kind == SPHERE:
        return np.broadcast_to(np.sqrt(acc) - shape["radius"], tuple(grid.n))
    if kind == ELLIPSOID:
        return np.broadcast_to(acc - shape["radius"], tuple(grid.n))
    raise ValueError("unknown shape kind %r" % kind)


def implicit_surface(grid, shapes):
    """V at every node (array of shape grid.n) of the shapes combined in order."""
    v = np.array(primitive(grid, shapes[0]), dtype=np.float64)
    for sh in shapes[1:]:
        s = primitive(grid, sh)
        op = sh.get("op", UNION)
        if op == UNION:
            v = np.minimum(v, s)
        elif op == INTERSECT:
            v = np.maximum(v, s)
        elif op == SUBTRACT:
            v = np.maximum(v, -s)
        else:
            raise ValueError("unknown operation %r" % op)
    return np.asfortranarray(v)
