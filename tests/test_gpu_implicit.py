"""Initial surfaces built on the device (hj_implicit_surface) against the
oracle's (oracle/implicit.py), and solves started from them."""
from __future__ import annotations

import numpy as np
import pytest

from oracle import implicit as I
from oracle import oracle as O
from paper_2507_11542_gb300 import workloads as W
from helpers import AIR3D, lib_method, oracle_method, rel_err, to_dev, to_host

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_2507_11542_gb300 import solver
    c = solver.Context(0)
    yield c
    c.close()


MIX3 = [{"kind": I.SPHERE, "center": (0.2, -0.3, 0.1), "radius": 0.7},
        {"kind": I.SPHERE, "op": I.UNION, "dims": (0, 2), "center": (-0.6, 0.0, 0.4), "radius": 0.3},
        {"kind": I.RECTANGLE, "op": I.INTERSECT, "center": (0.0, 0.0, 0.0), "axes": (0.9, 0.8, 1.5)},
        {"kind": I.ELLIPSOID, "op": I.SUBTRACT, "center": (0.3, 0.2, 0.0), "axes": (1.0, 4.0, 9.0), "radius": 0.05}]


@pytest.mark.parametrize("shape,periodic", [((37, 29, 23), ()), ((40, 31, 19), (2,))])
@pytest.mark.parametrize("dtype", ["float64", "float32"])
def test_surface_matches_oracle(ctx, shape, periodic, dtype):
    from paper_2507_11542_gb300 import solver
    g = W.GridSpec(shape, (-1.2, -1.0, -0.8), (1.1, 1.3, 0.9), periodic)
    got = to_host(solver.implicit_surface(ctx, g, MIX3, dtype), g.n)
    ref = I.implicit_surface(g, MIX3)
    scale = float(np.max(np.abs(ref)))
    tol = 1e-14 if dtype == "float64" else 1e-6  # FP32: coordinates and terms rounded in FP32
    assert np.max(np.abs(got - ref)) <= tol * scale


def test_surface_2d_and_4d_and_host_output(ctx):
    from paper_2507_11542_gb300 import _lib as L
    g2 = W.GridSpec((51, 33), (-1.0, -1.0), (1.0, 1.0))
    sh2 = [{"kind": I.RECTANGLE, "center": (0.1, 0.0), "axes": (0.5, 0.25)},
           {"kind": I.SPHERE, "op": I.UNION, "center": (-0.5, 0.5), "radius": 0.2}]
    host = np.empty(51 * 33)
    L.hj_implicit_surface(ctx.handle, L.make_grid(g2), sh2, L.HJ_F64, host, out_on_device=False)
    np.testing.assert_allclose(host.reshape(g2.n, order="F"), I.implicit_surface(g2, sh2), rtol=0, atol=1e-15)
    from paper_2507_11542_gb300 import solver
    g4, _ = W.dubins4d(21)
    sh4 = [{"kind": I.SPHERE, "dims": (0, 1), "center": (0.5, -1.0), "radius": 1.0},
           {"kind": I.RECTANGLE, "op": I.INTERSECT, "dims": (3,), "center": (0, 0, 0, 1.0), "axes": (0, 0, 0, 0.6)}]
    got = to_host(solver.implicit_surface(ctx, g4, sh4, "float64"), g4.n)
    np.testing.assert_allclose(got, I.implicit_surface(g4, sh4), rtol=0, atol=1e-15)


def test_surface_full_size_sphere_sampled(ctx):
    # the 512^3 expanding-sphere initial surface, checked at sampled nodes
    from paper_2507_11542_gb300 import solver
    g, _ = W.expanding_sphere(512)
    sh = [{"kind": I.SPHERE, "center": (0.0, 0.0, 0.0), "radius": 0.25}]
    V = solver.implicit_surface(ctx, g, sh, "float32")
    rng = np.random.default_rng(3)
    idx = rng.integers(0, 512, size=(64, 3))
    flat = idx[:, 0] + 512 * (idx[:, 1] + 512 * idx[:, 2])
    got = V[flat.tolist()].double().cpu().numpy()
    h = 2.0 / 511
    X = -1.0 + idx * h
    ref = np.sqrt((X ** 2).sum(axis=1)) - 0.25
    assert np.max(np.abs(got - ref)) <= 4e-7 * 1.5


def test_solve_from_device_surface_equals_host_surface(ctx):
    from paper_2507_11542_gb300 import solver
    g, V0 = W.air3d(41)
    sh = [{"kind": I.SPHERE, "dims": (0, 1), "center": (0.0, 0.0), "radius": 5.0}]
    v0d = solver.implicit_surface(ctx, g, sh, "float64")
    assert rel_err(to_host(v0d, g.n), V0) <= 1e-15
    ts = [0.0, 0.5]
    m = lib_method(dynamics=AIR3D)
    a, _, _ = solver.solve(ctx, g, m, v0d, ts)
    b, _, _ = solver.solve(ctx, g, m, to_dev(V0), ts)
    assert rel_err(to_host(a[1], g.n), to_host(b[1], g.n)) <= 1e-12
    ref, _, _ = O.solve(g, oracle_method(dynamics=AIR3D), V0, ts)
    assert rel_err(to_host(a[1], g.n), ref[1]) <= 1e-12


def test_surface_errors(ctx):
    from paper_2507_11542_gb300 import _lib as L, solver
    g = W.GridSpec((9, 9), (-1.0, -1.0), (1.0, 1.0))
    bad = [
        [],
        [{"kind": 9, "center": (0, 0), "radius": 1.0}],
        [{"kind": I.SPHERE, "dims": (2,), "center": (0, 0, 0), "radius": 1.0}],
        [{"kind": I.ELLIPSOID, "center": (0, 0), "axes": (1.0, 0.0), "radius": 1.0}],
        [{"kind": I.SPHERE, "center": (0, 0), "radius": 1.0}, {"kind": I.SPHERE, "op": 7, "center": (0, 0)}],
        [{"kind": I.SPHERE, "center": (0, float("nan")), "radius": 1.0}],
        [{"kind": I.SPHERE, "center": (0, 0), "radius": 1.0}] * 33,
    ]
    for shapes in bad:
        with pytest.raises((L.HJError, ValueError)) as e:
            solver.implicit_surface(ctx, g, shapes, "float64")
        if isinstance(e.value, L.HJError):
            assert e.value.status == L.HJ_EINVAL
