"""Pins of the oracle's ghost cells and upwind derivatives (paper Sec. 2.1, 3.1-3.3).

Each test checks the oracle against something other than its own formulas:
polynomial exactness of ENO/WENO (Osher & Fedkiw Sec. 3.3-3.4), measured
convergence orders, the non-oscillatory property across a jump, a library
routine for periodic wrap, and hand-worked examples of the stated readings.
"""
import math

import numpy as np
import pytest

from oracle import oracle as O


def _exact_padded(f, x0, dx, n):
    """Line values of f at nodes -3 .. n+2 (exact ghosts)."""
    x = x0 + dx * np.arange(-3, n + 3)
    return f(x)


@pytest.mark.parametrize("scheme,degree", [(O.ENO1, 1), (O.ENO2, 2), (O.ENO3, 3), (O.WENO5, 3)])
def test_polynomial_exactness(scheme, degree):
    # ENO of order r is exact on polynomials of degree <= r; every WENO5
    # candidate is a third-order ENO stencil, so any convex weights keep
    # cubics exact.
    rng = np.random.default_rng(3)
    coef = rng.uniform(-2, 2, size=degree + 1)
    f = np.polynomial.Polynomial(coef)
    df = f.deriv()
    n, dx, x0 = 17, 0.1, -0.7
    pm, pp = O.upwind_line(_exact_padded(f, x0, dx, n), dx, scheme)
    x = x0 + dx * np.arange(n)
    np.testing.assert_allclose(pm, df(x), rtol=0, atol=1e-11)
    np.testing.assert_allclose(pp, df(x), rtol=0, atol=1e-11)


@pytest.mark.parametrize("scheme,degree", [(O.ENO1, 2), (O.ENO2, 3), (O.ENO3, 4)])
def test_one_degree_too_high_is_not_exact(scheme, degree):
    # guards against a scheme silently being of the wrong (higher) order
    f = np.polynomial.Polynomial([0.3] + [0.0] * (degree - 1) + [1.0])
    n, dx, x0 = 9, 0.25, 0.1
    pm, _ = O.upwind_line(_exact_padded(f, x0, dx, n), dx, scheme)
    x = x0 + dx * np.arange(n)
    assert np.max(np.abs(pm - f.deriv()(x))) > 1e-6


def test_weno5_ideal_weights_exact_for_quintics():
    # with the linear weights (0.1, 0.6, 0.3) the three candidates combine into
    # the fifth-order upwind-biased stencil on six differences: exact to degree 5
    f = np.polynomial.Polynomial([0.1, -0.4, 0.9, 0.3, -0.7, 0.5])
    n, dx, x0 = 13, 0.125, -0.8
    pm, pp = O.upwind_line(_exact_padded(f, x0, dx, n), dx, O.WENO5, weno_ideal=True)
    x = x0 + dx * np.arange(n)
    np.testing.assert_allclose(pm, f.deriv()(x), atol=1e-11)
    np.testing.assert_allclose(pp, f.deriv()(x), atol=1e-11)
    # ... and the nonlinear weights alone are not exact on a quintic
    pm2, _ = O.upwind_line(_exact_padded(f, x0, dx, n), dx, O.WENO5)
    assert np.max(np.abs(pm2 - f.deriv()(x))) > 1e-9


@pytest.mark.parametrize("scheme,order", [(O.ENO1, 1.0), (O.ENO2, 2.0), (O.ENO3, 3.0), (O.WENO5, 4.5)])
def test_convergence_order(scheme, order):
    # smooth function with no critical point on [0, 1]; L_inf error of p- and p+
    f = lambda x: np.sin(x + 0.3)
    df = lambda x: np.cos(x + 0.3)
    errs = []
    Ns = [32, 64, 128, 256, 512]
    for N in Ns:
        dx = 1.0 / N
        pm, pp = O.upwind_line(_exact_padded(f, 0.0, dx, N + 1), dx, scheme)
        x = dx * np.arange(N + 1)
        errs.append(max(np.max(np.abs(pm - df(x))), np.max(np.abs(pp - df(x)))))
    rates = [math.log2(errs[k] / errs[k + 1]) for k in range(len(errs) - 1)]
    # the finest levels can touch round-off for WENO5; use the first three ratios
    assert min(rates[:3]) >= order - 0.15, (errs, rates)


def test_weno5_non_oscillatory_across_jump():
    # A jump between nodes j and j+1. At node i = j-1 the left derivative's
    # third candidate crosses the jump; the smoothness weights must suppress
    # it, leaving the smooth one-sided value (here exactly the slope 0.01).
    n, dx = 20, 0.1
    x = dx * np.arange(-3, n + 3)
    v = 0.01 * x + np.where(np.arange(-3, n + 3) > 10, 1.0, 0.0)
    pm, pp = O.upwind_line(v, dx, O.WENO5)
    i = 9  # j = 10
    assert abs(pm[i] - 0.01) < 1e-9
    # far from the jump the data is linear and both sides are exact
    assert abs(pp[3] - 0.01) < 1e-12 and abs(pm[16] - 0.01) < 1e-12
    # and on the jump itself the derivative is bounded by the jump slope
    assert np.all(np.abs(pm) <= 1.0 / dx + 1e-9)


def _golden(name):
    import os
    vals = {}
    with open(os.path.join(os.path.dirname(__file__), "golden", name)) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                key, rest = line.split(":", 1)
                vals[key.strip()] = [float(t) for t in rest.split()]
    return vals


def test_eno2_tie_picks_left_candidate():
    # Reading R2, worked by hand in tests/golden/eno2_tie.txt
    g = _golden("eno2_tie.txt")
    pm, _ = O.upwind_line(np.array(g["padded"]), g["dx"][0], O.ENO2)
    assert pm[int(g["node"][0])] == g["pminus"][0]


def test_periodic_padding_matches_wrap():
    rng = np.random.default_rng(0)
    for n in (1, 2, 3, 5, 11):
        line = rng.normal(size=n)
        out = O.pad_line(line, periodic=True)
        np.testing.assert_array_equal(out, np.take(line, np.arange(-3, n + 3), mode="wrap"))


def test_extrapolation_worked_examples():
    # Reading R3, worked by hand in tests/golden/ghost_extrapolation.txt
    g = _golden("ghost_extrapolation.txt")
    for k in ("a", "b"):
        out = O.pad_line(np.array(g["line_" + k]), periodic=False)
        np.testing.assert_array_equal(out[:3], g["away_low_" + k])    # nodes -3, -2, -1
        np.testing.assert_array_equal(out[-3:], g["away_high_" + k])  # nodes n, n+1, n+2
    out = O.pad_line(np.array(g["line_a"]), periodic=False, extrap=O.EXTRAP_LINEAR)
    np.testing.assert_array_equal(out[:3], g["linear_low_a"])


def test_extrapolation_never_crosses_zero():
    rng = np.random.default_rng(1)
    for _ in range(200):
        line = rng.normal(size=rng.integers(2, 9))
        out = O.pad_line(line, periodic=False)
        lo, hi = out[:3], out[-3:]
        assert np.all(np.sign(lo) * np.sign(line[0]) >= 0) and np.all(np.abs(lo) >= abs(line[0]))
        assert np.all(np.sign(hi) * np.sign(line[-1]) >= 0) and np.all(np.abs(hi) >= abs(line[-1]))


def test_extrapolated_linear_data_is_exact_at_the_boundary():
    # positive, outward-increasing linear data: the away-from-zero rule equals
    # linear extrapolation, so every scheme is exact up to the edge nodes
    class G:
        n = (12,)
        lo = (0.0,)
        hi = (1.1,)
        periodic = ()
    x = np.linspace(0.0, 1.1, 12)
    V = np.asfortranarray(3.0 + 0.0 * x)  # constant positive: slope 0 both sides
    V = 1.0 + np.abs(x - 0.55)  # V-shape: increasing outward on both ends
    for scheme in (O.ENO1, O.ENO2, O.ENO3, O.WENO5):
        m = O.method(scheme=scheme, dynamics=O.DYN_ADVECT, params=(1.0,))
        pm, pp = O.upwind(G, m, V, 0)
        assert abs(pm[0] + 1.0) < 1e-12 and abs(pp[0] + 1.0) < 1e-12
        assert abs(pm[-1] - 1.0) < 1e-12 and abs(pp[-1] - 1.0) < 1e-12


def test_upwind_nd_matches_line_along_each_dim():
    # the n-D driver must hand each grid line, in order, to the 1-D routine
    class G:
        n = (5, 7, 4)
        lo = (0.0, -1.0, 0.0)
        hi = (1.0, 1.0, 2 * math.pi)
        periodic = (2,)
    rng = np.random.default_rng(5)
    V = np.asfortranarray(rng.normal(size=G.n))
    m = O.method(scheme=O.WENO5, dynamics=O.DYN_ADVECT, params=(1.0, 1.0, 1.0))
    for d in range(3):
        pm, pp = O.upwind(G, m, V, d)
        dx = O.spacing(G, d)
        for idx in [(0, 0, 0), (4, 6, 3), (2, 3, 1)]:
            sl = list(idx)
            sl[d] = slice(None)
            line = V[tuple(sl)]
            lm, lp = O.upwind_line(O.pad_line(line, periodic=(d == 2)), dx, O.WENO5)
            np.testing.assert_array_equal(pm[tuple(sl)], lm)
            np.testing.assert_array_equal(pp[tuple(sl)], lp)
