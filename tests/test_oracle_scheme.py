"""Pins of the oracle's Hamiltonians, Lax-Friedrichs term, CFL bound, TVD-RK3
step and time loop (paper Sec. 4, 5 and 6.1).

The Hamiltonians are checked against brute-force optimisation over a grid of
controls of the dynamics as stated in the workload table; the scheme pieces
against textbook special cases (LF with alpha = |c| is the upwind scheme;
Shu-Osher RK3 of a linear operator is its third-order Taylor polynomial) and
against hand-derived step counts.
"""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_2507_11542_gb300 import workloads as W

U = np.linspace(-1.0, 1.0, 41)  # controls, endpoints included


def _brute_hg(dyn, params, x, p):
    if dyn == O.DYN_DOUBLE_INTEGRATOR:
        (umax,) = params
        return min(p[0] * x[1] + p[1] * (umax * u) for u in U)
    if dyn == O.DYN_AIR3D:
        va, vb, amax, bmax = params
        X, Y, psi = x
        best = -np.inf
        for a in amax * U:          # evader maximises
            worst = np.inf
            for b in bmax * U:      # pursuer minimises
                f = (-va + vb * math.cos(psi) + a * Y, vb * math.sin(psi) - a * X, b - a)
                worst = min(worst, float(np.dot(p, f)))
            best = max(best, worst)
        return best
    if dyn == O.DYN_DUBINS4D:
        wmax, accmax = params
        X, Y, th, v = x
        return min(float(np.dot(p, (v * math.cos(th), v * math.sin(th), w, acc)))
                   for w in wmax * U for acc in accmax * U)
    if dyn == O.DYN_ROCKETS:
        # Sec. 6.1 game: the evader's thrust ue maximises, the pursuer's up minimises
        a, g, uemax, upmax = params
        X, Z, th = x
        best = -np.inf
        for ue in uemax * U:
            worst = np.inf
            for up in upmax * U:
                f = (a * math.cos(th) + ue * X, a * math.sin(th) + a - g + up * X, up - ue)
                worst = min(worst, float(np.dot(p, f)))
            best = max(best, worst)
        return best
    raise AssertionError


def _brute_alpha(dyn, params, x):
    if dyn == O.DYN_DOUBLE_INTEGRATOR:
        (umax,) = params
        return [abs(x[1]), max(abs(umax * u) for u in U)]
    if dyn == O.DYN_AIR3D:
        va, vb, amax, bmax = params
        X, Y, psi = x
        fs = [(-va + vb * math.cos(psi) + a * Y, vb * math.sin(psi) - a * X, b - a)
              for a in amax * U for b in bmax * U]
        return list(np.max(np.abs(np.array(fs)), axis=0))
    if dyn == O.DYN_DUBINS4D:
        wmax, accmax = params
        X, Y, th, v = x
        fs = [(v * math.cos(th), v * math.sin(th), w, acc) for w in wmax * U for acc in accmax * U]
        return list(np.max(np.abs(np.array(fs)), axis=0))
    if dyn == O.DYN_ROCKETS:
        a, g, uemax, upmax = params
        X, Z, th = x
        fs = [(a * math.cos(th) + ue * X, a * math.sin(th) + a - g + up * X, up - ue)
              for ue in uemax * U for up in upmax * U]
        return list(np.max(np.abs(np.array(fs)), axis=0))
    raise AssertionError


CASES = [
    (O.DYN_DOUBLE_INTEGRATOR, (1.0,), 2),
    (O.DYN_AIR3D, (5.0, 5.0, 1.0, 1.0), 3),
    (O.DYN_AIR3D, (3.0, 4.0, 0.7, 1.3), 3),
    (O.DYN_DUBINS4D, (1.0, 0.5), 4),
    (O.DYN_ROCKETS, (1.0, 32.0, 1.0, 1.0), 3),
    (O.DYN_ROCKETS, (1.5, 9.8, 0.7, 1.2), 3),
]


@pytest.mark.parametrize("dyn,params,D", CASES)
def test_hamiltonian_is_the_control_optimum(dyn, params, D):
    rng = np.random.default_rng(11)
    m = O.method(dynamics=dyn, params=params)
    for _ in range(25):
        x = rng.uniform(-4, 4, size=D)
        p = rng.normal(size=D)
        assert O.hamiltonian(m, x, p) == pytest.approx(_brute_hg(dyn, params, x, p), abs=1e-12)


@pytest.mark.parametrize("dyn,params,D", CASES)
def test_alpha_is_the_max_speed(dyn, params, D):
    rng = np.random.default_rng(12)
    m = O.method(dynamics=dyn, params=params)
    for _ in range(25):
        x = rng.uniform(-4, 4, size=D)
        np.testing.assert_allclose(O.alpha(m, x), _brute_alpha(dyn, params, x), atol=1e-12)
        # alpha bounds every partial derivative of Hg in p (LF stability)
        p = rng.normal(size=D)
        h = 1e-6
        for d in range(D):
            e = np.zeros(D)
            e[d] = h
            slope = (O.hamiltonian(m, x, p + e) - O.hamiltonian(m, x, p - e)) / (2 * h)
            assert abs(slope) <= O.alpha(m, x)[d] + 1e-6


def test_level_set_hamiltonians():
    # -c|p| (normal motion), -c.p (advection), rotation field omega(-y, x)
    m = O.method(dynamics=O.DYN_NORM, params=(2.0,))
    assert O.hamiltonian(m, [0.3, 0.1], [3.0, 4.0]) == pytest.approx(-10.0)
    np.testing.assert_allclose(O.alpha(m, [0.3, 0.1]), [2.0, 2.0])
    assert O.hamiltonian(m, [0.0, 0.0], [0.0, 0.0]) == 0.0
    m = O.method(dynamics=O.DYN_ADVECT, params=(1.5, -2.0))
    assert O.hamiltonian(m, [9.0, 9.0], [1.0, 1.0]) == pytest.approx(0.5)
    m = O.method(dynamics=O.DYN_ROTATE, params=(2.0,))
    # F(x=1, y=0) = (0, 2): Hg = -p.F
    assert O.hamiltonian(m, [1.0, 0.0], [0.0, 1.0]) == pytest.approx(-2.0)
    np.testing.assert_allclose(O.alpha(m, [1.0, -3.0]), [6.0, 2.0])


class Line:
    def __init__(self, n, lo=0.0, hi=1.0, periodic=True):
        self.n = (n,)
        self.lo = (lo,)
        self.hi = (hi,)
        self.periodic = (0,) if periodic else ()


@pytest.mark.parametrize("c", [1.3, -0.7])
def test_lax_friedrichs_with_alpha_c_is_upwind(c):
    # Hg = -c p, alpha = |c|: Hg(pbar) + |c|(p+ - p-)/2 = -c p- (c > 0) or -c p+ (c < 0)
    g = Line(40)
    rng = np.random.default_rng(2)
    V = rng.normal(size=40)
    dx = 1.0 / 40
    m = O.method(scheme=O.ENO1, dynamics=O.DYN_ADVECT, params=(c,), brt=O.BRT_NONE)
    back = (V - np.roll(V, 1)) / dx
    fwd = (np.roll(V, -1) - V) / dx
    expect = -c * back if c > 0 else -c * fwd
    np.testing.assert_allclose(O.term(g, m, V), expect, rtol=1e-13, atol=1e-12)


def test_term_on_linear_data_equals_hamiltonian():
    # p- = p+ = grad V for linear V, so the dissipation vanishes and
    # ydot = Hg(x, grad V); with the BRT clamp, min(0, Hg)
    class G:
        n = (9, 11)
        lo = (-1.0, -1.0)
        hi = (1.0, 1.0)
        periodic = ()
    X, Y = np.meshgrid(np.linspace(-1, 1, 9), np.linspace(-1, 1, 11), indexing="ij")
    a, b = 0.7, -1.9
    V = np.asfortranarray(a * X + b * Y + 5.0)   # positive and interior-exact
    for brt in (O.BRT_NONE, O.BRT_MIN0):
        m = O.method(scheme=O.WENO5, dynamics=O.DYN_DOUBLE_INTEGRATOR, params=(1.0,), brt=brt)
        yd = O.term(G, m, V)
        expect = a * Y - abs(b)
        if brt == O.BRT_MIN0:
            expect = np.minimum(0.0, expect)
        inner = (slice(3, -3), slice(3, -3))
        np.testing.assert_allclose(yd[inner], expect[inner], atol=1e-12)


def test_brt_min0_is_the_clamped_term():
    class G:
        n = (13, 12, 10)
        lo = (-6.0, -10.0, 0.0)
        hi = (20.0, 10.0, 2 * math.pi)
        periodic = (2,)
    rng = np.random.default_rng(8)
    V = np.asfortranarray(rng.normal(size=G.n))
    free = O.term(G, O.method(dynamics=O.DYN_AIR3D, params=(5, 5, 1, 1), brt=O.BRT_NONE), V)
    clamped = O.term(G, O.method(dynamics=O.DYN_AIR3D, params=(5, 5, 1, 1), brt=O.BRT_MIN0), V)
    np.testing.assert_array_equal(clamped, np.minimum(free, 0.0))
    assert (free > 0).any() and (free < 0).any()


def test_rk3_of_linear_operator_is_taylor_polynomial():
    # Shu-Osher RK3 applied to V' = L V (L linear) equals
    # (I + dt L + dt^2 L^2 / 2 + dt^3 L^3 / 6) V exactly.
    n, c, dt = 24, 0.9, 0.013
    g = Line(n)
    dx = 1.0 / n
    L = -c * (np.eye(n) - np.roll(np.eye(n), -1, axis=1)) / dx  # first-order upwind, periodic
    rng = np.random.default_rng(4)
    V = rng.normal(size=n)
    m = O.method(scheme=O.ENO1, dynamics=O.DYN_ADVECT, params=(c,), brt=O.BRT_NONE)
    np.testing.assert_allclose(O.term(g, m, V), L @ V, rtol=1e-12, atol=1e-12)
    A = dt * L
    taylor = V + A @ V + A @ (A @ V) / 2 + A @ (A @ (A @ V)) / 6
    np.testing.assert_allclose(O.rk3_step(g, m, V, dt), taylor, rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("order", [1, 2, 3])
def test_rk_orders_of_linear_operator_are_taylor_polynomials(order):
    # forward Euler, the two-stage and the three-stage Shu-Osher schemes applied
    # to V' = L V (L linear) equal the Taylor polynomial of exp(dt L) of their order
    n, c, dt = 24, 0.9, 0.013
    g = Line(n)
    dx = 1.0 / n
    L = -c * (np.eye(n) - np.roll(np.eye(n), -1, axis=1)) / dx
    rng = np.random.default_rng(5)
    V = rng.normal(size=n)
    m = O.method(scheme=O.ENO1, dynamics=O.DYN_ADVECT, params=(c,), brt=O.BRT_NONE, order=order)
    A = dt * L
    terms, T = [V], V
    for k in range(1, order + 1):
        T = A @ T / k
        terms.append(T)
    np.testing.assert_allclose(O.rk_step(g, m, V, dt), sum(terms), rtol=1e-12, atol=1e-12)
    # and they differ from each other at the next order
    if order < 3:
        higher = O.rk_step(g, O.method(scheme=O.ENO1, dynamics=O.DYN_ADVECT, params=(c,), brt=O.BRT_NONE,
                                       order=order + 1), V, dt)
        assert np.max(np.abs(higher - sum(terms))) > 1e-8


def test_global_lax_friedrichs_uses_the_grid_maximum():
    # double integrator on [-1, 1]^2: alpha = (|x1|, umax), so the global
    # alpha is (1, umax) (|x1| = 1 on the edge rows); on the rows x1 = +-1
    # local and global terms coincide, elsewhere the global one adds
    # (1 - |x1|) (p+_0 - p-_0) / 2
    g = W.GridSpec((21, 17), (-1.0, -1.0), (1.0, 1.0))
    rng = np.random.default_rng(6)
    V = np.asfortranarray(rng.normal(size=g.n))
    loc = O.method(dynamics=O.DYN_DOUBLE_INTEGRATOR, params=(0.7,), brt=O.BRT_NONE)
    glo = O.method(dynamics=O.DYN_DOUBLE_INTEGRATOR, params=(0.7,), brt=O.BRT_NONE, alpha_global=True)
    np.testing.assert_array_equal(O.alpha_max(g, loc), [1.0, 0.7])
    yl, yg = O.term(g, loc, V), O.term(g, glo, V)
    np.testing.assert_array_equal(yl[:, 0], yg[:, 0])
    np.testing.assert_array_equal(yl[:, -1], yg[:, -1])
    pm, pp = O.upwind(g, loc, V, 0)
    x1 = np.linspace(-1.0, 1.0, 17)[None, :]
    np.testing.assert_allclose(yg - yl, (1.0 - np.abs(x1)) * (pp - pm) / 2, rtol=0, atol=1e-12)
    # CFL bound of the global scheme: sum_d max alpha_d / dx_d = 1/0.1 + 0.7/0.125
    assert O.step_bound_inv(g, glo) == pytest.approx(1.0 / 0.1 + 0.7 / 0.125, rel=1e-15)
    # air3D (va = vb = 5, |a|, |b| <= 1) on a grid holding psi = pi and |y| = 10:
    # max alpha = (|-5 + 5 cos psi| + 10, 5 |sin psi| + 20, 2) = (20, 25, 2)
    ga = W.GridSpec((27, 21, 8), (-6.0, -10.0, 0.0), (20.0, 10.0, 2 * np.pi), (2,))
    ma = O.method(dynamics=O.DYN_AIR3D, params=(5.0, 5.0, 1.0, 1.0), alpha_global=True)
    np.testing.assert_allclose(O.alpha_max(ga, ma), [20.0, 25.0, 2.0], rtol=1e-15)


def test_brt_minv_keeps_the_pointwise_minimum():
    g = Line(30)
    rng = np.random.default_rng(6)
    V = rng.normal(size=30)
    free = O.rk3_step(g, O.method(scheme=O.WENO5, dynamics=O.DYN_ADVECT, params=(0.5,), brt=O.BRT_NONE), V, 0.01)
    minv = O.rk3_step(g, O.method(scheme=O.WENO5, dynamics=O.DYN_ADVECT, params=(0.5,), brt=O.BRT_MINV), V, 0.01)
    np.testing.assert_array_equal(minv, np.minimum(free, V))


def test_step_bound_closed_forms():
    class DI:
        n = (101, 101)
        lo = (-1.0, -1.0)
        hi = (1.0, 1.0)
        periodic = ()
    # max_x |x1|/dx0 + umax/dx1 = 1/0.02 + 1/0.02
    sbi = O.step_bound_inv(DI, O.method(dynamics=O.DYN_DOUBLE_INTEGRATOR, params=(1.0,)))
    assert sbi == pytest.approx(100.0, rel=1e-14)
    g = Line(50)
    sbi = O.step_bound_inv(g, O.method(dynamics=O.DYN_ADVECT, params=(-2.0,)))
    assert sbi == pytest.approx(2.0 * 50, rel=1e-14)


def test_time_loop_lands_on_slices():
    # advection with |c| = 2 on 50 periodic cells: stepBoundInv = 100, so
    # dt = 0.8/100 = 0.008 and a slice of length T takes ceil(T/0.008) steps
    g = Line(50)
    m = O.method(scheme=O.WENO5, dynamics=O.DYN_ADVECT, params=(2.0,), brt=O.BRT_NONE, cfl=0.8)
    V0 = np.sin(2 * np.pi * np.arange(50) / 50)
    ts = [0.0, 0.02, 0.05, 0.05, 0.1]
    slices, steps, reached = O.solve(g, m, V0, ts)
    np.testing.assert_array_equal(slices[0], V0)          # tau = 0: no step
    np.testing.assert_array_equal(slices[2], slices[3])   # repeated slice time: no step
    # 0 -> 0.02: 3 steps (0.008, 0.008, 0.004); 0.02 -> 0.05: 4 steps; 0.05 -> 0.1: 7 steps
    assert steps == 3 + 4 + 7
    np.testing.assert_allclose(reached, ts, rtol=0, atol=1e-15)
    # max_step caps dt
    _, steps2, _ = O.solve(g, O.method(scheme=O.WENO5, dynamics=O.DYN_ADVECT, params=(2.0,),
                                       brt=O.BRT_NONE, max_step=0.005), V0, [0.1])
    assert steps2 == 20


def test_solve_equals_repeated_steps():
    g = Line(32)
    m = O.method(scheme=O.WENO5, dynamics=O.DYN_ADVECT, params=(1.0,), brt=O.BRT_MIN0)
    V0 = np.cos(2 * np.pi * np.arange(32) / 32)
    slices, steps, _ = O.solve(g, m, V0, [0.1])
    V = V0.copy()
    dt_full = 0.8 / 32.0
    t = 0.0
    for k in range(steps):
        dt = min(0.1 - t, dt_full)
        V = O.rk3_step(g, m, V, dt)
        t += dt
    np.testing.assert_array_equal(slices[0], V)


def test_invalid_arguments_are_rejected():
    g = Line(10)
    m = O.method(dynamics=O.DYN_AIR3D, params=(5, 5, 1, 1))
    with pytest.raises(ValueError):
        O.term(g, m, np.zeros(10))          # air3D needs 3 dims
    with pytest.raises(ValueError):
        O.solve(g, O.method(dynamics=O.DYN_ADVECT, params=(1.0,)), np.zeros(10), [0.2, 0.1])
    with pytest.raises(ValueError):
        O.upwind_line(np.zeros(10), 0.1, scheme=4)


# ---------------------------------------------------------------------------
# Lax-Friedrichs dissipation local in p (R12): alpha_d = max of |dHg/dp_d|
# over the box of gradients spanned by a node's p- and p+.
# ---------------------------------------------------------------------------

def _game_dynamics(dyn, params, x):
    """f(x, a, b) on the control grid for the two-player games (a maximises,
    b minimises), shape (41, 41, 3)."""
    if dyn == O.DYN_AIR3D:
        va, vb, amax, bmax = params
        X, Y, psi = x
        A, B = np.meshgrid(amax * U, bmax * U, indexing="ij")
        return np.stack([-va + vb * math.cos(psi) + A * Y, vb * math.sin(psi) - A * X, B - A], axis=-1)
    a, g, uemax, upmax = params
    X, Z, th = x
    UE, UP = np.meshgrid(uemax * U, upmax * U, indexing="ij")
    return np.stack([a * math.cos(th) + UE * X, a * math.sin(th) + a - g + UP * X, UP - UE], axis=-1)


def _generalized_slopes(F, p, tol=1e-9):
    """max over the optimal control pairs at p of |f_d|: the extreme points of
    the generalized gradient of Hg(p) = max_a min_b p . f(a, b) (envelope
    theorem; tied optima give every one-sided slope)."""
    P = F @ p
    inner = P.min(axis=1)
    val = inner.max()
    best = np.zeros(F.shape[-1])
    for i in np.nonzero(inner >= val - tol)[0]:
        for j in np.nonzero(P[i] <= inner[i] + tol)[0]:
            best = np.maximum(best, np.abs(F[i, j]))
    return best


def _box_vertices(lo, hi, planes):
    """Vertices of the arrangement of the box faces and the switching planes
    n . p = 0 inside the box: every cell of constant optimal controls that
    meets the box has one of them in its closure."""
    import itertools
    D = len(lo)
    rows = []
    for d in range(D):
        e = np.zeros(D)
        e[d] = 1.0
        rows += [(e, lo[d]), (e, hi[d])]
    rows += [(np.asarray(n, dtype=float), 0.0) for n in planes]
    out = []
    for combo in itertools.combinations(rows, D):
        M = np.array([r[0] for r in combo])
        if abs(np.linalg.det(M)) < 1e-12:
            continue
        p = np.linalg.solve(M, np.array([r[1] for r in combo]))
        if np.all(p >= np.asarray(lo) - 1e-12) and np.all(p <= np.asarray(hi) + 1e-12):
            out.append(np.clip(p, lo, hi))
    return out


def _switching_planes(dyn, params, x):
    # p . f is affine in each control; it switches where the control's
    # coefficient p . (f(u = 1) - f(u = 0)) vanishes
    F = _game_dynamics(dyn, (params[0], params[1], 1.0, 1.0), x)
    i0, i1 = len(U) // 2, len(U) - 1   # U[20] = 0, U[40] = 1
    return [F[i1, i0] - F[i0, i0], F[i0, i1] - F[i0, i0]]


def _random_box(rng, D, scale):
    kind = rng.integers(0, 4)
    c = rng.normal(size=D) * scale
    w = np.abs(rng.normal(size=D)) * scale * (0.05 if kind == 0 else 0.6)
    if kind == 3:
        w[rng.integers(0, D)] = 0.0      # flat along one dimension
    return c - w, c + w


@pytest.mark.parametrize("dyn,params", [(O.DYN_AIR3D, (5.0, 5.0, 1.0, 1.0)), (O.DYN_AIR3D, (3.0, 4.0, 0.7, 1.3)),
                                        (O.DYN_ROCKETS, (1.0, 32.0, 1.0, 1.0)), (O.DYN_ROCKETS, (1.5, 9.8, 0.7, 1.2))])
def test_box_alpha_of_the_games_is_the_largest_slope_over_the_box(dyn, params):
    rng = np.random.default_rng(31)
    m = O.method(dynamics=dyn, params=params)
    for trial in range(40):
        x = np.array([rng.uniform(-6, 6), rng.uniform(-6, 6), rng.uniform(-3, 3)])
        lo, hi = _random_box(rng, 3, 1.0)
        F = _game_dynamics(dyn, params, x)
        brute = np.zeros(3)
        for p in _box_vertices(lo, hi, _switching_planes(dyn, params, x)):
            brute = np.maximum(brute, _generalized_slopes(F, p))
        got = O.alpha_box(m, x, lo, hi)
        np.testing.assert_allclose(got, brute, rtol=0, atol=1e-9, err_msg=str((trial, x, lo, hi)))
        # never above the maximum over every p (the CFL bound stays valid)
        assert np.all(got <= O.alpha(m, x) + 1e-12)
    # a box holding a neighbourhood of p = 0 meets every switching pattern
    x = np.array([1.3, -2.2, 0.7])
    np.testing.assert_allclose(O.alpha_box(m, x, -np.ones(3), np.ones(3)), O.alpha(m, x), rtol=0, atol=1e-12)


@pytest.mark.parametrize("D", [2, 3])
def test_box_alpha_of_the_norm_is_the_largest_slope_over_the_box(D):
    # Hg = -c |p|: dHg/dp = -c p / |p| (the ball of radius c at p = 0); over a
    # box the largest |p_d| / |p| sits at the largest |p_d| and the smallest
    # |p_j| the box holds, which are box ends or 0: all on the sample grid
    import itertools
    c = 1.7
    m = O.method(dynamics=O.DYN_NORM, params=(c,))
    rng = np.random.default_rng(32)
    for trial in range(40):
        lo, hi = _random_box(rng, D, 1.0)
        axes = [sorted(set(list(np.linspace(l, h, 5)) + ([0.0] if l < 0.0 < h else []))) for l, h in zip(lo, hi)]
        brute = np.zeros(D)
        for p in itertools.product(*axes):
            p = np.array(p)
            r = np.sqrt(np.sum(p * p))
            brute = np.maximum(brute, c * np.abs(p) / r if r > 0 else np.full(D, c))
        got = O.alpha_box(m, np.zeros(D), lo, hi)
        np.testing.assert_allclose(got, brute, rtol=1e-13, atol=1e-15, err_msg=str((trial, lo, hi)))
    # a box that is one point p: the slope of -c|p| there
    p = np.array([0.3, -0.4, 1.2])[:D]
    np.testing.assert_allclose(O.alpha_box(m, np.zeros(D), p, p), c * np.abs(p) / np.linalg.norm(p), rtol=1e-15)
    # the point p = 0: the generalized gradient is the ball of radius c
    np.testing.assert_array_equal(O.alpha_box(m, np.zeros(D), np.zeros(D), np.zeros(D)), np.full(D, c))


@pytest.mark.parametrize("dyn,params,D", [(O.DYN_DOUBLE_INTEGRATOR, (1.0,), 2), (O.DYN_DUBINS4D, (1.0, 0.5), 4),
                                          (O.DYN_ADVECT, (0.7, -1.3, 0.4), 3), (O.DYN_ROTATE, (1.3,), 2)])
def test_box_alpha_equals_the_node_alpha_where_slopes_do_not_depend_on_p(dyn, params, D):
    # |dHg/dp_d| is the same on both sides of every |p_d| kink of these
    # Hamiltonians, so the box maximum is the maximum over every p; checked
    # against slopes of the brute-force control optimum at box corners
    import itertools
    rng = np.random.default_rng(33)
    m = O.method(dynamics=dyn, params=params)
    for _ in range(10):
        x = rng.uniform(-3, 3, size=D)
        lo, hi = _random_box(rng, D, 1.0)
        got = O.alpha_box(m, x, lo, hi)
        np.testing.assert_array_equal(got, O.alpha(m, x))
        if dyn in (O.DYN_DOUBLE_INTEGRATOR, O.DYN_DUBINS4D):
            h = 1e-7
            for corner in itertools.product(*zip(lo, hi)):
                p = np.array(corner) + 0.01   # off the kinks
                for d in range(D):
                    e = np.zeros(D)
                    e[d] = h
                    slope = (_brute_hg(dyn, params, x, p + e) - _brute_hg(dyn, params, x, p - e)) / (2 * h)
                    assert abs(slope) <= got[d] + 1e-6


def test_box_lax_friedrichs_term():
    # 1-D norm: |dHg/dp| = c on both sides of 0, so the box term is the node term
    g = Line(40)
    rng = np.random.default_rng(34)
    V = rng.normal(size=40)
    node = O.method(scheme=O.WENO5, dynamics=O.DYN_NORM, params=(1.2,), brt=O.BRT_NONE)
    box = O.method(scheme=O.WENO5, dynamics=O.DYN_NORM, params=(1.2,), brt=O.BRT_NONE, alpha_box=True)
    np.testing.assert_array_equal(O.term(g, box, V), O.term(g, node, V))
    # 2-D norm: at each node the term takes the box maximum of the node's own p-, p+
    g2 = W.GridSpec((17, 13), (-1.0, -1.0), (1.0, 1.0))
    V2 = np.asfortranarray(rng.normal(size=g2.n))
    node2 = O.method(scheme=O.ENO2, dynamics=O.DYN_NORM, params=(1.2,), brt=O.BRT_NONE)
    box2 = O.method(scheme=O.ENO2, dynamics=O.DYN_NORM, params=(1.2,), brt=O.BRT_NONE, alpha_box=True)
    pm = [O.upwind(g2, node2, V2, d)[0] for d in range(2)]
    pp = [O.upwind(g2, node2, V2, d)[1] for d in range(2)]
    yb, yn = O.term(g2, box2, V2), O.term(g2, node2, V2)
    for idx in [(0, 0), (5, 7), (16, 12), (9, 3)]:
        lo = [min(pm[d][idx], pp[d][idx]) for d in range(2)]
        hi = [max(pm[d][idx], pp[d][idx]) for d in range(2)]
        a = O.alpha_box(box2, [0.0, 0.0], lo, hi)
        half = [(pp[d][idx] - pm[d][idx]) / 2 for d in range(2)]
        assert yb[idx] - yn[idx] == pytest.approx(sum((a[d] - 1.2) * half[d] for d in range(2)), abs=1e-12)


def test_contracted_build_is_the_same_scheme():
    # the oracle compiled with contraction (the parity tests' measure of its
    # own rounding sensitivity) solves a well-conditioned problem alike
    spec, V0 = W.double_integrator(31)
    m = O.method(scheme=O.WENO5, dynamics=O.DYN_DOUBLE_INTEGRATOR, params=(1.0,), brt=O.BRT_MIN0)
    a, steps_a, ta = O.solve(spec, m, V0, [0.25, 0.5])
    b, steps_b, tb = O.solve(spec, m, V0, [0.25, 0.5], fma=True)
    assert steps_a == steps_b
    np.testing.assert_array_equal(ta, tb)
    assert np.max(np.abs(a - b)) <= 1e-13 * np.max(np.abs(a))
