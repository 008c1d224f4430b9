"""One grid stepped slab by slab on one GPU (the layout of a multi-GPU solve
of one large grid): three halo planes per side refreshed by device copies
before every RK stage, dt from the maximum of the slabs' CFL bounds. The
step must equal the whole-grid step."""
import math

import numpy as np
import pytest

from paper_2507_11542_gb300 import workloads as W

from helpers import AIR3D, DUBINS, lib_method, rel_err, to_dev, to_host

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    import torch
    from paper_2507_11542_gb300 import build, solver
    build.build()
    assert torch.cuda.is_available()
    c = solver.Context(0)
    yield c
    c.close()


CASES = {
    # split along psi (periodic): halos wrap around
    "air3d": (W.GridSpec((37, 29, 23), (-6.0, -10.0, 0.0), (20.0, 10.0, 2.0 * math.pi), (2,)), AIR3D, [2, 3]),
    # split along v (not periodic): the end slabs keep the grid's own edge
    "dubins": (W.GridSpec((13, 11, 9, 12), (-5.0, -5.0, 0.0, 0.0), (5.0, 5.0, 2.0 * math.pi, 2.0), (2,)), DUBINS,
               [2, 4]),
}


@pytest.mark.parametrize("which", ["air3d", "dubins"])
@pytest.mark.parametrize("dtype,tol", [("float64", 1e-14), ("float32", 1e-6)])
def test_slab_step_equals_whole_grid_step(ctx, which, dtype, tol):
    from paper_2507_11542_gb300 import slabs, solver
    spec, dyn, counts = CASES[which]
    V0 = W.sphere(spec, (0.5, -0.3), 2.0, dims=(0, 1)) + 0.3 * W.random_field(spec, 5)
    m = lib_method(dynamics=dyn, brt=1)
    whole_bound = solver.step_bound(ctx, spec, m)
    dt = 0.8 / whole_bound
    want = to_dev(V0, dtype)
    solver.rk3_step(ctx, spec, m, want, dt)
    for n_slabs in counts:
        assert slabs.step_bound_slabs(ctx, spec, m, n_slabs) == pytest.approx(whole_bound, rel=1e-14)
        got = to_dev(V0, dtype)
        slabs.rk3_step_slabs(ctx, spec, m, got, dt, n_slabs)
        assert rel_err(to_host(got, spec.n), to_host(want, spec.n)) <= tol, n_slabs
