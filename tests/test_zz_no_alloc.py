"""The no-allocation RK3 step (hj_rk3_step_static).

It serves callers that may not allocate device memory while running -- a
real-time loop that forbids allocation after start-up, or a host that owns
the GPU memory pool -- by keeping its stage buffers in a fixed device array.
This file is collected last so that a run stopping at the first failure has
already run every other test; it also passes on its own in a fresh process.
"""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_2507_11542_gb300 import workloads as W

from helpers import AIR3D, DI, DUBINS, lib_method, oracle_method, rel_err, to_dev, to_host

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


AIR_SPEC = W.GridSpec((41, 37, 33), (-6.0, -10.0, 0.0), (20.0, 10.0, 2 * math.pi), (2,))
CASES = [
    # (dynamics, grid, dtype, kernel): kernel 2 is the one-node-per-thread kernel
    (AIR3D, AIR_SPEC, "float64", 0),
    (AIR3D, AIR_SPEC, "float32", 0),
    (DI, W.GridSpec((61, 47), (-1.0, -1.0), (1.0, 1.0)), "float64", 0),
    (DUBINS, W.GridSpec((15, 13, 11, 9), (-5.0, -5.0, 0.0, 0.0), (5.0, 5.0, 2 * math.pi, 2.0), (2,)), "float64", 0),
    # grids the row kernel cannot take, so both entry points use the other kernel:
    # a dimension of 3 nodes, and FP64 rows of 600 nodes (wider than a 512-thread block)
    (DI, W.GridSpec((45, 3), (-1.0, -1.0), (1.0, 1.0)), "float64", 0),
    (DI, W.GridSpec((600, 9), (-1.0, -1.0), (1.0, 1.0)), "float64", 0),
    (AIR3D, AIR_SPEC, "float64", 2),
]


@pytest.mark.parametrize("dyn,spec,dtype,kernel", CASES)
def test_static_step_matches_rk3_step_twice(ctx, dyn, spec, dtype, kernel):
    # Same arithmetic, the same angle tables and the same kernel kind as
    # hj_rk3_step, whose results do not depend on the launch shape: the two
    # entry points agree bit for bit, on two calls in a row (the shared
    # scratch is reused), and both stay within the parity bar of the oracle.
    import torch
    from paper_2507_11542_gb300 import _lib as L, solver
    V0 = W.sphere(spec, (0.3,) * 2, 1.0, dims=(0, 1)) + 0.1 * W.random_field(spec, 3)
    m = lib_method(dynamics=dyn, brt=1, kernel=kernel)
    dt = 0.8 / solver.step_bound(ctx, spec, m)
    a = to_dev(V0, dtype)   # stepped by the existing entry point
    b = to_dev(V0, dtype)   # stepped by the no-allocation entry point
    grid = L.make_grid(spec)
    stream = ctx.stream.cuda_stream
    ref = V0.astype(np.float32).astype(np.float64) if dtype == "float32" else V0
    for _ in range(2):
        solver.rk3_step(ctx, spec, m, a, dt)
        st = L.hj_rk3_step_static(stream, 0, grid, m, L.dtype_code(b.dtype), b, dt)
        assert st == L.HJ_OK
        torch.cuda.synchronize()
        np.testing.assert_array_equal(to_host(b, spec.n), to_host(a, spec.n))
        ref = O.rk3_step(spec, oracle_method(dynamics=dyn, brt=1), ref, dt)
    # FP64 within 1e-12 of the oracle; FP32 within its rounding (two steps of O(1) data)
    assert rel_err(to_host(b, spec.n), ref) <= (1e-12 if dtype == "float64" else 2e-6)


def test_static_step_rejects_what_does_not_fit(ctx):
    from paper_2507_11542_gb300 import _lib as L
    import torch
    m = lib_method(dynamics=DI, brt=1)
    big = W.GridSpec((1025, 1025), (-1.0, -1.0), (1.0, 1.0))   # more than HJ_STATIC_MAX_NODES nodes
    v = torch.zeros(8, dtype=torch.float64, device="cuda")      # never touched: the call is rejected first
    assert L.hj_rk3_step_static(ctx.stream.cuda_stream, 0, L.make_grid(big), m, L.HJ_F64, v, 0.01) == L.HJ_EINVAL
    # a product of node counts that overflows 64 bits (4 * (2^62 + 8) wraps to 32) is rejected too
    huge = L.make_grid(W.GridSpec((4, 2), (-1.0, -1.0), (1.0, 1.0)))
    huge.n[1] = (1 << 62) + 8
    assert L.hj_rk3_step_static(ctx.stream.cuda_stream, 0, huge, m, L.HJ_F64, v, 0.01) == L.HJ_EINVAL
    # the launch shape is the entry point's own: a tile override is refused
    assert L.hj_rk3_step_static(ctx.stream.cuda_stream, 0, L.make_grid(W.GridSpec((64, 64), (-1.0, -1.0),
                                (1.0, 1.0))), lib_method(dynamics=DI, brt=1, tile=(2, 1, 1, 0)), L.HJ_F64, v, 0.01) \
        == L.HJ_EINVAL
    ok = W.GridSpec((64, 64), (-1.0, -1.0), (1.0, 1.0))
    assert L.hj_rk3_step_static(ctx.stream.cuda_stream, 0, L.make_grid(ok), m, L.HJ_F64, v, -1.0) == L.HJ_EINVAL
    assert L.hj_rk3_step_static(ctx.stream.cuda_stream, 0, L.make_grid(ok), m, 7, v, 0.01) == L.HJ_EINVAL
    # only the three-stage scheme with per-node dissipation
    for other in (lib_method(dynamics=DI, brt=1, order=2), lib_method(dynamics=DI, brt=1, alpha_global=True)):
        assert L.hj_rk3_step_static(ctx.stream.cuda_stream, 0, L.make_grid(ok), other, L.HJ_F64, v, 0.01) == \
            L.HJ_EINVAL


@pytest.mark.parametrize("scheme", [1, 2, 3])
def test_static_step_runs_every_scheme(ctx, scheme):
    # the ENO schemes also run on the row kernel inside the no-allocation step
    import torch
    from paper_2507_11542_gb300 import _lib as L, solver
    dyn, spec = AIR3D, AIR_SPEC
    V0 = W.sphere(spec, (0.3,) * 2, 1.0, dims=(0, 1)) + 0.1 * W.random_field(spec, 4)
    m = lib_method(scheme=scheme, dynamics=dyn, brt=1)
    dt = 0.8 / solver.step_bound(ctx, spec, m)
    b = to_dev(V0, "float64")
    st = L.hj_rk3_step_static(ctx.stream.cuda_stream, 0, L.make_grid(spec), m, L.HJ_F64, b, dt)
    assert st == L.HJ_OK
    torch.cuda.synchronize()
    ref = O.rk3_step(spec, oracle_method(scheme=scheme, dynamics=dyn, brt=1), V0, dt)
    assert rel_err(to_host(b, spec.n), ref) <= 1e-12
