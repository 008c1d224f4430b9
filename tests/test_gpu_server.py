"""The continuous-batching server (hj_server_*): every result equals the same
problem solved alone, admission respects the HBM budget while requests
overlap on the device, and cancellation, timeouts, refusals and shutdown
behave as documented. Failures are made on the host (cancelled tickets,
malformed requests, a stopped server); nothing faults the GPU."""
import math
import threading
import time

import numpy as np
import pytest

from paper_2507_11542_gb300 import workloads as W

from helpers import AIR3D, DI, DUBINS, lib_method, rel_err, to_dev, to_host

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


def _requests(seed, count, dtype):
    rng = np.random.default_rng(seed)
    reqs = []
    for k in range(count):
        kind = k % 3
        if kind == 0:
            g, V0 = W.double_integrator(int(rng.integers(31, 71)), float(rng.uniform(0.3, 0.6)))
            m, ts = lib_method(dynamics=DI), [0.0, float(rng.uniform(0.2, 0.6))]
        elif kind == 1:
            g, V0 = W.air3d(int(rng.integers(21, 35)), float(rng.uniform(3.0, 6.0)))
            m, ts = lib_method(dynamics=AIR3D), [float(rng.uniform(0.2, 0.8))]
        else:
            g, V0 = W.dubins4d(int(rng.integers(11, 17)), seed=k)
            m, ts = lib_method(dynamics=DUBINS), [0.2, float(rng.uniform(0.4, 0.9))]
        reqs.append((g, m, to_dev(V0, dtype), ts))
    return reqs


@pytest.mark.parametrize("dtype,tol", [("float64", 1e-13), ("float32", 2e-6)])
def test_served_results_equal_solo_solves(ctx, dtype, tol):
    from paper_2507_11542_gb300 import _lib as L, solver
    reqs = _requests(7, 9, dtype)
    with solver.Server(ctx, hbm_budget=512 << 20, max_slots=8) as srv:
        tickets = []
        for k, (g, m, v0, ts) in enumerate(reqs):
            tickets.append(srv.submit(g, m, v0, ts))
            if k % 3 == 2:
                time.sleep(0.01)  # later requests arrive while earlier ones run
        results = [srv.wait(t, 60000) for t in tickets]
        counters = srv.counters()
    assert counters["status"] == L.HJ_OK and counters["completed"] == len(reqs)
    for (g, m, v0, ts), (st, out, times, stats) in zip(reqs, results):
        assert st == L.HJ_OK
        alone, t_alone, st_alone = solver.solve(ctx, g, m, v0, ts)
        assert stats["steps"] == st_alone["steps"]
        np.testing.assert_array_equal(times, t_alone)
        for s in range(len(ts)):
            assert rel_err(to_host(out[s], g.n), to_host(alone[s], g.n)) <= tol
        assert stats["elapsed_ms"] > 0


def test_rate_lanes_let_small_requests_finish_first(ctx):
    # Rate lanes: instances above 16M nodes step once per server step, then
    # twice (above 8M), four times (above 4M), eight times (smaller): a
    # request that needs fewer server steps retires first, and every result
    # still equals the problem solved alone.
    from paper_2507_11542_gb300 import _lib as L, solver
    reqs = []
    g, V0 = W.air3d(161, 5.0)  # 4.17M nodes: four steps per server step, 140 steps
    reqs.append((g, lib_method(dynamics=AIR3D), to_dev(V0, "float32"), [0.1, 0.3]))
    g, V0 = W.air3d(101, 4.0)  # 1.03M nodes: eight steps per server step, 84 steps
    reqs.append((g, lib_method(dynamics=AIR3D), to_dev(V0, "float32"), [0.3]))
    g, V0 = W.double_integrator(81, 0.5)  # 6561 nodes: eight steps per server step, 50 steps
    reqs.append((g, lib_method(dynamics=DI), to_dev(V0, "float32"), [0.25, 0.5]))
    with solver.Server(ctx, hbm_budget=1 << 30, max_slots=4) as srv:
        tickets = [srv.submit(g, m, v0, ts) for g, m, v0, ts in reqs]
        results = [srv.wait(t, 120000) for t in tickets]
    lat = []
    for (g, m, v0, ts), (st, out, times, stats) in zip(reqs, results):
        assert st == L.HJ_OK
        alone, t_alone, st_alone = solver.solve(ctx, g, m, v0, ts)
        assert stats["steps"] == st_alone["steps"]
        np.testing.assert_array_equal(times, t_alone)
        for s in range(len(ts)):
            assert rel_err(to_host(out[s], g.n), to_host(alone[s], g.n)) <= 2e-6
        lat.append(stats["elapsed_ms"])
    assert lat[2] < lat[1] < lat[0], lat


def test_admission_keeps_within_the_budget(ctx):
    # each 2-D request needs three grids of 81x81 doubles plus bookkeeping
    # (about 160 KiB); a 400 KiB budget admits two at a time
    from paper_2507_11542_gb300 import _lib as L, solver
    g, V0 = W.double_integrator(81, 0.5)
    m = lib_method(dynamics=DI)
    budget = 400 << 10
    with solver.Server(ctx, hbm_budget=budget, max_slots=8) as srv:
        tickets = [srv.submit(g, m, to_dev(V0), [0.5]) for _ in range(6)]
        peak_running, peak_bytes = 0, 0
        pending = set(tickets)
        while pending:
            c = srv.counters()
            peak_running = max(peak_running, c["running"])
            peak_bytes = max(peak_bytes, c["bytes_in_use"])
            for t in list(pending):
                st, out, times, stats = srv.wait(t, 1)
                if st != L.HJ_ETIMEOUT:
                    assert st == L.HJ_OK
                    pending.discard(t)
    assert peak_bytes <= budget
    assert 1 <= peak_running <= 2


def test_cancel_timeout_and_refusals(ctx):
    from paper_2507_11542_gb300 import _lib as L, solver
    g, V0 = W.air3d(41, 5.0)
    with solver.Server(ctx, hbm_budget=64 << 20, max_slots=1) as srv:
        long_t = srv.submit(g, lib_method(dynamics=AIR3D), to_dev(V0), [2.8])
        queued_t = srv.submit(g, lib_method(dynamics=AIR3D), to_dev(V0), [2.8])
        st, _, _, _ = srv.wait(long_t, 0)
        assert st == L.HJ_ETIMEOUT                      # still running; the ticket stays valid
        assert srv.cancel(queued_t) == L.HJ_OK         # waiting for the single slot: cancelled at once
        st, _, _, _ = srv.wait(queued_t, 1000)
        assert st == L.HJ_ECANCELLED
        assert srv.cancel(long_t) == L.HJ_OK           # on the device: cancelled at the next tick
        st, _, _, _ = srv.wait(long_t, 30000)
        assert st == L.HJ_ECANCELLED
        assert srv.cancel(long_t) == L.HJ_EINVAL       # forgotten after wait
        # a second-order-in-time problem is not served by the batched kernel; a grid beyond the budget cannot fit
        with pytest.raises(L.HJError) as e:
            srv.submit(g, lib_method(scheme=2, dynamics=AIR3D, order=2), to_dev(V0), [0.1])
        assert e.value.status == L.HJ_EINVAL
        gb, Vb = W.air3d(161, 5.0)
        with pytest.raises(L.HJError) as e:
            srv.submit(gb, lib_method(dynamics=AIR3D), to_dev(Vb), [0.1])
        assert e.value.status == L.HJ_ENOMEM
        # a NaN in v0 fails that request only
        bad = W.double_integrator(31)[1]
        bad[4, 4] = np.nan
        gd = W.double_integrator(31)[0]
        t_bad = srv.submit(gd, lib_method(dynamics=DI), to_dev(bad), [0.1])
        st, _, _, _ = srv.wait(t_bad, 30000)
        assert st == L.HJ_ENONFINITE
        t_ok = srv.submit(gd, lib_method(dynamics=DI), to_dev(W.double_integrator(31)[1]), [0.1])
        st, _, _, _ = srv.wait(t_ok, 30000)
        assert st == L.HJ_OK


def test_shutdown_with_requests_in_flight(ctx):
    from paper_2507_11542_gb300 import solver
    g, V0 = W.air3d(51, 5.0)
    srv = solver.Server(ctx, hbm_budget=128 << 20, max_slots=2)
    for _ in range(4):
        srv.submit(g, lib_method(dynamics=AIR3D), to_dev(V0), [2.8])
    time.sleep(0.05)
    t0 = time.time()
    srv.close()                       # running requests are cancelled between ticks
    assert time.time() - t0 < 30
    # the context is still usable
    out, _, stats = solver.solve(ctx, g, lib_method(dynamics=AIR3D), to_dev(V0), [0.05])
    assert stats["steps"] > 0
