"""The slab decomposition of one grid along its slowest dimension (the layout
of a one-grid solve spread over several GPUs), tested on the host:
- the plan partitions the planes, wraps halos along a periodic dimension and
  stops them at a non-periodic edge;
- each slab is a grid whose nodes sit exactly where the whole grid's do;
- two gloo ranks, each owning one slab, exchange three halo planes before
  every RK stage and all-reduce the CFL bound (the oracle computes each
  slab's stage terms). Their step equals the oracle's step on the whole grid.
"""
import math
import os
import socket
import sys

import numpy as np
import pytest

from oracle import oracle as O
from paper_2507_11542_gb300 import slabs as SL
from paper_2507_11542_gb300 import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _air(n=(21, 17, 16)):
    return W.GridSpec(n, (-6.0, -10.0, 0.0), (20.0, 10.0, 2.0 * math.pi), (2,))


@pytest.mark.parametrize("n_slabs", [1, 2, 3, 5])
@pytest.mark.parametrize("periodic", [True, False])
def test_plan_partitions_planes_and_places_halos(n_slabs, periodic):
    g = _air() if periodic else W.GridSpec((9, 7, 17), (0.0, 0.0, -1.0), (1.0, 1.0, 1.0))
    n = g.n[-1]
    plan = SL.plan(g, n_slabs)
    owned = [z for s in plan for z in range(s.z0, s.z1)]
    assert owned == list(range(n))
    for s in plan:
        assert s.spec.n[-1] == len(s.planes) == s.below + (s.z1 - s.z0) + s.above
        assert list(s.planes[s.owned]) == list(range(s.z0, s.z1))
        if n_slabs > 1:
            assert s.below == (3 if periodic or s.z0 > 0 else 0)
            assert s.above == (3 if periodic or s.z1 < n else 0)
            assert 2 not in s.spec.periodic
        # the slab's nodes are the whole grid's nodes (coordinates to rounding)
        full_axis = g.axis(2)
        dz = full_axis[1] - full_axis[0]
        want = g.lo[2] + (np.arange(s.z0 - s.below, s.z1 + s.above)) * dz
        np.testing.assert_allclose(s.spec.axis(2), want, rtol=0, atol=1e-12)
    for s, src in zip(plan, SL.halo_sources(plan)):
        assert len(src) == s.below + s.above
        for local, k, k_local in src:
            assert plan[k].planes[k_local] == s.planes[local]
            assert plan[k].below <= k_local < plan[k].below + plan[k].z1 - plan[k].z0


def test_plan_rejects_slabs_thinner_than_the_halo():
    with pytest.raises(ValueError):
        SL.plan(W.GridSpec((5, 5, 8), (0.0,) * 3, (1.0,) * 3), 3)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _slab_worker(rank, world, port, q):
    sys.path.insert(0, ROOT)
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port), "RANK": str(rank),
                       "WORLD_SIZE": str(world)})
    import torch
    import torch.distributed as dist
    from oracle import oracle as O
    from paper_2507_11542_gb300 import slabs as SL, workloads as W
    dist.init_process_group("gloo", rank=rank, world_size=world)
    g = _air()
    V0 = np.asfortranarray(W.sphere(g, (0.5, -0.3), 4.0, dims=(0, 1)) + 0.3 * W.random_field(g, 9))
    m = O.method(scheme=O.WENO5, dynamics=O.DYN_AIR3D, params=(5.0, 5.0, 1.0, 1.0), brt=O.BRT_MIN0)
    plan = SL.plan(g, world)
    sources = SL.halo_sources(plan)
    s = plan[rank]
    # dt from the all-reduced maximum of the slabs' CFL bounds
    bound = torch.tensor([O.step_bound_inv(s.spec, m)], dtype=torch.float64)
    dist.all_reduce(bound, op=dist.ReduceOp.MAX)
    dt = 0.8 / float(bound.item())

    def exchange(U):
        sends = []
        for other, src in enumerate(sources):
            for local, k, k_local in src:
                if k == rank and other != rank:
                    sends.append(dist.isend(torch.from_numpy(np.ascontiguousarray(U[..., k_local])), other, tag=local))
        for local, k, k_local in sources[rank]:
            if k == rank:
                U[..., local] = U[..., k_local]
            else:
                buf = torch.empty(U.shape[:-1], dtype=torch.float64)
                dist.recv(buf, k, tag=local)
                U[..., local] = buf.numpy()
        for r in sends:
            r.wait()
        return U

    Vn = np.asfortranarray(V0[..., list(s.planes)])
    L = lambda U: O.term(s.spec, m, U)
    V1 = exchange(np.asfortranarray(Vn + dt * L(Vn)))
    V2 = exchange(np.asfortranarray(0.75 * Vn + 0.25 * (V1 + dt * L(V1))))
    V3 = (Vn + 2.0 * (V2 + dt * L(V2))) / 3.0
    mine = torch.from_numpy(np.ascontiguousarray(V3[..., s.owned]))
    if rank == 0:
        parts = [mine.numpy()]
        for k in range(1, world):
            buf = torch.empty(g.n[:-1] + (plan[k].z1 - plan[k].z0,), dtype=torch.float64)
            dist.recv(buf, k, tag=1000)
            parts.append(buf.numpy())
        got = np.concatenate(parts, axis=-1)
        ref = O.rk3_step(g, m, V0, 0.8 / O.step_bound_inv(g, m))
        q.put((float(bound.item()), O.step_bound_inv(g, m),
               float(np.max(np.abs(got - ref)) / np.max(np.abs(ref)))))
    else:
        dist.send(mine, 0, tag=1000)
    dist.destroy_process_group()


def test_two_gloo_ranks_step_one_grid_by_halo_exchange():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_slab_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    bound, bound_whole, err = q.get(timeout=300)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    assert bound == pytest.approx(bound_whole, rel=1e-14)
    assert err <= 1e-13


def test_plan_splits_the_last_dimension_of_a_4d_grid():
    g = W.GridSpec((7, 6, 5, 12), (0.0,) * 4, (1.0, 1.0, 2.0 * math.pi, 2.0), (2,))
    plan = SL.plan(g, 4)
    assert [(s.z0, s.z1) for s in plan] == [(0, 3), (3, 6), (6, 9), (9, 12)]
    for s in plan:
        assert s.spec.n[:3] == g.n[:3] and s.spec.periodic == (2,)  # theta stays periodic, v is split
        assert s.below == (0 if s.z0 == 0 else 3) and s.above == (0 if s.z1 == 12 else 3)
