"""One grid split into slabs along its slowest dimension: the layout a solve of
one grid too large for one GPU would use, one slab per GPU.

- Each slab owns a range of planes and holds three halo planes on each side
  (one RK stage reads three nodes per side). Along a periodic dimension the
  halos wrap around; at a non-periodic grid edge a slab has no halo on that
  side, and the edge's own ghost rule applies.
- A slab is a grid of its own (the extended plane range, not periodic along
  the split dimension). Its stage kernel computes every node, but only the
  owned planes are kept: an owned plane lies at least three planes inside the
  extended range, so its stencils read only true data.
- Before each RK stage the halo planes of the stage's input are refreshed from
  the slabs that own them (the halo exchange).
- dt comes from the maximum over slabs of their CFL bounds (an all-reduce);
  since alpha depends on x only, it is the full grid's bound.

`rk3_step_slabs` runs the whole plan on one GPU, the slabs in turn, with
device-to-device copies as the halo exchange; it must equal `solver.rk3_step`
on the whole grid. The plan itself (`plan`, `halo_sources`) is host logic
only, so a multi-process run can share it.
"""
from __future__ import annotations

from dataclasses import dataclass
from typing import List, Tuple

from . import workloads as W

HALO = 3


@dataclass(frozen=True)
class Slab:
    index: int
    z0: int                 # owned planes [z0, z1) of the split dimension
    z1: int
    below: int              # halo planes below z0 (0 at a non-periodic edge)
    above: int              # halo planes above z1
    planes: Tuple[int, ...]  # global plane index of every extended plane (wrapped)
    spec: W.GridSpec        # the extended slab as a grid

    @property
    def owned(self) -> slice:
        """The owned planes, as local plane indices of the extended slab."""
        return slice(self.below, self.below + self.z1 - self.z0)


def _spacing(spec: W.GridSpec, d: int) -> float:
    return (spec.hi[d] - spec.lo[d]) / (spec.n[d] if d in spec.periodic else spec.n[d] - 1)


def plan(spec: W.GridSpec, n_slabs: int) -> List[Slab]:
    """Owned ranges as equal as possible, each with its halos."""
    D = spec.ndim
    d = D - 1
    n = spec.n[d]
    periodic = d in spec.periodic
    if n_slabs < 1 or n < n_slabs * HALO or (periodic and n_slabs > 1 and n < 2 * HALO + 1):
        raise ValueError("%d planes cannot be split into %d slabs of at least %d" % (n, n_slabs, HALO))
    if n_slabs == 1:
        return [Slab(0, 0, n, 0, 0, tuple(range(n)), spec)]
    dx = _spacing(spec, d)
    slabs = []
    for k in range(n_slabs):
        z0, z1 = k * n // n_slabs, (k + 1) * n // n_slabs
        below = HALO if periodic or z0 > 0 else 0
        above = HALO if periodic or z1 < n else 0
        planes = tuple((z % n) for z in range(z0 - below, z1 + above))
        m = len(planes)
        lo = spec.lo[d] + (z0 - below) * dx
        hi = lo + (m - 1) * dx
        keep_periodic = tuple(p for p in spec.periodic if p != d)
        sub = W.GridSpec(spec.n[:d] + (m,), spec.lo[:d] + (lo,), spec.hi[:d] + (hi,), keep_periodic)
        slabs.append(Slab(k, z0, z1, below, above, planes, sub))
    return slabs


def halo_sources(slabs: List[Slab]):
    """For each slab, the (local plane, owning slab, owner's local plane) of
    every halo plane."""
    owner = {}
    for s in slabs:
        for z in range(s.z0, s.z1):
            owner[z] = (s.index, s.below + (z - s.z0))
    out = []
    for s in slabs:
        src = []
        for local, z in enumerate(s.planes):
            if s.below <= local < s.below + (s.z1 - s.z0):
                continue
            src.append((local, owner[z][0], owner[z][1]))
        out.append(src)
    return out


def step_bound_slabs(ctx, spec: W.GridSpec, method, n_slabs: int) -> float:
    """The CFL bound as the maximum over the slabs' own bounds (the all-reduce)."""
    from . import solver
    return max(solver.step_bound(ctx, s.spec, method) for s in plan(spec, n_slabs))


def rk3_step_slabs(ctx, spec: W.GridSpec, method, V, dt: float, n_slabs: int):
    """One TVD-RK3 step in place on V (a flat CUDA tensor of the whole grid),
    computed slab by slab with a halo exchange before every stage."""
    import torch
    from . import solver
    slabs = plan(spec, n_slabs)
    sources = halo_sources(slabs)
    plane = spec.num_nodes // spec.n[-1]
    whole = V.view(spec.n[-1], plane)
    vn = [whole.index_select(0, torch.tensor(s.planes, device=V.device)).reshape(-1) for s in slabs]
    u = [x.clone() for x in vn]
    out = [torch.empty_like(x) for x in vn]

    def planes_of(k, bufs):
        return bufs[k].view(len(slabs[k].planes), plane)

    for stage in (1, 2, 3):
        for s in slabs:
            solver.rk3_stage(ctx, s.spec, method, stage, u[s.index], vn[s.index] if stage > 1 else None,
                             out[s.index], dt)
        for s, src in zip(slabs, sources):  # halo exchange: owned planes are never written
            dst = planes_of(s.index, out)
            for local, k, k_local in src:
                dst[local].copy_(planes_of(k, out)[k_local])
        u, out = out, u
    for s in slabs:
        whole[s.z0:s.z1].copy_(planes_of(s.index, u)[s.owned])
    return V
