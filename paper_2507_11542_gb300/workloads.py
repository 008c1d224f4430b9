"""Seeded synthetic inputs: grid specifications and initial implicit surfaces.

This module generates input data only (grids and initial value functions
V0). It holds none of the level-set method's arithmetic, and both the CUDA
path and the CPU oracle consume what it produces.

Initial surfaces are signed distance functions (negative inside, positive
outside, zero on the interface), the construction of Sec. 2.2 of the paper.
Arrays are float64 numpy arrays of shape ``(n0, ..., n_{D-1})`` in Fortran
order: dimension 0 is contiguous in memory.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import Sequence, Tuple

import numpy as np


@dataclass(frozen=True)
class GridSpec:
    """A dense Cartesian grid (the paper's ``createGrid(min, max, N, pdim)``)."""
    n: Tuple[int, ...]
    lo: Tuple[float, ...]
    hi: Tuple[float, ...]
    periodic: Tuple[int, ...] = field(default_factory=tuple)

    @property
    def ndim(self) -> int:
        return len(self.n)

    @property
    def num_nodes(self) -> int:
        return int(np.prod(self.n))

    def axis(self, d: int) -> np.ndarray:
        """Node positions along dimension d (periodic dims exclude hi)."""
        if d in self.periodic:
            return np.linspace(self.lo[d], self.hi[d], self.n[d], endpoint=False)
        return np.linspace(self.lo[d], self.hi[d], self.n[d])

    def mesh(self):
        return np.meshgrid(*[self.axis(d) for d in range(self.ndim)], indexing="ij")


def sphere(grid: GridSpec, center: Sequence[float], radius: float, dims: Sequence[int] | None = None) -> np.ndarray:
    """Signed distance to a sphere (a cylinder when ``dims`` omits dimensions)."""
    dims = list(range(grid.ndim)) if dims is None else list(dims)
    r2 = np.zeros([1] * grid.ndim)
    for k, d in enumerate(dims):
        shape = [1] * grid.ndim
        shape[d] = grid.n[d]
        r2 = r2 + ((grid.axis(d) - center[k]) ** 2).reshape(shape)   # broadcast: no full mesh
    return np.asfortranarray(np.broadcast_to(np.sqrt(r2) - radius, tuple(grid.n)))


# ----------------------------------------------------------------------------
# The workloads named in the configuration table of the benchmark.
# ----------------------------------------------------------------------------

def double_integrator(n: int = 101, radius: float = 0.5):
    """2-D double integrator: [-1,1]^2, extrapolated boundaries, disk target."""
    g = GridSpec((n, n), (-1.0, -1.0), (1.0, 1.0))
    return g, sphere(g, (0.0, 0.0), radius)


def air3d(n: int = 101, radius: float = 5.0):
    """3-D pursuit-evasion game: [-6,20]x[-10,10]x[0,2pi), psi periodic; cylinder target."""
    g = GridSpec((n, n, n), (-6.0, -10.0, 0.0), (20.0, 10.0, 2.0 * math.pi), (2,))
    return g, sphere(g, (0.0, 0.0), radius, dims=(0, 1))


def dubins4d(n: int = 81, seed: int = 1, radius: float = 1.0):
    """4-D Dubins car with speed: [-5,5]^2 x [0,2pi) x [0,2], theta periodic;
    target = disk of radius 1 in (x, y) at a seeded center uniform in [-2,2]^2."""
    rng = np.random.default_rng(seed)
    c = rng.uniform(-2.0, 2.0, size=2)
    g = GridSpec((n, n, n, n), (-5.0, -5.0, 0.0, 0.0), (5.0, 5.0, 2.0 * math.pi, 2.0), (2,))
    return g, sphere(g, (float(c[0]), float(c[1])), radius, dims=(0, 1))


def rockets(n: int = 100, radius: float = 1.5):
    """Rockets game (Sec. 6.1): (x, z) in [-64, 64]^2, theta in [-pi/2, pi/2],
    extrapolated boundaries; target = the capture cylinder x^2 + z^2 = 1.5^2
    along theta."""
    g = GridSpec((n, n, n), (-64.0, -64.0, -0.5 * math.pi), (64.0, 64.0, 0.5 * math.pi))
    return g, sphere(g, (0.0, 0.0), radius, dims=(0, 1))


def expanding_sphere(n: int = 512, radius: float = 0.25):
    """3-D sphere on [-1,1]^3 for the H = |p| closed-form check."""
    g = GridSpec((n, n, n), (-1.0, -1.0, -1.0), (1.0, 1.0, 1.0))
    return g, sphere(g, (0.0, 0.0, 0.0), radius)


def slice_times(horizon: float, n_slices: int = 11) -> np.ndarray:
    """n_slices equally spaced output times from 0 to horizon (11 slices as in Sec. 6.1)."""
    return np.linspace(0.0, horizon, n_slices)


def random_field(grid: GridSpec, seed: int, scale: float = 1.0) -> np.ndarray:
    """A smooth random field (sum of a few seeded Fourier modes plus a distance
    function) used for parity tests that need generic, tie-free data."""
    rng = np.random.default_rng(seed)
    X = grid.mesh()
    V = np.zeros(grid.n)
    for _ in range(4):
        k = rng.uniform(0.5, 2.0, size=grid.ndim)
        ph = rng.uniform(0, 2 * math.pi)
        arg = ph
        for d in range(grid.ndim):
            span = grid.hi[d] - grid.lo[d]
            arg = arg + 2 * math.pi * k[d] * (X[d] - grid.lo[d]) / span
        V = V + rng.uniform(0.2, 1.0) * np.sin(arg)
    return np.asfortranarray(scale * V)


def batch_mix(seed: int = 42, n_di: int = 32, n_air: int = 32):
    """The batched workload: n_di double-integrator solves with n ~ U{51..201}
    and target radius ~ U[0.2, 0.8] (horizon 1), and n_air air3D solves with
    n ~ U{41..121} and radius ~ U[3, 7] (horizon 2.8), seeded.
    Returns a list of (kind, GridSpec, V0, horizon)."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(n_di):
        n = int(rng.integers(51, 202))
        r = float(rng.uniform(0.2, 0.8))
        g, V0 = double_integrator(n, r)
        out.append(("di", g, V0, 1.0))
    for _ in range(n_air):
        n = int(rng.integers(41, 122))
        r = float(rng.uniform(3.0, 7.0))
        g, V0 = air3d(n, r)
        out.append(("air3d", g, V0, 2.8))
    return out
