"""The accuracy metric the benchmark reports for the FP32 path (zero-level-set
displacement in grid cells), checked on fields whose zero sets are known."""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def test_displacement_of_a_shifted_plane_is_the_shift_in_cells():
    # V = x - a on unit-spaced nodes: the zero set sits at x = a; shifting a by
    # 0.3 cells moves every crossing by 0.3
    x = np.arange(20, dtype=np.float64)[:, None, None] * np.ones((1, 5, 4))
    a = 7.25
    assert abs(bench.zero_set_displacement_cells(x - (a + 0.3), x - a) - 0.3) < 1e-12
    assert bench.zero_set_displacement_cells(x - a, x - a) == 0.0


def test_displacement_when_only_one_field_crosses_an_edge():
    # the moved crossing leaves an edge: the lower bound is the distance from
    # the remaining crossing to the nearer end of its edge
    x = np.arange(10, dtype=np.float64)[:, None]
    ref = x - 4.2          # crossing at 4.2 (edge 4-5, 0.2 from node 4)
    moved = x - 5.1        # crossing at 5.1 (edge 5-6)
    d = bench.zero_set_displacement_cells(moved, ref)
    assert abs(d - 0.2) < 1e-12


def test_displacement_of_a_circle_grown_by_a_known_radius():
    n = 81
    h = 2.0 / (n - 1)
    X, Y = np.meshgrid(np.linspace(-1, 1, n), np.linspace(-1, 1, n), indexing="ij")
    r = np.sqrt(X * X + Y * Y)
    d = bench.zero_set_displacement_cells(r - 0.5 - 0.2 * h, r - 0.5)
    # measured along grid lines, a crossing of the circle moves by at least
    # the radial change (exactly that where the line is normal to the circle,
    # more where it meets the circle at a grazing angle): the metric bounds
    # the normal displacement from above
    assert d >= 0.2 - 1e-9
    assert d < 1.0
