"""Pins for the oracle's solid fraction eps (covered area/volume of a lattice
cell; the definition in the text after the Omega^S equation).  Each test fixes
eps by something other than the oracle's own integration: closed forms of
circle/sphere pieces, exact totals, and brute-force point sampling."""
import math

import numpy as np
import pytest

from oracle import oracle as O


@pytest.mark.parametrize("R", [0.3, 0.5, 1.7, 4.0, 6.0, 8.0])
def test_cells_sum_to_disk_area(R):
    rng = np.random.default_rng(int(R * 10))
    for _ in range(4):
        c = rng.random(2) * 3
        lo, hi = int(math.floor(c.min() - R)) - 2, int(math.ceil(c.max() + R)) + 2
        tot = sum(O.cell_fraction(2, c, R, (i, j)) for i in range(lo, hi) for j in range(lo, hi))
        assert abs(tot / (math.pi * R * R) - 1) < 1e-13


@pytest.mark.parametrize("R", [0.5, 1.7, 3.75, 5.0])
def test_cells_sum_to_ball_volume(R):
    rng = np.random.default_rng(int(R * 10) + 1)
    c = rng.random(3) * 2
    lo, hi = int(math.floor(c.min() - R)) - 1, int(math.ceil(c.max() + R)) + 2
    tot = 0.0
    for i in range(lo, hi):
        for j in range(lo, hi):
            for k in range(lo, hi):
                tot += O.cell_fraction(3, c, R, (i, j, k))
    assert abs(tot / (4.0 / 3.0 * math.pi * R ** 3) - 1) < 1e-13


def test_special_values():
    # radius-1/2 disk / ball centred on a node fills the inscribed circle / sphere
    assert abs(O.cell_fraction(2, (0.0, 0.0), 0.5, (0, 0)) - math.pi / 4) < 1e-15
    assert abs(O.cell_fraction(3, (0.0, 0.0, 0.0), 0.5, (0, 0, 0)) - math.pi / 6) < 1e-15
    # a node deeper than R - sqrt(d)/2 is fully covered, one beyond R + sqrt(d)/2 is empty
    assert O.cell_fraction(2, (0.3, 0.1), 4.0, (2, 2)) == 1.0  # |r|^2 = 4.9+3.6 -> corner 3.63 < 4
    assert O.cell_fraction(2, (0.3, 0.1), 4.0, (4, 3)) == 0.0
    assert O.cell_fraction(3, (0.2, 0.1, 0.4), 3.75, (1, 1, 1)) == 1.0
    assert O.cell_fraction(3, (0.2, 0.1, 0.4), 3.75, (4, 3, 0)) == 0.0


@pytest.mark.parametrize("a", [-3.9, -2.5, -0.7, 0.0, 0.3, 1.9, 3.2, 3.999])
def test_circular_segment_closed_form(a):
    R = 4.0
    seg = R * R * math.acos(a / R) - a * math.sqrt(R * R - a * a)  # area of {x > a} in the disk
    got = O.area_disk_rect(0.0, 0.0, R, a, 50.0, -50.0, 50.0)
    assert abs(got - seg) < 1e-13 * R * R


@pytest.mark.parametrize("c", [-3.7, -2.0, -0.4, 0.0, 0.9, 2.5, 3.74])
def test_spherical_cap_closed_form(c):
    R = 3.75
    cap = math.pi * (R - c) ** 2 * (2 * R + c) / 3.0  # volume of {z > c} in the ball
    got = O.volume_ball_box(0.0, 0.0, 0.0, R, -50, 50, -50, 50, c, 50)
    assert abs(got - cap) < 1e-13 * R ** 3


def test_quadrant_and_octant():
    R = 2.3
    assert abs(O.area_disk_rect(0, 0, R, 0, 9, 0, 9) - math.pi * R * R / 4) < 1e-14
    assert abs(O.volume_ball_box(0, 0, 0, R, 0, 9, 0, 9, 0, 9) - math.pi * R ** 3 / 6) < 1e-13


def test_reflection_symmetry():
    rng = np.random.default_rng(7)
    for _ in range(20):
        c = rng.random(3)
        n = rng.integers(-3, 4, size=3)
        v = O.cell_fraction(3, c, 3.75, n)
        w = O.cell_fraction(3, -c, 3.75, -n)
        assert abs(v - w) < 1e-14


def _brute_2d(c, R, node, m):
    h = 1.0 / m
    s = (np.arange(m) + 0.5) * h - 0.5
    X, Y = np.meshgrid(node[0] + s - c[0], node[1] + s - c[1], indexing="ij")
    return np.count_nonzero(X * X + Y * Y < R * R) * h * h


def _brute_3d(c, R, node, m):
    h = 1.0 / m
    s = (np.arange(m) + 0.5) * h - 0.5
    X, Y = np.meshgrid(node[0] + s - c[0], node[1] + s - c[1], indexing="ij")
    XY = X * X + Y * Y
    tot = 0
    for zk in node[2] + s - c[2]:
        tot += np.count_nonzero(XY + zk * zk < R * R)
    return tot * h ** 3


def test_brute_force_supersampling_2d():
    """Stratified 4096^2 point count per cell (error ~1e-5) on partially
    covered cells of a small grid."""
    c, R = (0.37, -0.21), 2.6
    checked = 0
    for i in range(-3, 4):
        for j in range(-3, 4):
            e = O.cell_fraction(2, c, R, (i, j))
            if 0.0 < e < 1.0:
                assert abs(e - _brute_2d(c, R, (i, j), 4096)) < 5e-5
                checked += 1
    assert checked >= 8


def test_brute_force_supersampling_3d():
    """Stratified 256^3 point count per cell (error ~1e-4) on a sample of
    partially covered cells."""
    c, R = (0.29, -0.13, 0.41), 1.9
    cells = [(i, j, k) for i in range(-2, 3) for j in range(-2, 3) for k in range(-2, 3)]
    checked = 0
    for n in cells[::3]:
        e = O.cell_fraction(3, c, R, n)
        if 0.0 < e < 1.0:
            assert abs(e - _brute_3d(c, R, n, 256)) < 3e-4
            checked += 1
    assert checked >= 6
