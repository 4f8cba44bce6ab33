"""The closed forms the CUDA rasteriser evaluates for the covered area and
volume of a cell (K1), written out in numpy and checked against the oracle's
independent integration (the oracle integrates chord lengths and slice areas;
it never uses these forms).  Corner functions, with the cell reflected into
the positive quadrant/octant:
  2D  U(a, b)    = area of {X > a, Y > b} inside the disk of radius R
                 = R^2/2 (psi(a) + psi(b) - pi/2) - (a s(a) + b s(b))/2 + ab,
                   s(v) = sqrt(R^2 - v^2), psi(v) = atan2(s(v), v);
  3D  P(a, b, c) = volume of {X > a, Y > b, Z > c} inside the ball, from the
                   divergence theorem 3P = R^3 Omega - a A_a - b A_b - c A_c
                   collected into
                 = [R^3 (sum alpha - pi) - sum_d k_d (s_d - pi/2)
                    + ab z_ab + ac z_ac + bc z_bc - 3abc] / 3,
  with z_uv = sqrt(R^2 - u^2 - v^2) (the edge line X = u, Y = v meets the
  sphere at height z_uv), alpha_uv = atan2(R z_uv, u v) (the vertex angle),
  s_a = atan2(z_ab, b) + atan2(z_ac, c) (and cyclically; th_a = s_a - pi/2 is
  the angle of the face X = a), k_v = v (3R^2 - v^2) / 2."""
import math

import numpy as np
import pytest

from oracle import oracle as O


def corner_area(R, a, b):
    if a * a + b * b >= R * R:
        return 0.0
    sa, sb = math.sqrt(R * R - a * a), math.sqrt(R * R - b * b)
    return 0.5 * R * R * (math.atan2(sa, a) + math.atan2(sb, b) - math.pi / 2) - 0.5 * (a * sa + b * sb) + a * b


def corner_volume(R, a, b, c):
    if a * a + b * b + c * c >= R * R:
        return 0.0
    z = lambda u, v: math.sqrt(max(R * R - u * u - v * v, 0.0))
    zab, zac, zbc = z(a, b), z(a, c), z(b, c)
    alpha = math.atan2(R * zab, a * b) + math.atan2(R * zac, a * c) + math.atan2(R * zbc, b * c)
    s_a = math.atan2(zab, b) + math.atan2(zac, c)
    s_b = math.atan2(zab, a) + math.atan2(zbc, c)
    s_c = math.atan2(zac, a) + math.atan2(zbc, b)
    k = lambda v: 0.5 * v * (3 * R * R - v * v)
    t3 = R ** 3 * (alpha - math.pi) - (k(a) * s_a + k(b) * s_b + k(c) * s_c) + math.pi / 2 * (k(a) + k(b) + k(c))
    t3 += a * b * zab + a * c * zac + b * c * zbc - 3 * a * b * c
    return t3 / 3.0


@pytest.mark.parametrize("R", [1.3, 3.75, 6.0])
def test_corner_area_against_oracle(R):
    rng = np.random.default_rng(int(R * 100))
    pts = list(rng.uniform(0, R, (200, 2))) + [(0.0, 0.0), (0.0, 0.5 * R), (0.7 * R, 0.0)]
    for a, b in pts:
        ref = O.area_disk_rect(0.0, 0.0, R, a, R, b, R)
        assert abs(corner_area(R, a, b) - ref) < 1e-12 * R * R


def corner_volume_by_slices(R, a, b, c):
    """P(a, b, c) as the integral over x of the 2D corner area of the slice
    (radius sqrt(R^2 - x^2)), in 30-digit arithmetic."""
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 30
    R, a, b, c = (mp.mpf(v) for v in (R, a, b, c))

    def area(x):
        r2 = R * R - x * x
        if r2 <= b * b + c * c:
            return mp.mpf(0)
        sb, sc = mp.sqrt(r2 - b * b), mp.sqrt(r2 - c * c)
        return r2 / 2 * (mp.atan2(sb, b) + mp.atan2(sc, c) - mp.pi / 2) - (b * sb + c * sc) / 2 + b * c

    top = R * R - b * b - c * c
    return float(mp.quad(area, [a, mp.sqrt(top)])) if top > a * a else 0.0


@pytest.mark.parametrize("R", [1.3, 3.75, 6.0])
def test_corner_volume_against_slices(R):
    """Includes corners on coordinate planes (a, b or c = 0, where
    atan2(z, 0) = pi/2), near the rim, and the octant itself."""
    rng = np.random.default_rng(int(R * 100) + 7)
    pts = [tuple(p) for p in rng.uniform(0, R / math.sqrt(3) * 1.6, (40, 3))]
    pts += [(0.0, 0.0, 0.4 * R), (0.3 * R, 0.0, 0.5 * R), (0.5 * R, 0.5 * R, 0.69 * R)]
    n_inside = 0
    for a, b, c in pts:
        got = corner_volume(R, a, b, c)
        n_inside += got > 0
        assert abs(got - corner_volume_by_slices(R, a, b, c)) < 1e-13 * R ** 3, (a, b, c)
    assert n_inside > 10
    assert abs(corner_volume(R, 0.0, 0.0, 0.0) - math.pi * R ** 3 / 6) < 1e-13 * R ** 3


def cell_fraction_from_corners(R, off):
    """Covered volume of the unit cell centred at off from the centre: each
    axis interval reflected onto the non-negative half-axis (split at 0 when
    it straddles it), then inclusion-exclusion over the box corners."""
    pieces = []
    for o in off:
        lo, hi = o - 0.5, o + 0.5
        if lo >= 0:
            pieces.append([(lo, hi)])
        elif hi <= 0:
            pieces.append([(-hi, -lo)])
        else:
            pieces.append([(0.0, -lo), (0.0, hi)])
    tot = 0.0
    for pa in pieces[0]:
        for pb in pieces[1]:
            for pc in pieces[2]:
                for sx in (0, 1):
                    for sy in (0, 1):
                        for sz in (0, 1):
                            v = corner_volume(R, pa[sx], pb[sy], pc[sz])
                            tot += -v if (sx + sy + sz) & 1 else v
    return tot


@pytest.mark.parametrize("R", [1.3, 3.75, 6.0])
def test_cell_fractions_from_corners_against_oracle(R):
    """The rasteriser's route (corners, then inclusion-exclusion) against the
    oracle's slice integration of whole cells.  The bound is the oracle's:
    its 24-point Gauss-Legendre pieces are good to about 5e-12 on the cells
    of a small sphere (R = 1.3), where the corner forms agree with 30-digit
    integration to 1e-15; 1e-13 and better from R = 3.75 on."""
    rng = np.random.default_rng(int(R * 10) + 3)
    c = rng.random(3)
    n = int(R) + 2
    worst, checked = 0.0, 0
    for i in range(-n, n + 1):
        for j in range(-n, n + 1):
            for k in range(-n, n + 1):
                off = (i - c[0], j - c[1], k - c[2])
                d = math.sqrt(sum(max(abs(o) - 0.5, 0.0) ** 2 for o in off))
                if d >= R or math.sqrt(sum((abs(o) + 0.5) ** 2 for o in off)) <= R:
                    continue  # only cells the surface crosses
                ref = O.cell_fraction(3, c, R, (i, j, k))
                worst = max(worst, abs(cell_fraction_from_corners(R, off) - ref))
                checked += 1
    assert checked > 20 and worst < (1e-11 if R < 2 else 1e-12)
