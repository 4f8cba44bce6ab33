"""Pins for the oracle's drag-sample definition (mlp_oracle.drag_samples).

The sample of a particle is defined on the nodes at distance (R, R + shell]
from its centre: their mean solid fraction, the (1 - eps)-weighted mean
fluid velocity minus the particle velocity (slip), the Reynolds number
2 R |slip| / nu, the density ratio, and the force over the Stokes scale
6 pi rho nu R (3D) or 4 pi rho nu (2D).  Each case below is small enough to
work out by hand: the shell's node set is written down explicitly, and every
expected value is computed from those few nodes, so a wrong shell test
(R excluded, R + shell included), a dropped (1 - eps) weight, a missing
periodic image, a wrap across a wall or a wrong Stokes scale fails one of
them.
"""
import math

import numpy as np
import pytest

from oracle import mlp_oracle as M


class FakeSim:
    """The attributes and accessors drag_samples reads, with fields set by
    hand (rho is not used)."""

    def __init__(self, dim, shape, tau, rho0, wall_y, radius, pos, vel, force, mass, u, eps):
        self.dim = dim
        self.shape = shape
        self.tau = tau
        self.rho0 = rho0
        self.wall_y = wall_y
        self.radius = np.asarray(radius, dtype=float)
        self.np = len(self.radius)
        self._p = {"pos": np.asarray(pos, float), "vel": np.asarray(vel, float),
                   "force": np.asarray(force, float)}
        self._m = np.asarray(mass, float)
        self._u = u
        self._eps = eps

    def fields(self):
        nx, ny, nz = self.shape
        return np.ones((nz, ny, nx)), self._u, self._eps

    def particles(self):
        return self._p

    def masses(self):
        return self._m, np.zeros_like(self._m)


def blank(dim, shape):
    nx, ny, nz = shape
    return np.zeros((dim, nz, ny, nx)), np.zeros((nz, ny, nx))


def test_uniform_flow_2d_slip_re_ratio_and_stokes_scale():
    """Uniform u0 and eps = 0 everywhere: slip = u0 - v_p exactly, mean eps
    0, Re = 2 R |u0 - v_p| / nu, ratio = m / (pi R^2 rho0), target =
    F / (4 pi rho0 nu)."""
    dim, shape = 2, (16, 12, 1)
    u, eps = blank(dim, shape)
    u0 = np.array([3e-3, -1e-3])
    u[0], u[1] = u0[0], u0[1]
    tau, rho0, R = 0.8, 1.25, 2.0
    nu = (tau - 0.5) / 3
    vp = np.array([1e-3, 2e-3, 0.0])
    m = 7.0 * math.pi * R * R * rho0  # density ratio 7
    F = np.array([0.03, -0.01, 0.0])
    sim = FakeSim(dim, shape, tau, rho0, 0, [R], [[7.0, 6.0, 0.0]], [vp], [F], [m], u, eps)
    feats, tgt = M.drag_samples(sim, shell=3.0)
    slip = np.array([u0[0] - vp[0], u0[1] - vp[1], 0.0])
    assert feats[0, 0] == 0.0
    assert np.allclose(feats[0, 1:4], slip, rtol=0, atol=1e-18)
    assert feats[0, 4] == pytest.approx(2 * R * np.linalg.norm(slip) / nu, rel=1e-14)
    assert feats[0, 5] == pytest.approx(7.0, rel=1e-14)
    assert np.allclose(tgt[0], F / (4 * math.pi * rho0 * nu), rtol=1e-14, atol=0)


def test_shell_edges_and_weights_2d():
    """R = 1, shell = 1, centre on node (5, 4): the nodes at distance 1 = R
    are outside the shell, those at sqrt 2 and 2 = R + shell inside, those at
    sqrt 5 outside.  The shell is therefore the 4 diagonal neighbours and the
    4 nodes two steps away on the axes.  eps and u are set on exactly these
    8 nodes (and on the excluded ones, to catch a wrong edge test)."""
    dim, shape = 2, (12, 10, 1)
    u, eps = blank(dim, shape)
    cx, cy = 5, 4
    shell = [(1, 1), (-1, 1), (1, -1), (-1, -1), (2, 0), (-2, 0), (0, 2), (0, -2)]
    e_vals = [0.1, 0.2, 0.3, 0.4, 0.0, 0.5, 0.6, 0.7]
    ux_vals = [1.0, 2.0, 3.0, 4.0, 5.0, 6.0, 7.0, 8.0]
    for (dx, dy), e, ux in zip(shell, e_vals, ux_vals):
        eps[0, cy + dy, cx + dx] = e
        u[0, 0, cy + dy, cx + dx] = ux * 1e-3
        u[1, 0, cy + dy, cx + dx] = -ux * 1e-3
    # excluded nodes: distance exactly R (on the axes) and sqrt 5
    for dx, dy in [(1, 0), (-1, 0), (0, 1), (0, -1), (2, 1), (1, 2)]:
        eps[0, cy + dy, cx + dx] = 0.9
        u[0, 0, cy + dy, cx + dx] = 1.0
    tau, rho0, R = 1.0, 1.0, 1.0
    sim = FakeSim(dim, shape, tau, rho0, 0, [R], [[cx, cy, 0.0]], [[0.0, 0.0, 0.0]], [[0.0, 0.0, 0.0]],
                  [math.pi], u, eps)
    feats, _ = M.drag_samples(sim, shell=1.0)
    w = [1 - e for e in e_vals]
    ux_mean = sum(wi * v for wi, v in zip(w, ux_vals)) * 1e-3 / sum(w)
    assert feats[0, 0] == pytest.approx(sum(e_vals) / 8, rel=1e-14)
    assert feats[0, 1] == pytest.approx(ux_mean, rel=1e-13)
    assert feats[0, 2] == pytest.approx(-ux_mean, rel=1e-13)
    assert feats[0, 3] == 0.0


def test_periodic_seam_and_wall_2d():
    """A particle at x = 0.0: its shell wraps to x = nx - 1 in a periodic
    lattice.  Along y a wall (wall_y = 1) stops the wrap: with the centre on
    row 0, the shell node at y = -2 does not exist and row ny - 2 is not its
    image."""
    dim, shape = 2, (10, 8, 1)
    u, eps = blank(dim, shape)
    R, shell = 1.0, 1.0
    # shell of centre (0, 0): (+-1, +-1), (+-2, 0), (0, +-2); x wraps, y does not
    inside = [(1, 1), (9, 1), (2, 0), (8, 0), (0, 2)]
    for x, y in inside:
        u[0, 0, y, x] = 2e-3
    # the periodic images along y that a wrong wrap would pick up
    for x, y in [(1, 7), (9, 7), (0, 6)]:
        u[0, 0, y, x] = 1.0
        eps[0, y, x] = 0.5
    sim = FakeSim(dim, shape, 0.8, 1.0, 1, [R], [[0.0, 0.0, 0.0]], [[0.0, 0.0, 0.0]], [[0.0, 0.0, 0.0]],
                  [math.pi], u, eps)
    feats, _ = M.drag_samples(sim, shell=shell)
    assert feats[0, 0] == 0.0
    assert feats[0, 1] == pytest.approx(2e-3, rel=1e-14)
    # without the wall the images belong to the shell and change the mean
    sim.wall_y = 0
    feats_p, _ = M.drag_samples(sim, shell=shell)
    assert feats_p[0, 0] == pytest.approx(3 * 0.5 / 8, rel=1e-14)
    assert feats_p[0, 1] == pytest.approx((5 * 2e-3 + 3 * 0.5 * 1.0) / (5 + 3 * 0.5), rel=1e-13)


def test_3d_stokes_scale_and_ratio():
    """3D: target = F / (6 pi rho0 nu R), ratio = m / (4/3 pi R^3 rho0);
    the shell of R = 1, shell = 0.5 around a node is its 12 edge neighbours
    (distance sqrt 2; face neighbours at 1 = R are out, corners at sqrt 3 >
    1.5 are out)."""
    dim, shape = 3, (9, 8, 7)
    u, eps = blank(dim, shape)
    c = (4, 3, 3)
    n_in = 0
    for dx in (-1, 0, 1):
        for dy in (-1, 0, 1):
            for dz in (-1, 0, 1):
                if abs(dx) + abs(dy) + abs(dz) == 2:
                    eps[c[2] + dz, c[1] + dy, c[0] + dx] = 0.25
                    u[2, c[2] + dz, c[1] + dy, c[0] + dx] = 4e-3
                    n_in += 1
                elif abs(dx) + abs(dy) + abs(dz) in (1, 3):
                    eps[c[2] + dz, c[1] + dy, c[0] + dx] = 1.0
                    u[2, c[2] + dz, c[1] + dy, c[0] + dx] = 1.0
    assert n_in == 12
    tau, rho0, R = 0.65, 0.9, 1.0
    nu = (tau - 0.5) / 3
    m = 1000.0 * 4 / 3 * math.pi * R ** 3 * rho0
    F = np.array([1e-4, 2e-4, -3e-4])
    vp = np.array([0.0, 0.0, 1e-3])
    sim = FakeSim(dim, shape, tau, rho0, 0, [R], [list(map(float, c))], [vp], [F], [m], u, eps)
    feats, tgt = M.drag_samples(sim, shell=0.5)
    assert feats[0, 0] == pytest.approx(0.25, rel=1e-14)
    assert np.allclose(feats[0, 1:4], [0.0, 0.0, 3e-3], rtol=1e-13, atol=1e-18)
    assert feats[0, 4] == pytest.approx(2 * R * 3e-3 / nu, rel=1e-13)
    assert feats[0, 5] == pytest.approx(1000.0, rel=1e-14)
    assert np.allclose(tgt[0], F / (6 * math.pi * rho0 * nu * R), rtol=1e-14, atol=0)
