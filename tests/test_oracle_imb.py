"""Pins for the oracle's immersed-moving-boundary coupling: Eq. (1), beta of
Eq. (2), the Omega^S term, the force/torque sums of Eq. (3), and the readings
for several owners per node, the rotation term and the force sign."""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_1011_2613_gb300 import inputs as I
from tests.lattice_ref import lattice

TAU = 0.7


def rand_ft(dim, rng):
    Q = 9 if dim == 2 else 19
    return 1.0 / Q * (1 + 0.1 * rng.standard_normal(Q))


def moments(dim, f):
    c, _ = lattice(dim)
    rho = f.sum()
    return rho, c.T.astype(float) @ f / rho


def test_beta_special_values():
    rng = np.random.default_rng(0)
    ft = rand_ft(3, rng)
    g = np.zeros(3)
    v = np.array([[0.01, -0.02, 0.005]])
    _, _, b0 = O.collide_node(3, TAU, g, ft, [0.0], v)
    _, _, b1 = O.collide_node(3, TAU, g, ft, [1.0], v)
    _, _, bh = O.collide_node(3, 1.0, g, ft, [0.5], v)
    assert b0 == 0.0 and b1 == 1.0
    assert abs(bh - 0.25) < 1e-16  # 0.5*0.5 / (0.5 + 0.5)
    # monotone in eps
    bs = [O.collide_node(3, TAU, g, ft, [e], v)[2] for e in np.linspace(0, 1, 11)]
    assert all(b2 > b1_ for b1_, b2 in zip(bs, bs[1:]))


@pytest.mark.parametrize("dim", [2, 3])
def test_uncovered_node_is_plain_bgk(dim):
    rng = np.random.default_rng(1)
    ft = rand_ft(dim, rng)
    g = np.array([1e-4, 2e-4, -1e-4 if dim == 3 else 0.0])
    f_plain, m_plain, _ = O.collide_node(dim, TAU, g, ft)
    f_zero, m_zero, _ = O.collide_node(dim, TAU, g, ft, [0.0], [[0.1, 0.2, 0.3]])
    assert np.array_equal(f_plain, f_zero) and np.all(m_zero == 0)
    # and equals the textbook BGK update with F_i = 3 w_i rho c_i.g
    c, w = lattice(dim)
    rho, u = moments(dim, ft)
    cu = c @ u
    feq = w * rho * (1 + 3 * cu + 4.5 * cu ** 2 - 1.5 * u @ u)
    ref = ft - (ft - feq) / TAU + 3 * w * rho * (c @ g)
    assert np.max(np.abs(f_plain - ref)) < 1e-15 * rho


@pytest.mark.parametrize("dim", [2, 3])
def test_fully_covered_node_takes_solid_velocity(dim):
    """beta = 1: the post-collision momentum is rho (V_S + g_f) exactly."""
    rng = np.random.default_rng(2)
    ft = rand_ft(dim, rng)
    g = np.array([1e-4, -3e-4, 2e-4 if dim == 3 else 0.0])
    VS = np.array([0.02, -0.01, 0.015 if dim == 3 else 0.0])
    fo, m, beta = O.collide_node(dim, TAU, g, ft, [1.0], [VS])
    c, _ = lattice(dim)
    rho, u = moments(dim, ft)
    assert beta == 1.0
    assert np.allclose(c.T @ fo, rho * (VS + g), atol=1e-16)
    assert abs(fo.sum() - rho) < 1e-15


@pytest.mark.parametrize("dim", [2, 3])
def test_momentum_exchange_closed_form(dim):
    """sum_i Omega_i^S c_i = rho (V_S - u) for any populations, so the
    node's momentum exchange is beta rho (V_S - u); mass is untouched."""
    rng = np.random.default_rng(3)
    for _ in range(10):
        ft = rand_ft(dim, rng)
        e = rng.random()
        VS = 0.03 * rng.standard_normal(3)
        if dim == 2:
            VS[2] = 0
        fo, m, beta = O.collide_node(dim, TAU, np.zeros(3), ft, [e], [VS])
        rho, u = moments(dim, ft)
        assert np.allclose(m, beta * rho * (VS - u), atol=1e-16)
        assert abs(fo.sum() - rho) < 1e-15
        assert beta == pytest.approx(e * (TAU - 0.5) / ((1 - e) + (TAU - 0.5)), rel=1e-15)


def test_two_owners_average_velocity_and_cap():
    """Reading for shared nodes: eps = min(1, e1 + e2), V_S weighted by e."""
    rng = np.random.default_rng(4)
    ft = rand_ft(3, rng)
    v1, v2 = np.array([0.01, 0.0, -0.02]), np.array([-0.03, 0.02, 0.01])
    fo2, m2, b2 = O.collide_node(3, TAU, np.zeros(3), ft, [0.3, 0.5], [v1, v2])
    fo1, m1, b1 = O.collide_node(3, TAU, np.zeros(3), ft, [0.8], [(0.3 * v1 + 0.5 * v2) / 0.8])
    assert abs(b1 - b2) < 1e-15 and np.allclose(fo1, fo2, atol=1e-16) and np.allclose(m1, m2, atol=1e-17)
    _, _, bcap = O.collide_node(3, TAU, np.zeros(3), ft, [0.7, 0.6], [v1, v2])
    assert bcap == 1.0


def periodic_cfg(dim, n, parts, vel, omg, density=5.0, g=(0, 0, 0), tau=0.8):
    pos = np.array(parts, dtype=float)
    k = len(pos)
    cfg = I.SuspensionConfig(dim=dim, nx=n, ny=n, nz=n if dim == 3 else 1, wall_y=0, tau=tau,
                             body_force=np.zeros(3), gravity=np.asarray(g, dtype=float), rho_fluid=1.0,
                             k_n=100.0, restitution=0.9, dem_substeps=1, pos=pos,
                             vel=np.asarray(vel, dtype=float), omega=np.asarray(omg, dtype=float),
                             radius=np.full(k, 3.2 if dim == 2 else 2.7), density=np.full(k, density))
    return cfg


def total_momentum(s, dim):
    c, _ = lattice(dim)
    f = s.populations()
    p = s.particles()
    m, _ = s.masses()
    return np.einsum("qd,qzyx->d", c.astype(float), f) + (m[:, None] * p["vel"]).sum(axis=0)


@pytest.mark.parametrize("dim", [2, 3])
def test_total_momentum_conserved_with_moving_particles(dim):
    """Periodic box, no gravity: the momentum the IMB term gives the fluid is
    taken from the particles (force sign reading), and contacts are pairwise,
    so fluid + particle momentum is conserved to round-off.  A flipped force
    sign or a dropped term breaks this by O(1)."""
    n = 28 if dim == 2 else 18
    if dim == 2:
        parts = [[7.3, 8.1, 0], [15.2, 9.4, 0], [20.6, 20.2, 0]]
    else:
        parts = [[5.2, 5.7, 6.1], [12.3, 10.4, 11.8]]
    rng = np.random.default_rng(5)
    vel = 0.01 * rng.standard_normal((len(parts), 3))
    omg = 0.002 * rng.standard_normal((len(parts), 3))
    if dim == 2:
        vel[:, 2] = 0
        omg[:, :2] = 0
    s = O.OracleSim(periodic_cfg(dim, n, parts, vel, omg))
    P0 = total_momentum(s, dim)
    pscale = np.abs((s.masses()[0][:, None] * vel)).sum()
    for _ in range(30 if dim == 2 else 12):
        s.step(1)
    P1 = total_momentum(s, dim)
    assert np.max(np.abs(P1 - P0)) < 1e-12 * pscale
    # the particles did exchange momentum with the fluid
    assert np.max(np.abs(s.particles()["force"])) > 1e-6 * pscale


@pytest.mark.parametrize("dim", [2, 3])
def test_moving_particle_feels_drag(dim):
    n = 24 if dim == 2 else 16
    c0 = [n / 2 + 0.23, n / 2 - 0.17, n / 2 + 0.11 if dim == 3 else 0]
    v = np.array([[0.01, 0.004, 0.002 if dim == 3 else 0.0]])
    s = O.OracleSim(periodic_cfg(dim, n, [c0], v, np.zeros((1, 3))))
    for _ in range(5):
        s.step(1)
        p = s.particles()
        assert float(p["force"][0] @ p["vel"][0]) < 0.0


@pytest.mark.parametrize("dim", [2, 3])
def test_spinning_particle_torque_sign(dim):
    """A spinning particle in fluid at rest loses spin (T . omega < 0) and the
    fluid gains angular momentum about the centre in the same sense as the
    spin, of comparable size.  Pins the sign of omega x r in V_S and of the
    torque sum of Eq. (3) separately (one flipped sign breaks one of the
    two conditions)."""
    n = 24 if dim == 2 else 16
    ctr = np.array([n / 2 + 0.13, n / 2 - 0.21, n / 2 + 0.07 if dim == 3 else 0.0])
    w = np.array([[0.0, 0.0, 0.004]]) if dim == 2 else np.array([[0.001, -0.002, 0.003]])
    s = O.OracleSim(periodic_cfg(dim, n, [ctr], np.zeros((1, 3)), w, density=3.0))
    c, _ = lattice(dim)

    def fluid_L():
        f = s.populations()
        j = np.einsum("qd,qzyx->dzyx", c.astype(float), f)
        nz, ny, nx = f.shape[1:]
        Z, Y, X = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
        r = np.stack([X - ctr[0], Y - ctr[1], (Z - ctr[2]) if dim == 3 else 0 * X])
        return np.cross(r, j, axis=0).reshape(3, -1).sum(axis=1)

    _, I0 = s.masses()
    L0 = fluid_L()
    w0 = s.particles()["omega"][0].copy()
    s.step(3)
    p = s.particles()
    assert float(p["torque"][0] @ p["omega"][0]) < 0
    dLp = I0[0] * (p["omega"][0] - w0)
    dLf = fluid_L() - L0
    assert float(dLf @ w0) > 0
    assert np.linalg.norm(dLf + dLp) < 0.3 * np.linalg.norm(dLp)


def test_symmetric_particle_at_rest_feels_nothing():
    """Particle at rest centred on a node, fluid at rest, no gravity: the
    force and torque vanish by symmetry."""
    s = O.OracleSim(periodic_cfg(3, 14, [[7.0, 7.0, 7.0]], np.zeros((1, 3)), np.zeros((1, 3))))
    s.step(3)
    p = s.particles()
    assert np.max(np.abs(p["force"])) < 1e-15 and np.max(np.abs(p["torque"])) < 1e-15


def test_fluid_mass_conserved_with_particles():
    rng = np.random.default_rng(9)
    vel = 0.01 * rng.standard_normal((2, 3))
    s = O.OracleSim(periodic_cfg(3, 16, [[4.1, 5.2, 6.3], [11.7, 10.2, 9.9]], vel, np.zeros((2, 3))))
    M0 = s.populations().sum()
    s.step(6)
    assert abs(s.populations().sum() - M0) < 1e-13 * M0


def test_eps_field_is_capped_sum():
    s = O.OracleSim(periodic_cfg(2, 24, [[8.0, 12.0, 0], [14.5, 12.3, 0]], np.zeros((2, 3)), np.zeros((2, 3))))
    cnt, ids, e = s.owners()
    _, _, eps = s.fields()
    assert cnt.max() == 2  # the two disks (gap 0.1 lu) share the cells around x = 11
    assert np.allclose(eps.reshape(-1), np.minimum(1.0, e.sum(axis=1)))
    shared = cnt == 2
    assert np.all(ids[shared, 0] < ids[shared, 1])
    for p, R in [(0, 3.2), (1, 3.2)]:
        assert abs(e[ids == p].sum() - math.pi * R * R) < 1e-12
