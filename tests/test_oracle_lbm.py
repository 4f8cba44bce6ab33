"""Pins for the oracle's fluid part: LBGK D2Q9/D3Q19 with body force
(section "Numerical scheme", Eq. 1 with beta = 0), pull streaming and halfway
bounce-back walls.  Checked against an independent numpy LBGK, exact
conservation laws and the analytic body-force-driven channel profile."""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_1011_2613_gb300 import inputs as I
from tests.lattice_ref import lattice, numpy_lbgk_step


def fluid_cfg(dim, nx, ny, nz=1, wall_y=0, tau=0.6, g=(0.0, 0.0, 0.0)):
    return I.SuspensionConfig(dim=dim, nx=nx, ny=ny, nz=nz if dim == 3 else 1, wall_y=wall_y, tau=tau,
                              body_force=np.asarray(g, dtype=float), gravity=np.zeros(3), rho_fluid=1.0,
                              k_n=1.0, restitution=0.9, dem_substeps=1, pos=np.zeros((0, 3)),
                              vel=np.zeros((0, 3)), omega=np.zeros((0, 3)), radius=np.zeros(0),
                              density=np.zeros(0))


@pytest.mark.parametrize("dim,wall", [(2, 0), (2, 1), (3, 0), (3, 1)])
def test_matches_independent_numpy_lbgk(dim, wall):
    cfg = fluid_cfg(dim, 10, 7, 6, wall_y=wall, tau=0.73, g=(2e-4, -1e-4, 3e-4 if dim == 3 else 0.0))
    rng = np.random.default_rng(11)
    f0 = I.random_populations(rng, cfg)
    s = O.OracleSim(cfg)
    s.set_populations(f0)
    f = f0.copy()
    for _ in range(5):
        s.step(1)
        f = numpy_lbgk_step(f, dim, cfg.tau, cfg.body_force, wall)
    got = s.populations()
    assert np.max(np.abs(got - f) / np.abs(f)) < 1e-13


@pytest.mark.parametrize("dim", [2, 3])
def test_mass_and_momentum_budget_periodic(dim):
    g = np.array([1e-5, -2e-5, 0.5e-5 if dim == 3 else 0.0])
    cfg = fluid_cfg(dim, 9, 8, 7, wall_y=0, tau=0.81, g=g)
    rng = np.random.default_rng(3)
    s = O.OracleSim(cfg)
    s.set_populations(I.random_populations(rng, cfg))
    c, _ = lattice(dim)
    f = s.populations()
    M0 = f.sum()
    P0 = np.einsum("qd,qzyx->d", c.astype(float), f)
    for k in range(1, 4):
        s.step(1)
        f = s.populations()
        assert abs(f.sum() - M0) < 1e-13 * M0
        P = np.einsum("qd,qzyx->d", c.astype(float), f)
        # every step adds sum_n rho_n g = M g of momentum (sum_i F_i c_i = rho g)
        assert np.allclose(P - P0, k * M0 * g, rtol=0, atol=1e-13 * M0)


@pytest.mark.parametrize("dim", [2, 3])
def test_poiseuille_exact_at_magic_tau(dim):
    """Body-force driven channel between halfway bounce-back walls: at
    (tau - 1/2)^2 = 3/16 the walls sit exactly at y = -1/2 and H - 1/2 and the
    velocity u(y) = g y'(H - y') / (2 nu), y' = y + 1/2, nu = (tau - 1/2)/3."""
    tau = 0.5 + math.sqrt(3.0 / 16.0)
    H, g = 16, 1e-5
    nu = (tau - 0.5) / 3.0
    s = O.OracleSim(fluid_cfg(dim, 1, H, 2, wall_y=1, tau=tau, g=(g, 0, 0)))
    s.step(6000)
    rho, u, _ = s.fields()
    ux = u[0, 0, :, 0]
    y = np.arange(H) + 0.5
    ua = g / (2 * nu) * y * (H - y)
    assert np.max(np.abs(ux - ua)) < 1e-10 * ua.max()
    assert np.max(np.abs(u[1])) < 1e-14


@pytest.mark.parametrize("tau", [0.6, 1.0, 1.3])
def test_poiseuille_curvature_any_tau(tau):
    """In the bulk the discrete second difference of u equals -g/nu for any
    tau (only the wall position depends on tau)."""
    H, g = 20, 1e-6
    nu = (tau - 0.5) / 3.0
    s = O.OracleSim(fluid_cfg(2, 1, H, wall_y=1, tau=tau, g=(g, 0, 0)))
    s.step(int(25 * H * H / (nu * math.pi ** 2)))  # ~25 e-folds of the slowest mode
    _, u, _ = s.fields()
    ux = u[0, 0, :, 0]
    d2 = ux[2:] - 2 * ux[1:-1] + ux[:-2]
    assert np.allclose(d2[2:-2], -g / nu, rtol=1e-8)
