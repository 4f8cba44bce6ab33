"""Pins for the oracle's Eq. 6 table (covered fraction looked up over the
cell's offset from the centre): the entries are the exact fractions at the
grid points, interpolation stays within its bound, the table respects the
reflection/permutation symmetry of a cell, and a whole particle still covers
its area/volume."""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_1011_2613_gb300 import inputs as I


def one_particle(dim, R, centre):
    n = 24
    return I.SuspensionConfig(
        dim=dim, nx=n, ny=n, nz=n if dim == 3 else 1, wall_y=0, tau=0.8, body_force=np.zeros(3),
        gravity=np.zeros(3), rho_fluid=1.0, k_n=0.0, restitution=0.9, dem_substeps=1,
        pos=np.array([centre]), vel=np.zeros((1, 3)), omega=np.zeros((1, 3)), radius=np.array([R]),
        density=np.array([2.0]), eps_method=1)


def grid_offset(dim, R, i, j, k=0):
    """Cell-centre offset of table point (i, j[, k]) (the table's grid)."""
    if dim == 2:
        r = (R - math.sqrt(2) / 2) + i * (math.sqrt(2) / 255)
        t = j / 127
        a = r / math.sqrt(1 + t * t)
        return (a, a * t, 0.0)
    r = (R - math.sqrt(3) / 2) + i * (math.sqrt(3) / 95)
    s = j * (math.sqrt(2) / 63)
    t = k / 47
    a = r / math.sqrt(1 + s * s)
    b = a * s / math.sqrt(1 + t * t)
    return (a, b, b * t)


@pytest.mark.parametrize("dim,R", [(2, 4.0), (2, 6.3), (3, 3.75), (3, 5.2)])
def test_entries_are_exact_fractions(dim, R):
    sim = O.OracleSim(one_particle(dim, R, [12.3, 11.7, 12.1 if dim == 3 else 0.0]))
    rng = np.random.default_rng(dim)
    for _ in range(40):
        if dim == 2:
            off = grid_offset(2, R, rng.integers(0, 256), rng.integers(0, 128))
        else:
            off = grid_offset(3, R, rng.integers(0, 96), rng.integers(0, 64), rng.integers(0, 48))
        exact = O.cell_fraction(dim, (0.0, 0.0, 0.0), R, off)
        # at a grid point the interpolation weights are 0 up to FP32 rounding
        assert abs(sim.eps_table_value(off) - exact) < 2e-5


@pytest.mark.parametrize("dim,R,bound", [(2, 4.0, 4e-4), (3, 3.75, 6e-4)])
def test_interpolation_error_bound(dim, R, bound):
    sim = O.OracleSim(one_particle(dim, R, [12.0, 12.0, 12.0 if dim == 3 else 0.0]))
    rng = np.random.default_rng(7)
    errs = []
    for _ in range(600):
        v = rng.standard_normal(dim)
        v = v / np.linalg.norm(v) * rng.uniform(R - math.sqrt(dim) / 2, R + math.sqrt(dim) / 2)
        off = tuple(v) + (0.0,) * (3 - dim)
        exact = O.cell_fraction(dim, (0.0, 0.0, 0.0), R, off)
        errs.append(abs(min(max(sim.eps_table_value(off), 0.0), 1.0) - exact))
    assert max(errs) < bound
    assert np.mean(errs) < bound / 10


def test_symmetry_of_the_lookup():
    sim = O.OracleSim(one_particle(3, 3.75, [12.0, 12.0, 12.0]))
    rng = np.random.default_rng(3)
    for _ in range(50):
        a, b, c = rng.uniform(0, 4.5, 3)
        ref = sim.eps_table_value((a, b, c))
        for off in [(b, c, a), (c, a, b), (-a, b, -c), (a, -c, b), (-b, -a, -c)]:
            assert sim.eps_table_value(off) == ref


@pytest.mark.parametrize("dim,R", [(2, 5.3), (3, 3.75)])
def test_particle_covers_its_volume(dim, R):
    rng = np.random.default_rng(11)
    for _ in range(3):
        c = [12.0 + rng.uniform(-0.5, 0.5) for _ in range(3)]
        if dim == 2:
            c[2] = 0.0
        sim = O.OracleSim(one_particle(dim, R, c))
        _, _, eps = sim.fields()
        vol = math.pi * R * R if dim == 2 else 4.0 / 3.0 * math.pi * R ** 3
        assert abs(eps.sum() - vol) < 2e-4 * vol
        exact = O.OracleSim(one_particle(dim, R, c).replace(eps_method=0))
        _, _, ee = exact.fields()
        assert np.max(np.abs(eps - ee)) < 1e-3
        assert np.array_equal(eps == 1.0, ee == 1.0)  # the same full cells
        assert np.array_equal(eps > 0, ee > 0) or np.sum((eps > 0) != (ee > 0)) <= 2


def test_table_needs_one_radius():
    cfg = I.periodic2d_config(nx=64, ny=64, phi=0.1, radius=4.0, seed=1)
    cfg = cfg.replace(radius=cfg.radius * np.linspace(1.0, 1.1, cfg.n_particles), eps_method=1)
    with pytest.raises(ValueError):
        O.OracleSim(cfg)
