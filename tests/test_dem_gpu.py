"""The standalone DEM contact-force entry point (cell-list kernel of the time
step, Eqs. 4-5) against the oracle's all-pairs contact sum."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1011_2613_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def dense_state(dim, n_side, R, seed, wall):
    """Particles on a jittered grid with spacing below 2R (many overlaps)."""
    rng = np.random.default_rng(seed)
    sp = 2 * R * 0.97
    ext = [int(np.ceil(n_side * sp)) + (2 if wall else 0)] * dim + [1] * (3 - dim)
    g = np.stack(np.meshgrid(*([np.arange(n_side)] * dim), indexing="ij"), -1).reshape(-1, dim)
    pos = np.zeros((len(g), 3))
    pos[:, :dim] = (g + 0.5) * sp + rng.uniform(-0.08, 0.08, (len(g), dim)) * R
    if wall:
        pos[:, 1] += 0.5
        pos[:, 1] -= 1.0  # some touch the bottom wall
    vel = 0.01 * rng.standard_normal((len(g), 3))
    if dim == 2:
        vel[:, 2] = 0
    rad = R * (1 + 0.05 * rng.random(len(g)))
    mass = 100 * rad ** dim
    return ext, pos, vel, rad, mass


@pytest.mark.parametrize("dim,wall", [(2, 0), (2, 1), (3, 0), (3, 1)])
def test_dem_forces_match_oracle(dim, wall):
    import torch
    from paper_1011_2613_gb300 import lbm

    ext, pos, vel, rad, mass = dense_state(dim, 12 if dim == 2 else 6, 3.0, 5 + dim, wall)
    kn, e = 40.0, 0.85
    ref = O.dem_contacts(dim, ext, wall, pos, vel, rad, mass, kn, e)
    t = lambda a: torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")
    fc = lbm.dem_forces(dim, ext, wall, t(pos), t(vel), t(rad), t(mass), kn, e).cpu().numpy()
    nonzero = np.count_nonzero(np.abs(ref).sum(axis=1))
    assert nonzero > len(rad) // 2
    assert np.max(np.abs(fc - ref)) <= 1e-15 * np.max(np.abs(ref))


def test_dem_forces_reject_oversize_radius():
    import torch
    from paper_1011_2613_gb300 import lbm

    ext, pos, vel, rad, mass = dense_state(2, 6, 3.0, 1, 0)
    t = lambda a: torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")
    with pytest.raises(lbm.LbmImbError) as ei:
        lbm.dem_forces(2, ext, 0, t(pos), t(vel), t(rad), t(mass), 40.0, 0.9, rmax=2.0)
    assert ei.value.status == lbm.EBIN
