"""GPU: DEM contacts from Verlet neighbour lists (dem_skin > 0, rebuilt on
the device when a particle has moved more than half the skin) give the
trajectories of the per-step cell list and of the oracle's all-pairs DEM."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1011_2613_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def lbm():
    from paper_1011_2613_gb300 import lbm as L
    return L


@pytest.mark.parametrize("dim", [2, 3])
def test_verlet_matches_cell_list_and_oracle(dim):
    if dim == 2:
        cfg = I.periodic2d_config(nx=100, ny=72, phi=0.25, radius=4.0, seed=9, v0=0.03, density_ratio=4.0)
        steps = 150
    else:
        cfg = I.periodic3d_config(nx=36, ny=32, nz=30, phi=0.2, radius=3.5, seed=5, v0=0.03, density_ratio=3.0)
        steps = 60
    L = lbm()
    cell = L.Simulation(cfg)
    ver = L.Simulation(cfg.replace(dem_skin=0.6))
    ref = O.OracleSim(cfg)
    cell.step(steps)
    ver.step(steps)
    ref.step(steps)
    pc, pv, pr = cell.particles(), ver.particles(), ref.particles()
    builds = ver.dem_rebuilds()
    assert 2 <= builds < steps  # moved past half the skin, but not every step
    assert cell.dem_rebuilds() == 0
    for k in ("pos", "vel", "force"):
        scale = max(np.max(np.abs(pr[k])), 1e-300)
        assert np.max(np.abs(pv[k] - pc[k])) / scale < 1e-9, k
        assert np.max(np.abs(pv[k] - pr[k])) / scale < 1e-9, k
    assert float(np.max(np.abs(ver.populations() - ref.populations()) / ref.populations())) < 1e-10


def test_verlet_rejected_in_batch():
    L = lbm()
    cfgs = [I.periodic2d_config(nx=96, ny=128, phi=0.1, radius=4.0, seed=s).replace(dem_skin=0.5) for s in (1, 2)]
    with pytest.raises(L.LbmImbError) as ei:
        L.Batch(cfgs)
    assert ei.value.status == L.EUNSUPPORTED
