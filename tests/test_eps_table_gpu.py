"""GPU: the Eq. 6 table rasterisation against the oracle's table (same
method on both sides) and against the exact covered fractions."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1011_2613_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def lbm():
    from paper_1011_2613_gb300 import lbm as L
    return L


@pytest.mark.parametrize("dim", [2, 3])
def test_table_eps_matches_oracle_table(dim):
    if dim == 2:
        cfg = I.periodic2d_config(nx=96, ny=80, phi=0.2, radius=5.3, seed=4, density_ratio=3.0)
    else:
        cfg = I.periodic3d_config(nx=40, ny=36, nz=32, phi=0.15, radius=3.75, seed=4)
    cfg = cfg.replace(eps_method=1)
    _, _, eg = lbm().Simulation(cfg).fields()
    _, _, er = O.OracleSim(cfg).fields()
    assert np.max(np.abs(eg - er)) < 1e-6
    _, _, ex = lbm().Simulation(cfg.replace(eps_method=0)).fields()
    assert 0 < np.max(np.abs(eg - ex)) < 1e-3


@pytest.mark.parametrize("storage,form", [("f64", 0), ("dfdev", 0), ("dfdev", 6), ("dfdev", 7)])
def test_table_coupled_parity(storage, form):
    """Cut-down config 3 with the table: GPU against the oracle's table run
    (FP64, and the pair storage in its queue and split forms: the split
    form's covered-node list comes from the table rasteriser)."""
    cfg = I.config3_scaled(nx=40, ny=48, nz=36, storage=storage).replace(eps_method=1)
    gpu = lbm().Simulation(cfg)
    gpu.set_collide_variant(form)
    ref = O.OracleSim(cfg)
    gpu.step(30)
    ref.step(30)
    gpu.sync()
    fg, fr = gpu.populations(), ref.populations()
    assert float(np.max(np.abs(fg - fr) / np.abs(fr))) < 1e-10
    pg, pr = gpu.particles(), ref.particles()
    scale = np.max(np.abs(pr["force"]))
    assert np.max(np.abs(pg["force"] - pr["force"])) / scale < 1e-9


def test_table_needs_one_radius():
    L = lbm()
    cfg = I.periodic2d_config(nx=64, ny=64, phi=0.1, radius=4.0, seed=1)
    cfg = cfg.replace(radius=cfg.radius * np.linspace(1.0, 1.1, cfg.n_particles), eps_method=1)
    with pytest.raises(L.LbmImbError) as ei:
        L.Simulation(cfg)
    assert ei.value.status == L.EUNSUPPORTED


def test_batch_members_with_table_match_standalone():
    L = lbm()
    cfgs = [I.periodic2d_config(nx=96, ny=128, phi=0.1, radius=4.0, seed=s).replace(eps_method=1) for s in (1, 2)]
    batch = L.Batch(cfgs)
    alone = [L.Simulation(c) for c in cfgs]
    batch.step(10)
    batch.sync()
    for m, s in zip(batch.members, alone):
        s.step(10)
        s.sync()
        fa, fb = s.populations(), m.populations()
        assert np.max(np.abs(fb - fa) / np.abs(fa)) < 1e-12
