"""Batched persistent step: every member of a batch evolves exactly as the
same suspension run alone (the same device code; only the order of the FP64
force atomics may differ), for several launch shapes; the grid-barrier
timeout path returns LBM_IMB_ETIMEOUT and leaves the context usable."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1011_2613_gb300 import inputs as I

pytestmark = pytest.mark.gpu
TOL = 1e-12


def small_batch(storage="f64"):
    cfgs = I.batch_configs(n=4, seed=11, nx_range=(40, 130), ny_range=(64, 200), np_range=(3, 40),
                           r_range=(3.0, 5.0), v0=0.02, storage=storage)
    return cfgs


def compare(member, alone):
    fb, fa = member.populations(), alone.populations()
    pb, pa = member.particles(), alone.particles()
    assert np.max(np.abs(fb - fa) / np.abs(fa)) < TOL
    if len(pa["pos"]):
        assert np.max(np.abs(pb["pos"] - pa["pos"])) < TOL
        scale = max(np.max(np.abs(pa["force"])), 1e-300)
        assert np.max(np.abs(pb["force"] - pa["force"])) / scale < 1e-9


@pytest.mark.parametrize("tile_x,bps", [(0, 0), (32, 1), (64, 2)])
def test_batch_members_match_standalone(tile_x, bps):
    from paper_1011_2613_gb300 import lbm

    cfgs = small_batch()
    batch = lbm.Batch(cfgs, tile_x=tile_x, blocks_per_sm=bps)
    alone = [lbm.Simulation(c) for c in cfgs]
    batch.step(30)
    batch.sync()
    for s in alone:
        s.step(30)
        s.sync()
    for m, s in zip(batch.members, alone):
        compare(m, s)


def test_batch_3d_members_and_oracle():
    from paper_1011_2613_gb300 import lbm

    cfgs = [I.config3_scaled(nx=24, ny=30, nz=20, seed=3), I.periodic3d_config(nx=20, ny=26, nz=22, phi=0.1, seed=6)]
    batch = lbm.Batch(cfgs)
    batch.step(12)
    batch.sync()
    for m, c in zip(batch.members, cfgs):
        ref = O.OracleSim(c)
        ref.step(12)
        fr = ref.populations()
        assert np.max(np.abs(m.populations() - fr) / np.abs(fr)) < 1e-10
        pr, pm = ref.particles(), m.particles()
        scale = max(np.max(np.abs(pr["force"])), 1e-300)
        assert np.max(np.abs(pm["force"] - pr["force"])) / scale < 1e-9


def test_batch_reduced_storage_runs():
    from paper_1011_2613_gb300 import lbm

    cfgs = small_batch(storage="f32dev")
    batch = lbm.Batch(cfgs)
    alone = [lbm.Simulation(c) for c in cfgs]
    batch.step(10)
    batch.sync()
    for m, s in zip(batch.members, alone):
        s.step(10)
        fa, fb = s.populations(), m.populations()
        assert np.max(np.abs(fb - fa)) < 1e-6


def test_batch_barrier_timeout_is_reported():
    """Every barrier waits for one arrival that never comes; each wait gives
    up after 2000 polls, the launch ends and the status says so.  Afterwards
    the same batch steps normally."""
    from paper_1011_2613_gb300 import lbm

    batch = lbm.Batch(small_batch())
    batch.set_barrier_test(2000, 1)
    batch.step(1)
    with pytest.raises(lbm.LbmImbError) as ei:
        batch.sync()
    assert ei.value.status == lbm.ETIMEOUT
    batch.set_barrier_test(1 << 25, 0)
    batch.step(2)
    batch.sync()
