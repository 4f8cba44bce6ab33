"""GPU: a lattice decomposed into y slabs with halo exchange (the paper's
multi-GPU subdomains, emulated on one device) follows the single-lattice
run; the paper reports a difference of about 1e-13 between its multi- and
single-GPU runs, here the only difference is the order of the FP64 force
sums."""
import numpy as np
import pytest

from paper_1011_2613_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def lbm():
    from paper_1011_2613_gb300 import lbm as L
    return L


@pytest.mark.parametrize("case,nslabs", [("channel2d", 2), ("channel2d", 3), ("periodic3d", 3),
                                         ("channel3d", 4)])
def test_slabs_follow_the_whole_lattice(case, nslabs):
    if case == "channel2d":
        cfg = I.channel_config(nx=96, ny=130, n_particles=10, radius=5.0)
        steps = 200
    elif case == "periodic3d":
        cfg = I.periodic3d_config(nx=32, ny=45, nz=28, phi=0.12, radius=3.5, seed=2, v0=0.02)
        steps = 60
    else:
        cfg = I.config3_scaled(nx=40, ny=50, nz=32)
        steps = 40
    L = lbm()
    whole = L.Simulation(cfg)
    slabs = L.Slabs(cfg, nslabs)
    # one step: every node's arithmetic is the same as in the whole lattice
    # (only the order of owner slots claimed concurrently may differ)
    whole.step(1)
    slabs.step(1)
    whole.sync()
    slabs.sync()
    fw, fs = whole.populations(), slabs.populations()
    assert fs.shape == fw.shape
    assert float(np.max(np.abs(fs - fw) / np.abs(fw))) < 1e-14
    whole.step(steps - 1)
    slabs.step(steps - 1)
    whole.sync()
    slabs.sync()
    fw, fs = whole.populations(), slabs.populations()
    d_pop = float(np.max(np.abs(fs - fw) / np.abs(fw)))
    pw, ps = whole.particles(), slabs.particles()
    d_part = {k: float(np.max(np.abs(ps[k] - pw[k])) / max(np.max(np.abs(pw[k])), 1e-300))
              for k in ("pos", "vel", "force")}
    print(f"{case} {nslabs} slabs, {steps} steps: populations {d_pop:.2e}, particles {d_part}")
    assert d_pop < 1e-11
    assert d_part["pos"] < 1e-12 and d_part["vel"] < 1e-10 and d_part["force"] < 1e-9


def test_slab_rows_split():
    L = lbm()
    assert L.slab_rows(10, 3) == [(0, 4), (4, 3), (7, 3)]
    with pytest.raises(L.LbmImbError):
        L.Slabs(I.channel_config(nx=32, ny=5, n_particles=0), 3)  # a slab of one row


@pytest.mark.parametrize("storage", ["f32dev", "f16dev"])
def test_slabs_reduced_precision_storage(storage):
    """The halo rows carry the stored form (FP32 / FP16 deviations) byte for
    byte: after one step the slabs hold the whole lattice's values; later the
    force sums' order reaches the FP32 arithmetic only through the particle
    velocities."""
    cfg = I.config3_scaled(nx=40, ny=48, nz=32, storage=storage)
    L = lbm()
    whole = L.Simulation(cfg)
    slabs = L.Slabs(cfg, 3)
    whole.step(1)
    slabs.step(1)
    fw, fs = whole.populations(), slabs.populations()
    assert float(np.max(np.abs(fs - fw) / np.abs(fw))) < 1e-14
    whole.step(30)
    slabs.step(30)
    fw, fs = whole.populations(), slabs.populations()
    assert float(np.max(np.abs(fs - fw) / np.abs(fw))) < 1e-5


def test_slabs_pair_storage():
    """The halo rows of the pair storage carry both FP32 halves of every
    population: the slabs follow the whole lattice at FP64 level."""
    cfg = I.config3_scaled(nx=40, ny=48, nz=32, storage="dfdev")
    L = lbm()
    whole = L.Simulation(cfg)
    slabs = L.Slabs(cfg, 3)
    whole.step(30)
    slabs.step(30)
    fw, fs = whole.populations(), slabs.populations()
    assert float(np.max(np.abs(fs - fw) / np.abs(fw))) < 1e-12
