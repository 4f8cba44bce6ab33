"""More paths beside the FP64 CPU oracle, on the same seeded inputs.

* The reduced-precision storages (FP32 and FP16 deviations, and the FP32-pair
  storage) against the oracle itself, not against the library's own FP64
  run: the velocity-field L2 error, the particle positions and the mass
  drift after 60 steps of the cut-down config 3.  FP32/FP16 are reported
  and bounded loosely (their error is what they trade for bandwidth); the
  pair storage must meet the FP64 tolerances.
* The y-slab decomposition (the paper's multi-GPU subdomains on one device)
  against the oracle's whole-lattice run: 2, 3 and 4 slabs, walls and
  periodic, 200 steps, at the FP64 parity tolerances.
* The fixed-sphere configuration of the validation (density ratio 1e12, a
  body force on the gas, tau = 1, fully periodic) stepped beside the oracle.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1011_2613_gb300 import inputs as I

pytestmark = pytest.mark.gpu

POP_TOL = 1e-10
FORCE_TOL = 1e-9


def lbm():
    from paper_1011_2613_gb300 import lbm as L
    return L


def rel_err(a, b):
    return float(np.max(np.abs(a - b) / np.abs(b)))


def force_err(pg, pr, key="force"):
    scale = max(float(np.max(np.abs(pr[key]))), 1e-300)
    return float(np.max(np.abs(pg[key] - pr[key]))) / scale


def errors_vs_oracle(sim, ref):
    """velocity-field L2 (relative), particle position max (lattice units,
    minimum image on periodic axes), relative mass drift."""
    _, ug, _ = sim.fields()
    _, ur, _ = ref.fields()
    l2 = float(np.linalg.norm(ug - ur) / np.linalg.norm(ur))
    pg, pr = sim.particles(), ref.particles()
    d = pg["pos"] - pr["pos"]
    for ax, n in enumerate(sim.shape):
        if not (ax == 1 and sim.cfg.wall_y):
            d[:, ax] -= n * np.round(d[:, ax] / n)
    pos = float(np.sqrt((d ** 2).sum(axis=1)).max())
    mg = float(sim.populations().sum())
    mr = float(ref.populations().sum())
    return l2, pos, abs(mg - mr) / mr, force_err(pg, pr)


@pytest.mark.parametrize("storage,tol_u,tol_pos,tol_m,tol_f", [
    ("f32dev", 1e-4, 1e-6, 1e-8, 1e-3),
    ("f16dev", 3e-2, 1e-4, 1e-6, 3e-2),
    ("dfdev", 1e-10, 1e-9, 1e-13, FORCE_TOL),
])
def test_reduced_storage_against_oracle(storage, tol_u, tol_pos, tol_m, tol_f):
    cfg = I.config3_scaled(nx=40, ny=48, nz=36, storage=storage)
    sim = lbm().Simulation(cfg)
    ref = O.OracleSim(cfg)
    sim.step(60)
    ref.step(60)
    sim.sync()
    l2, pos, dm, ferr = errors_vs_oracle(sim, ref)
    print(f"{storage} vs FP64 oracle after 60 steps: velocity L2 rel {l2:.2e}, position max {pos:.2e} lu, "
          f"mass drift {dm:.2e}, force max rel {ferr:.2e}")
    assert l2 < tol_u and pos < tol_pos and dm < tol_m and ferr < tol_f


@pytest.mark.parametrize("case,nslabs", [("channel2d", 2), ("channel2d", 4), ("periodic2d", 3),
                                         ("channel3d", 3), ("periodic3d", 2), ("periodic3d", 4)])
def test_slabs_against_oracle(case, nslabs):
    """The whole decomposed step (per-slab eps, collision, halo exchange,
    shared particle sums, DEM) against the oracle's single lattice."""
    if case == "channel2d":
        cfg = I.channel_config(nx=80, ny=96, n_particles=8, radius=5.0)
    elif case == "periodic2d":
        cfg = I.periodic2d_config(nx=72, ny=90, phi=0.15, radius=4.0, seed=6, v0=0.02, density_ratio=5.0)
    elif case == "channel3d":
        cfg = I.config3_scaled(nx=24, ny=42, nz=20)
    else:
        cfg = I.periodic3d_config(nx=24, ny=40, nz=22, phi=0.1, radius=3.5, seed=4, v0=0.02)
    L = lbm()
    sl = L.Slabs(cfg, nslabs)
    ref = O.OracleSim(cfg)
    sl.step(200)
    ref.step(200)
    sl.sync()
    pe = rel_err(sl.populations(), ref.populations())
    ps, pr = sl.particles(), ref.particles()
    fe = force_err(ps, pr)
    print(f"{case}, {nslabs} slabs, 200 steps vs oracle: populations {pe:.2e}, forces {fe:.2e}")
    assert pe < POP_TOL
    assert fe < FORCE_TOL
    assert np.max(np.abs(ps["pos"] - pr["pos"])) < 1e-9


@pytest.mark.parametrize("storage", ["f64", "dfdev"])
def test_fixed_sphere_against_oracle(storage):
    """The validation's fixed sphere (R = 3, L = 24, density ratio 1e12, gas
    driven along x, tau = 1) for 300 steps: populations and the drag force
    at the parity tolerances, and the sphere stays put."""
    cfg = I.fixed_sphere_config(3.0, 0.008, tau=1.0, re_p=0.2, storage=storage)
    sim = lbm().Simulation(cfg)
    ref = O.OracleSim(cfg)
    sim.step(300)
    ref.step(300)
    sim.sync()
    assert rel_err(sim.populations(), ref.populations()) < POP_TOL
    pg, pr = sim.particles(), ref.particles()
    assert force_err(pg, pr) < FORCE_TOL
    assert pr["force"][0, 0] > 0.0  # the gas drags the sphere downstream
    assert np.max(np.abs(pg["pos"] - pr["pos"])) < 1e-13
    assert np.max(np.abs(pg["pos"] - cfg.pos)) < 1e-10  # held in place by its mass
