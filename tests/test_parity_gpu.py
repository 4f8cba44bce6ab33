"""GPU parity: the CUDA library (through its C ABI) against the FP64 CPU
oracle on the same seeded inputs.

Tolerances (FP64 storage): populations 1e-10 relative, particle forces 1e-9
relative to the largest force; the two sides differ only in rounding order
(FMA contraction in the collision, atomic summation of forces).  The FP64
deviation storage with double-FP32 arithmetic ("dfdev") is held to the same
tolerances: its 48-bit arithmetic on g = f - w rho0 is finer than FP64 on f.
"""
import math

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


def fluid_cfg(dim, nx, ny, nz=1, wall_y=0, tau=0.6, g=(0.0, 0.0, 0.0), storage="f64"):
    return I.SuspensionConfig(dim=dim, nx=nx, ny=ny, nz=nz if dim == 3 else 1, wall_y=wall_y, tau=tau,
                              body_force=np.asarray(g, dtype=float), gravity=np.zeros(3), rho_fluid=1.0,
                              k_n=1.0, restitution=0.9, dem_substeps=1, pos=np.zeros((0, 3)),
                              vel=np.zeros((0, 3)), omega=np.zeros((0, 3)), radius=np.zeros(0),
                              density=np.zeros(0), storage=storage)


def rel_err(a, b):
    return float(np.max(np.abs(a - b) / np.abs(b)))


def force_err(pg, pr, key="force"):
    scale = max(float(np.max(np.abs(pr[key]))), 1e-300)
    return float(np.max(np.abs(pg[key] - pr[key]))) / scale


def run_pair(cfg, steps, f0=None):
    gpu = lbm().Simulation(cfg)
    ref = O.OracleSim(cfg)
    if f0 is not None:
        gpu.set_populations(f0)
        ref.set_populations(f0)
    gpu.step(steps)
    ref.step(steps)
    gpu.sync()
    return gpu, ref


# ---------------------------------------------------------------------------
# fluid only (beta = 0): pull streaming, walls, body force
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("storage", ["f64", "dfdev"])
@pytest.mark.parametrize("dim,nx,ny,nz,wall", [(2, 37, 29, 1, 0), (2, 130, 64, 1, 1), (3, 19, 23, 17, 0),
                                               (3, 33, 20, 9, 1)])
def test_fluid_parity_nonequilibrium(dim, nx, ny, nz, wall, storage):
    """Ragged sizes (x not a multiple of the 32-wide warp or 128-wide CTA),
    non-equilibrium start, body force, periodic and wall boundaries."""
    cfg = fluid_cfg(dim, nx, ny, nz, wall_y=wall, tau=0.71, g=(3e-5, -2e-5, 1e-5 if dim == 3 else 0),
                    storage=storage)
    f0 = I.random_populations(np.random.default_rng(5), cfg)
    gpu, ref = run_pair(cfg, 25, f0)
    assert rel_err(gpu.populations(), ref.populations()) < POP_TOL
    rg, ug, _ = gpu.fields()
    rr, ur, _ = ref.fields()
    assert np.max(np.abs(rg - rr)) < 1e-12 and np.max(np.abs(ug - ur)) < 1e-12


def test_population_roundtrip_exact():
    cfg = fluid_cfg(3, 21, 10, 7)
    f0 = I.random_populations(np.random.default_rng(1), cfg)
    gpu = lbm().Simulation(cfg)
    gpu.set_populations(f0)
    assert np.array_equal(gpu.populations(), f0)


def test_population_roundtrip_dfdev():
    """f -> g = f - w rho0 -> FP32 pair (48 bits) -> f in FP64: g rounded
    to 48 bits, then one rounding of g and one of f."""
    cfg = fluid_cfg(3, 21, 10, 7, storage="dfdev")
    f0 = I.random_populations(np.random.default_rng(1), cfg)
    gpu = lbm().Simulation(cfg)
    gpu.set_populations(f0)
    w = np.array([1 / 3] + [1 / 18] * 6 + [1 / 36] * 12).reshape(19, 1, 1, 1)
    g = np.abs(f0 - w * cfg.rho_fluid)
    bound = 2.0 ** -48 * g + 2.0 ** -53 * (g + np.abs(f0))
    assert np.all(np.abs(gpu.populations() - f0) <= bound)


# ---------------------------------------------------------------------------
# eps rasterisation
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("storage", ["f64", "dfdev"])
@pytest.mark.parametrize("dim", [2, 3])
def test_eps_matches_exact_cell_fractions(dim, storage):
    """FP64 rasteriser (1e-12), and the pair-arithmetic one of the pair
    storage: its 48-bit angles enter corner terms of size R^3 (about 50)
    that cancel to the cell's volume, and 8 corners combine per cell; 32
    times FP64's error here is 2e-11, its bound."""
    rng = np.random.default_rng(11 + dim)
    if dim == 2:
        cfg = I.periodic2d_config(nx=96, ny=80, phi=0.2, radius=5.3, seed=4, density_ratio=3.0, storage=storage)
    else:
        cfg = I.periodic3d_config(nx=40, ny=36, nz=32, phi=0.15, radius=3.75, seed=4, storage=storage)
    gpu = lbm().Simulation(cfg)
    ref = O.OracleSim(cfg)
    _, _, eg = gpu.fields()
    _, _, er = ref.fields()
    err = float(np.max(np.abs(eg - er)))
    print(f"dim {dim} {storage}: max |eps - oracle| = {err:.2e}")
    assert err < (2e-11 if storage == "dfdev" else 1e-12)
    # covered volume: every particle's cells sum to its area/volume
    vol = (math.pi * cfg.radius ** 2) if dim == 2 else (4 / 3 * math.pi * cfg.radius ** 3)
    assert abs(eg.sum() - vol.sum()) < 1e-9 * vol.sum()
    del rng


@pytest.mark.parametrize("dim,R", [(3, 8.0), (3, 6.0), (2, 29.0), (2, 16.0)])
def test_pair_rasteriser_at_largest_radii(dim, R):
    """The pair storage's rasteriser at the largest radii the library
    accepts (3D R = 8, 2D R = 29) and between.  Its
    error comes from 48-bit angles in corner terms of size R^dim that cancel
    to a cell's area or volume, so the bound grows like R^dim from the
    2e-11 of R = 3.75 (3D) and R = 5.3 (2D).  A short coupled run at the same
    radius stays within the population and force tolerances."""
    R0 = 3.75 if dim == 3 else 5.3
    bound = 2e-11 * max(1.0, (R / R0) ** dim)
    if dim == 3:
        cfg = I.periodic3d_config(nx=48, ny=44, nz=40, phi=0.12, radius=R, seed=5, v0=0.01, storage="dfdev")
    else:
        cfg = I.periodic2d_config(nx=160, ny=150, phi=0.2, radius=R, seed=5, v0=0.01, density_ratio=3.0,
                                  storage="dfdev")
    gpu = lbm().Simulation(cfg)
    ref = O.OracleSim(cfg)
    _, _, eg = gpu.fields()
    _, _, er = ref.fields()
    err = float(np.max(np.abs(eg - er)))
    print(f"pair rasteriser, dim {dim}, R = {R}: max |eps - oracle| = {err:.2e} (bound {bound:.1e})")
    assert err < bound
    gpu.step(30)
    ref.step(30)
    gpu.sync()
    assert rel_err(gpu.populations(), ref.populations()) < POP_TOL
    pg, pr = gpu.particles(), ref.particles()
    assert force_err(pg, pr) < FORCE_TOL


def test_eps_two_owner_cells_and_wrap():
    """Disks 0.1 lu apart share cells; one straddles the periodic seam."""
    cfg = I.SuspensionConfig(dim=2, nx=40, ny=32, nz=1, wall_y=0, tau=0.8, body_force=np.zeros(3),
                             gravity=np.zeros(3), rho_fluid=1.0, k_n=10.0, restitution=0.9, dem_substeps=1,
                             pos=np.array([[8.0, 12.0, 0], [14.5, 12.3, 0], [0.4, 25.7, 0]]),
                             vel=np.zeros((3, 3)), omega=np.zeros((3, 3)), radius=np.array([3.2, 3.2, 4.1]),
                             density=np.full(3, 5.0))
    gpu = lbm().Simulation(cfg)
    ref = O.OracleSim(cfg)
    _, _, eg = gpu.fields()
    _, _, er = ref.fields()
    assert np.max(np.abs(eg - er)) < 1e-13
    assert ref.owners()[0].max() == 2


# ---------------------------------------------------------------------------
# coupled LB-IMB-DEM
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("storage", ["f64", "dfdev"])
def test_config1_1000_steps(storage):
    """D2Q9 128x256 channel, 20 disks R=6, density ratio 10, g=1e-6,
    1000 steps from rest: the parity target."""
    cfg = I.config1().replace(storage=storage)
    gpu, ref = run_pair(cfg, 1000)
    pe = rel_err(gpu.populations(), ref.populations())
    pg, pr = gpu.particles(), ref.particles()
    print(f"config 1, {storage}, 1000 steps: populations max rel {pe:.2e}, forces {force_err(pg, pr):.2e}, "
          f"positions max {np.max(np.abs(pg['pos'] - pr['pos'])):.2e} lu")
    assert pe < POP_TOL
    assert force_err(pg, pr) < FORCE_TOL
    assert force_err(pg, pr, "torque") < FORCE_TOL or np.max(np.abs(pr["torque"])) < 1e-14
    assert np.max(np.abs(pg["pos"] - pr["pos"])) < 1e-9
    assert np.max(np.abs(pg["vel"] - pr["vel"])) < 1e-12


@pytest.mark.parametrize("storage", ["f64", "dfdev"])
def test_periodic_2d_moving_particles_with_contacts(storage):
    """Fast disks in a dense periodic box collide within the run."""
    cfg = I.periodic2d_config(nx=100, ny=72, phi=0.25, radius=4.0, seed=9, v0=0.03, density_ratio=4.0,
                              storage=storage)
    gpu, ref = run_pair(cfg, 150)
    pg, pr = gpu.particles(), ref.particles()
    assert rel_err(gpu.populations(), ref.populations()) < POP_TOL
    assert force_err(pg, pr) < FORCE_TOL
    assert np.max(np.abs(pg["pos"] - pr["pos"])) < 1e-9


@pytest.mark.parametrize("storage", ["f64", "dfdev"])
def test_spinning_particles_torque_3d(storage):
    cfg = I.periodic3d_config(nx=28, ny=30, nz=26, phi=0.1, radius=3.75, seed=3, v0=0.01, storage=storage)
    cfg.omega = 0.003 * np.random.default_rng(2).standard_normal((cfg.n_particles, 3))
    gpu, ref = run_pair(cfg, 40)
    pg, pr = gpu.particles(), ref.particles()
    assert rel_err(gpu.populations(), ref.populations()) < POP_TOL
    assert force_err(pg, pr) < FORCE_TOL
    assert force_err(pg, pr, "torque") < FORCE_TOL
    assert np.max(np.abs(pg["omega"] - pr["omega"])) < 1e-12


@pytest.mark.parametrize("storage,form", [("f64", 0), ("dfdev", 0), ("dfdev", 6), ("dfdev", 7), ("dfdev", 8),
                                          ("dfdev", 9)])
def test_config3_shape_channel_3d(storage, form):
    """Cut-down config 3 (D3Q19, walls in y, spheres R=3.75, ratio 1000)."""
    cfg = I.config3_scaled(nx=40, ny=48, nz=36, storage=storage)
    gpu = lbm().Simulation(cfg)
    gpu.set_collide_variant(form)
    ref = O.OracleSim(cfg)
    gpu.step(30)
    ref.step(30)
    gpu.sync()
    pg, pr = gpu.particles(), ref.particles()
    assert rel_err(gpu.populations(), ref.populations()) < POP_TOL
    assert force_err(pg, pr) < FORCE_TOL
    assert force_err(pg, pr, "torque") < FORCE_TOL


def test_momentum_conserved_on_gpu():
    cfg = I.periodic3d_config(nx=24, ny=24, nz=24, phi=0.12, radius=3.0, seed=8, v0=0.02, gs=0.0)
    gpu = lbm().Simulation(cfg)
    m0, j0, p0 = gpu.totals()
    gpu.step(20)
    m1, j1, p1 = gpu.totals()
    scale = np.abs(p0).sum() + 1e-300
    assert abs(m1 - m0) < 1e-12 * m0
    assert np.max(np.abs((j1 + p1) - (j0 + p0))) < 1e-11 * max(scale, 1.0)


def test_error_on_too_many_owners():
    """Four particles stacked on one point exceed nothing; five do."""
    pos = np.tile([[10.0, 10.0, 0.0]], (5, 1)) + np.array([[0, 0, 0], [0.01, 0, 0], [0, 0.01, 0],
                                                            [0.01, 0.01, 0], [0.02, 0, 0]])
    cfg = I.SuspensionConfig(dim=2, nx=24, ny=24, nz=1, wall_y=0, tau=0.8, body_force=np.zeros(3),
                             gravity=np.zeros(3), rho_fluid=1.0, k_n=10.0, restitution=0.9, dem_substeps=1,
                             pos=pos, vel=np.zeros((5, 3)), omega=np.zeros((5, 3)), radius=np.full(5, 2.0),
                             density=np.full(5, 2.0))
    L = lbm()
    with pytest.raises(L.LbmImbError) as ei:
        L.Simulation(cfg)
    assert ei.value.status == L.EOWNERS
    L.Simulation(cfg.replace(pos=pos[:4], vel=np.zeros((4, 3)), omega=np.zeros((4, 3)),
                             radius=np.full(4, 2.0), density=np.full(4, 2.0)))


# ---------------------------------------------------------------------------
# reduced-precision storage: error reported against FP64, bounded loosely
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("storage,tol_u,tol_f", [("f32dev", 1e-4, 1e-3), ("f16dev", 3e-2, 3e-2)])
def test_reduced_storage_error(storage, tol_u, tol_f):
    cfg = I.config3_scaled(nx=40, ny=48, nz=36)
    ref = lbm().Simulation(cfg)
    red = lbm().Simulation(cfg.replace(storage=storage))
    ref.step(40)
    red.step(40)
    _, u64, _ = ref.fields()
    _, ulo, _ = red.fields()
    l2 = float(np.linalg.norm(ulo - u64) / np.linalg.norm(u64))
    p64, plo = ref.particles(), red.particles()
    ferr = force_err(plo, p64)
    m64 = ref.totals()[0]
    mlo = red.totals()[0]
    print(f"{storage}: velocity L2 rel {l2:.2e}, force rel {ferr:.2e}, mass drift {abs(mlo - m64) / m64:.2e}")
    assert l2 < tol_u and ferr < tol_f and abs(mlo - m64) / m64 < 1e-5


# ---------------------------------------------------------------------------
# kernel forms of the plain collision: the same populations
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("storage", ["f64", "f32dev", "f16dev", "dfdev"])
@pytest.mark.parametrize("dim", [2, 3])
def test_collide_variants_agree(dim, storage):
    """Every kernel form gives bitwise the populations of form 0 after one
    step (nx = 300 spans ragged row tiles), and the FP64 forms stay within
    the oracle tolerance after 12 steps.  Forms 7, 8 and 9 of the pair
    storage update covered nodes in pair arithmetic instead of FP64: within
    1e-14 there."""
    if dim == 3:
        cfg = I.config3_scaled(nx=300, ny=20, nz=12).replace(storage=storage)
    else:
        cfg = I.channel_config(nx=300, ny=64, n_particles=12, radius=5.0, storage=storage)
    L = lbm()
    base = L.Simulation(cfg)
    base.step(1)
    f_base = base.populations()
    for var in (1, 2, 3, 4, 5, 6, 7, 8, 9):
        sim = L.Simulation(cfg)
        sim.set_collide_variant(var)
        sim.step(1)
        if storage == "dfdev" and var in (7, 8, 9):
            assert rel_err(sim.populations(), f_base) < 1e-14, f"variant {var}"
        else:
            assert np.array_equal(sim.populations(), f_base), f"variant {var}"
        if storage in ("f64", "dfdev"):
            ref = O.OracleSim(cfg)
            ref.step(12)
            sim.step(11)
            assert rel_err(sim.populations(), ref.populations()) < POP_TOL, f"variant {var}"
    with pytest.raises(L.LbmImbError):
        base.set_collide_variant(10)


@pytest.mark.parametrize("nx", [300, 131, 64])
@pytest.mark.parametrize("dim", [2, 3])
def test_pair_storage_two_node_plain_part_is_bitwise(dim, nx):
    """Form 8 of the pair storage (plain part two nodes per thread in paired
    FP32 instructions) gives bitwise the populations of form 7 (one node per
    thread) after a step: the paired instructions round every lane on its
    own.  Odd and even row lengths, walls in y, random populations.  Later
    steps differ in the order of the force atomics (and so in the
    particles' last bits and, through the rasteriser's pair arithmetic, in
    the covered fractions' rounding); from the configuration's start both
    forms stay within the parity tolerance of the oracle."""
    if dim == 3:
        cfg = I.config3_scaled(nx=nx, ny=20, nz=12).replace(storage="dfdev")
    else:
        cfg = I.channel_config(nx=nx, ny=64, n_particles=6, radius=5.0, storage="dfdev")
    L = lbm()
    a = L.Simulation(cfg)
    a.set_collide_variant(7)
    b = L.Simulation(cfg)
    b.set_collide_variant(8)
    f0 = I.random_populations(np.random.default_rng(4), cfg)
    a.set_populations(f0)
    b.set_populations(f0)
    a.step(1)
    b.step(1)
    assert np.array_equal(a.populations(), b.populations())
    # from the configuration's own start (near equilibrium, where the pair
    # storage's deviations are small), 12 steps beside the oracle
    a, b = L.Simulation(cfg), L.Simulation(cfg)
    a.set_collide_variant(7)
    b.set_collide_variant(8)
    ref = O.OracleSim(cfg)
    ref.step(12)
    a.step(12)
    b.step(12)
    ea, eb = rel_err(a.populations(), ref.populations()), rel_err(b.populations(), ref.populations())
    print(f"dim {dim} nx {nx}: 12 steps vs oracle, form 7 {ea:.2e}, form 8 {eb:.2e}, "
          f"between them {rel_err(b.populations(), a.populations()):.2e}")
    assert ea < POP_TOL and eb < POP_TOL


@pytest.mark.parametrize("storage", ["f32dev", "f16dev"])
@pytest.mark.parametrize("dim", [2, 3])
def test_pair_form_odd_row_length(dim, storage):
    """The two-node form with an odd row length (a lone last node per row,
    and the x wrap inside a pair) gives the populations of form 0."""
    if dim == 3:
        cfg = I.config3_scaled(nx=131, ny=20, nz=12).replace(storage=storage)
    else:
        cfg = I.channel_config(nx=131, ny=64, n_particles=6, radius=5.0, storage=storage)
    L = lbm()
    base = L.Simulation(cfg)
    base.step(1)
    f1 = base.populations()
    base.step(2)
    f3 = base.populations()
    for var in (8, 9):
        sim = L.Simulation(cfg)
        sim.set_collide_variant(var)
        sim.step(1)
        assert np.array_equal(sim.populations(), f1), f"variant {var}"
        # later steps see particles moved by forces summed in another atomic order
        sim.step(2)
        assert np.allclose(sim.populations(), f3, rtol=1e-5, atol=0), f"variant {var}"
