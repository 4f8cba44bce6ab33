"""The C ABI's state calls on the GPU: checkpoint / resume (lbm_imb_save,
lbm_imb_load), the health check (LBM_IMB_ENONFINITE) and the host-side
validation of lbm_imb_set_particles.  NaN values go only into the
populations of a particle-free lattice; no NaN particle is ever uploaded
(the host check rejects it before any copy)."""
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


def fluid_cfg(dim=3, nx=21, ny=18, nz=13, wall_y=1, storage="f64"):
    return I.SuspensionConfig(dim=dim, nx=nx, ny=ny, nz=nz if dim == 3 else 1, wall_y=wall_y, tau=0.7,
                              body_force=np.array([2e-5, -1e-5, 0.0]), gravity=np.zeros(3), rho_fluid=1.0,
                              k_n=1.0, restitution=0.9, dem_substeps=1, pos=np.zeros((0, 3)),
                              vel=np.zeros((0, 3)), omega=np.zeros((0, 3)), radius=np.zeros(0),
                              density=np.zeros(0), storage=storage)


# ---------------------------------------------------------------------------
# checkpoint / resume
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("storage", ["f64", "dfdev", "f16dev"])
def test_resume_of_fluid_run_is_bitwise(tmp_path, storage):
    """Without particles no atomics are involved: 40 + save/load + 40 steps
    equal 80 straight steps bit for bit, in every storage (the file holds
    the raw stored values)."""
    L = lbm()
    cfg = fluid_cfg(storage=storage)
    f0 = I.random_populations(np.random.default_rng(3), cfg)
    a = L.Simulation(cfg)
    a.set_populations(f0)
    a.step(80)
    b = L.Simulation(cfg)
    b.set_populations(f0)
    b.step(40)
    path = str(tmp_path / "fluid.ckpt")
    b.save(path)
    b.close()
    c = L.Simulation(cfg)
    c.load(path)
    assert c.steps_done() == 40
    c.step(40)
    assert c.steps_done() == 80
    assert np.array_equal(c.populations(), a.populations())


@pytest.mark.parametrize("skin", [0.0, 1.5])
def test_config1_500_plus_500_equals_1000(tmp_path, skin):
    """Config 1 (20 disks in a channel): 500 steps, save, a new simulation
    loads the file and runs 500 more; the result equals a straight 1000-step
    run within the order of the FP64 force atomics, and both stay within
    the oracle's parity tolerance.  With Verlet lists (skin > 0) the loaded
    simulation rebuilds its lists from the loaded positions."""
    L = lbm()
    cfg = I.config1().replace(dem_skin=skin)
    straight = L.Simulation(cfg)
    straight.step(1000)
    first = L.Simulation(cfg)
    first.step(500)
    path = str(tmp_path / "cfg1.ckpt")
    first.save(path)
    p_saved = first.particles()
    first.close()
    second = L.Simulation(cfg)
    second.load(path)
    p_loaded = second.particles()
    for k in ("pos", "vel", "omega", "force", "torque"):
        assert np.array_equal(p_loaded[k], p_saved[k]), k
    second.step(500)
    ref = O.OracleSim(cfg)
    ref.step(1000)
    fs, fr, fo = straight.populations(), second.populations(), ref.populations()
    assert rel_err(fr, fs) < 1e-12
    assert rel_err(fr, fo) < POP_TOL
    ps, pr, po = straight.particles(), second.particles(), ref.particles()
    assert force_err(pr, ps) < 1e-10
    assert force_err(pr, po) < FORCE_TOL
    assert np.max(np.abs(pr["pos"] - po["pos"])) < 1e-9


def test_load_rejects_other_configuration_and_batches(tmp_path):
    L = lbm()
    cfg = fluid_cfg()
    a = L.Simulation(cfg)
    a.step(3)
    path = str(tmp_path / "a.ckpt")
    a.save(path)
    f_before = a.populations()
    other = L.Simulation(cfg.replace(tau=0.71))  # same sizes, other physics: another hash
    with pytest.raises(L.LbmImbError) as ei:
        other.load(path)
    assert ei.value.status == L.EINVAL
    assert other.steps_done() == 0
    with pytest.raises(L.LbmImbError) as ei:
        a.load(str(tmp_path / "missing.ckpt"))
    assert ei.value.status == L.EINVAL
    assert np.array_equal(a.populations(), f_before)
    junk = tmp_path / "junk.ckpt"
    junk.write_bytes(b"not a checkpoint" * 8)
    with pytest.raises(L.LbmImbError) as ei:
        a.load(str(junk))
    assert ei.value.status == L.EINVAL
    batch = L.Batch([I.channel_config(nx=64, ny=64, n_particles=2, radius=4.0)])
    with pytest.raises(L.LbmImbError) as ei:
        L._check(L.lib().lbm_imb_save(batch.h, path.encode()), "lbm_imb_save")
    assert ei.value.status == L.EUNSUPPORTED


# ---------------------------------------------------------------------------
# health check
# ---------------------------------------------------------------------------
def test_nan_population_reported_by_health_check():
    """A NaN written into one moving population of a particle-free lattice
    reaches the rest direction of the node that pulls it after one step; the
    periodic check of step() then reports it at the next synchronising call,
    and an explicit check does too."""
    L = lbm()
    cfg = fluid_cfg(dim=2, nx=40, ny=30, nz=1, wall_y=0)
    sim = L.Simulation(cfg)
    sim.step(2)
    sim.sync()
    sim.check_health()  # clean state: no error
    f = sim.populations()
    f[3, 0, 11, 17] = np.nan  # direction (0, 1), node (17, 11)
    sim.set_populations(f)
    sim.set_health_check(1)
    sim.step(1)
    with pytest.raises(L.LbmImbError) as ei:
        sim.sync()
    assert ei.value.status == L.ENONFINITE
    with pytest.raises(L.LbmImbError) as ei:
        sim.check_health()
    assert ei.value.status == L.ENONFINITE
    # the NaN spread to the node that pulled it (17, 12), through its density
    assert np.isnan(sim.populations()[0, 0, 12, 17])


def test_health_check_interval_and_off():
    L = lbm()
    cfg = fluid_cfg(dim=3, nx=16, ny=12, nz=10, wall_y=0)
    sim = L.Simulation(cfg)
    f = sim.populations()
    f[7, 4, 5, 6] = np.inf
    sim.set_populations(f)
    sim.set_health_check(0)
    sim.step(3)
    sim.sync()  # no check ran: nothing reported
    with pytest.raises(L.LbmImbError) as ei:
        sim.check_health()
    assert ei.value.status == L.ENONFINITE
    sim2 = L.Simulation(cfg)
    sim2.set_populations(f)
    sim2.set_health_check(4)  # runs after steps 4, 8, ...
    sim2.step(3)
    sim2.sync()
    sim2.step(1)
    with pytest.raises(L.LbmImbError) as ei:
        sim2.sync()
    assert ei.value.status == L.ENONFINITE


def test_clean_runs_pass_health_checks():
    """The default check (every 100 steps) stays silent on a healthy coupled
    run with particles, in every storage."""
    L = lbm()
    for storage in ("f64", "f32dev", "f16dev", "dfdev"):
        sim = L.Simulation(I.config3_scaled(nx=32, ny=40, nz=28, storage=storage))
        sim.step(200)
        sim.sync()
        sim.check_health()


# ---------------------------------------------------------------------------
# lbm_imb_set_particles: host validation
# ---------------------------------------------------------------------------
def test_set_particles_rejects_bad_state_on_the_host():
    L = lbm()
    cfg = I.config1()
    sim = L.Simulation(cfg)
    sim.step(5)
    p0 = sim.particles()
    bad_cases = []
    pos = p0["pos"].copy()
    pos[3, 0] = np.nan
    bad_cases.append(dict(pos=pos))
    pos = p0["pos"].copy()
    pos[0, 1] = cfg.ny - 0.4  # beyond the upper wall at ny - 1/2
    bad_cases.append(dict(pos=pos))
    pos = p0["pos"].copy()
    pos[1, 1] = -0.6  # below the lower wall
    bad_cases.append(dict(pos=pos))
    pos = p0["pos"].copy()
    pos[2, 0] = cfg.nx + 0.1  # beyond [-1/2, nx) along the periodic x
    bad_cases.append(dict(pos=pos))
    pos = p0["pos"].copy()
    pos[2, 0] = -0.6
    bad_cases.append(dict(pos=pos))
    vel = p0["vel"].copy()
    vel[5, 1] = np.inf
    bad_cases.append(dict(vel=vel))
    om = p0["omega"].copy()
    om[6, 2] = np.nan
    bad_cases.append(dict(omega=om))
    for kw in bad_cases:
        with pytest.raises(L.LbmImbError) as ei:
            sim.set_particles(**kw)
        assert ei.value.status == L.EINVAL, kw.keys()
    p1 = sim.particles()
    for k in ("pos", "vel", "omega"):
        assert np.array_equal(p1[k], p0[k])  # nothing was copied
    # a centre in [-1/2, 0) along the periodic x is accepted (the DEM wraps it)
    pos = p0["pos"].copy()
    pos[0, 0] = -0.3
    sim.set_particles(pos=pos)
    sim.step(1)
    sim.sync()
    assert 0.0 <= sim.particles()["pos"][0, 0] < cfg.nx


def test_init_rejects_nonfinite_particles():
    L = lbm()
    cfg = I.config1()
    vel = cfg.vel.copy()
    vel[0, 0] = np.nan
    with pytest.raises(L.LbmImbError) as ei:
        L.Simulation(cfg.replace(vel=vel))
    assert ei.value.status == L.EINVAL
    pos = cfg.pos.copy()
    pos[0, 1] = -3.0
    with pytest.raises(L.LbmImbError) as ei:
        L.Simulation(cfg.replace(pos=pos))
    assert ei.value.status == L.EINVAL
