"""Pins for the oracle's DEM (Eqs. 4-5 with the garbles read as the standard
frictionless linear spring-dashpot) and for the parameter set of Table 2."""
import json
import math
import os

import numpy as np
import pytest

from oracle import oracle as O
from paper_1011_2613_gb300 import inputs as I

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "table2_parameters.json")))


def head_on(m, k, e, substeps, R=5.0, v=0.01, dim=3):
    """Two equal particles approaching along x in vacuum; returns the
    restitution measured from the relative velocity, the contact duration
    in steps and the momentum drift."""
    L = [200, 200, 200]
    pos = np.array([[100.0 - R - 0.05, 50.0, 50.0], [100.0 + R + 0.05, 50.0, 50.0]])
    vel = np.array([[v, 0.0, 0.0], [-v, 0.0, 0.0]])
    if dim == 2:
        pos[:, 2] = 0
    omg = np.zeros((2, 3))
    z = np.zeros(6)
    mass = np.array([m, m])
    inertia = 0.4 * mass * R * R
    p0 = (mass[:, None] * vel).sum(axis=0)
    in_contact = 0
    started = False
    for step in range(400):
        fc = O.dem_advance(dim, L[:dim], 0, pos, vel, omg, [R, R], mass, inertia, z, z, np.zeros(3), k, e, substeps)
        touching = np.linalg.norm(pos[0] - pos[1]) < 2 * R
        if touching:
            started = True
        if started:
            in_contact += 1  # counts steps that end while overlapping, plus the exit step
            if not touching:
                break
    vr = vel[0, 0] - vel[1, 0]
    drift = np.abs((mass[:, None] * vel).sum(axis=0) - p0).max()
    return -vr / (2 * v), in_contact, drift


def test_table2_masses_follow_solid_density():
    """m = rho_s pi R^2 (2D, unit depth) and rho_s (4/3) pi R^3 (3D) with
    rho_s = 900/1.3 reproduce the printed 54373 and 362491."""
    rs = GOLD["rho_solid_dimensional"] / GOLD["rho_gas_dimensional"]
    R = GOLD["diameter"] / 2
    cfg2 = I.SuspensionConfig(dim=2, nx=32, ny=32, nz=1, wall_y=0, tau=0.8, body_force=np.zeros(3),
                              gravity=np.zeros(3), rho_fluid=1.0, k_n=1.0, restitution=0.9, dem_substeps=1,
                              pos=np.array([[16.0, 16.0, 0]]), vel=np.zeros((1, 3)), omega=np.zeros((1, 3)),
                              radius=np.array([R]), density=np.array([rs]))
    m2, _ = O.OracleSim(cfg2).masses()
    cfg3 = cfg2.replace(dim=3, nz=32, pos=np.array([[16.0, 16.0, 16.0]]))
    m3, _ = O.OracleSim(cfg3).masses()
    assert abs(m2[0] - GOLD["mass_2d_printed"]) < 1.0
    assert abs(m3[0] - GOLD["mass_3d_printed"]) < 1.0
    assert abs(rs - GOLD["rho_solid_printed"]) < 0.01


@pytest.mark.parametrize("case", ["2d", "3d"])
def test_table2_stiffness_gives_ten_step_contact(case):
    """With the printed k_n, m and e = 0.9 the converged (many sub-steps)
    head-on collision lasts t_c = 10 steps and restitutes e; the stiffness
    derived from t_c = 10 reproduces the printed k_n."""
    m = GOLD["mass_%s_printed" % case]
    k = GOLD["k_n_%s_printed" % case]
    e = GOLD["restitution"]
    assert abs(I.stiffness_for_contact_time(m / 2, e, 10.0) - k) / k < 2e-3
    omega_d = math.sqrt(k / (m / 2)) * math.pi / math.sqrt(math.pi ** 2 + math.log(e) ** 2)
    assert abs(math.pi / omega_d - 10.0) < 0.01
    er, steps, drift = head_on(m, k, e, substeps=64)
    assert abs(er - e) < 2e-3
    assert 10 <= steps <= 12
    assert drift < 1e-15 * m * 0.01


def test_restitution_converges_with_substeps():
    m, e = 54373.0, 0.9
    k = I.stiffness_for_contact_time(m / 2, e)
    errs = [abs(head_on(m, k, e, s)[0] - e) for s in (1, 4, 16, 64)]
    assert errs[0] < 0.05
    assert errs[-1] < 2e-3
    assert errs[3] < errs[1] < errs[0] or errs[3] < 1e-3
    # kinetic energy ratio ~ e^2
    er = head_on(m, k, e, 64)[0]
    assert abs(er ** 2 - e ** 2) < 4e-3


def test_elastic_limit():
    m = 1000.0
    k = I.stiffness_for_contact_time(m / 2, 1.0)
    er, _, _ = head_on(m, k, 1.0, 64)
    assert abs(er - 1.0) < 2e-3


def test_overlap_repels_and_wall_bounces():
    m, R, e = 500.0, 3.0, 0.9
    k = I.stiffness_for_contact_time(m / 2, e)
    pos = np.array([[10.0, 20.0, 0.0], [15.5, 20.0, 0.0]])  # overlap 0.5
    vel = np.zeros((2, 3))
    z = np.zeros(6)
    fc = O.dem_advance(2, [40, 40], 0, pos, vel, np.zeros((2, 3)), [R, R], [m, m], [1.0, 1.0], z, z,
                       np.zeros(3), k, e)
    assert fc[0, 0] < 0 < fc[1, 0] and vel[0, 0] < 0 < vel[1, 0]
    # particle falling onto the bottom wall (y = -1/2) rebounds with ~e
    pos = np.array([[10.0, R + 0.5 + 0.02, 0.0]])
    vel = np.array([[0.0, -0.01, 0.0]])
    for _ in range(200):
        O.dem_advance(2, [40, 40], 1, pos, vel, np.zeros((1, 3)), [R], [m], [1.0], z[:3], z[:3], np.zeros(3),
                      k / 2, e, 64)
        if vel[0, 1] > 0 and pos[0, 1] > R + 0.5:
            break
    assert abs(vel[0, 1] / 0.01 - e) < 3e-3


def test_free_fall_is_symplectic_euler():
    pos = np.array([[5.0, 5.0, 5.0]])
    vel = np.array([[0.001, 0.0, 0.0]])
    g = np.array([0.0, -1e-4, 0.0])
    z = np.zeros(3)
    O.dem_advance(3, [20, 20, 20], 0, pos, vel, np.zeros((1, 3)), [1.0], [2.0], [1.0], z, z, g, 1.0, 0.9)
    assert vel[0, 1] == -1e-4 and pos[0, 1] == 5.0 - 1e-4 and pos[0, 0] == 5.001
