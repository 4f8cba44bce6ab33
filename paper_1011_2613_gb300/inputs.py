"""Seeded synthetic suspensions shaped like the paper's workloads.

This module only draws inputs (lattice sizes, particle positions, radii,
densities, initial velocities) and derives the physical parameters the paper
fixes through its unit conversion (Table 2).  It holds none of the method's
arithmetic, so both the CUDA library and the CPU oracle can be fed from it.

Parameter derivations (Table 2 and the section "Simulation results"):

* contact stiffness from the contact duration: the expression the paper prints
  as eta_n in Eq. (5) evaluates to the contact time t_c (10.00 time steps for
  both of its parameter sets), so k_n = m* (pi^2 + ln^2 e) / t_c^2 with
  m* = m/2 for a pair of equal particles.  With m = 54373, e = 0.9 this gives
  2686, the printed 2D value.
* a periodic gravity-driven suspension balances the particles' weight by a body
  force on the gas: g_f = -g_s sum_p m_p / (rho_f N_nodes).
* with walls the gas feels the same gravity as the particles (g_f = g_s) and
  the walls carry the load.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Optional

import numpy as np

STORAGE = {"f64": 0, "f32dev": 1, "f16dev": 2, "dfdev": 3}


@dataclasses.dataclass
class SuspensionConfig:
    dim: int
    nx: int
    ny: int
    nz: int
    wall_y: int
    tau: float
    body_force: np.ndarray  # (3,) fluid acceleration g_f
    gravity: np.ndarray  # (3,) particle acceleration g_s
    rho_fluid: float
    k_n: float
    restitution: float
    dem_substeps: int
    pos: np.ndarray  # (np,3)
    vel: np.ndarray  # (np,3)
    omega: np.ndarray  # (np,3)
    radius: np.ndarray  # (np,)
    density: np.ndarray  # (np,) solid density in lattice units
    storage: str = "f64"
    name: str = ""
    eps_method: int = 0  # 0 exact covered fractions, 1 the table lookup of Eq. 6
    dem_skin: float = 0.0  # 0 cell list every step, > 0 Verlet lists with this skin

    @property
    def n_nodes(self) -> int:
        return self.nx * self.ny * (self.nz if self.dim == 3 else 1)

    @property
    def n_particles(self) -> int:
        return int(len(self.radius))

    def masses(self) -> np.ndarray:
        r = np.asarray(self.radius, dtype=np.float64)
        if self.dim == 2:
            return np.asarray(self.density) * math.pi * r * r
        return np.asarray(self.density) * (4.0 / 3.0) * math.pi * r ** 3

    def replace(self, **kw) -> "SuspensionConfig":
        return dataclasses.replace(self, **kw)


def stiffness_for_contact_time(m_pair: float, e: float, t_c: float = 10.0) -> float:
    """k_n such that a spring-dashpot pair of reduced mass m_pair stays in
    contact for t_c lattice steps (the paper's choice, Table 2)."""
    le = math.log(e)
    return m_pair * (math.pi ** 2 + le * le) / (t_c * t_c)


def random_directions(rng: np.random.Generator, n: int, dim: int) -> np.ndarray:
    v = rng.standard_normal((n, 3))
    if dim == 2:
        v[:, 2] = 0.0
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    return v


def rsa_place(rng: np.random.Generator, radii: np.ndarray, box, dim: int, periodic,
              gap: float = 1.0, wall_gap: float = 1.0, max_tries: int = 500) -> np.ndarray:
    """Random sequential addition of non-overlapping disks/spheres, largest
    first.

    ``box`` = (nx, ny, nz) in lattice units (node i sits at coordinate i; the
    domain spans [-1/2, n-1/2) along each axis; periodic axes wrap [0, n)).
    Surfaces keep at least ``gap`` from each other and ``wall_gap`` from a
    non-periodic boundary.  An occupancy grid with cells small enough to hold
    at most one centre makes each trial a fixed-size neighbourhood lookup.
    Returns positions (n,3); raises if a particle cannot be placed.
    """
    radii = np.asarray(radii, dtype=np.float64)
    n = len(radii)
    pos = np.zeros((n, 3))
    if n == 0:
        return pos
    L = np.array([box[0], box[1], box[2] if dim == 3 else 1], dtype=np.float64)[:dim]
    per = np.array(list(periodic)[:dim], dtype=bool)
    rmin, rmax = float(radii.min()), float(radii.max())
    h = (2.0 * rmin + gap) / math.sqrt(dim) * 0.999  # at most one centre per cell
    ncell = np.maximum(1, np.floor(L / h).astype(int))
    h = L / ncell
    reach = int(math.ceil((2.0 * rmax + gap) / h.min()))
    grid = -np.ones(tuple(ncell), dtype=np.int64)
    offs = np.array(np.meshgrid(*([np.arange(-reach, reach + 1)] * dim), indexing="ij")).reshape(dim, -1).T
    origin = np.where(per, 0.0, -0.5)
    order = np.argsort(-radii, kind="stable")
    for idx in order:
        R = radii[idx]
        lo = np.where(per, 0.0, -0.5 + R + wall_gap)
        hi = np.where(per, L, L - 0.5 - R - wall_gap)
        if np.any(hi <= lo):
            raise RuntimeError("particle does not fit between the walls")
        placed = False
        for _ in range(max_tries):
            p = lo + rng.random(dim) * (hi - lo)
            c = np.minimum(((p - origin) / h).astype(int), ncell - 1)
            cc = c + offs
            ok_rows = np.ones(len(cc), dtype=bool)
            for d in range(dim):
                if per[d]:
                    cc[:, d] %= ncell[d]
                else:
                    ok_rows &= (cc[:, d] >= 0) & (cc[:, d] < ncell[d])
            cc = cc[ok_rows]
            if grid[tuple(cc.T)].max() >= 0:
                js = grid[tuple(cc.T)]
                js = js[js >= 0]
                dv = pos[js, :dim] - p
                for d in range(dim):
                    if per[d]:
                        dv[:, d] -= L[d] * np.round(dv[:, d] / L[d])
                if np.any((dv * dv).sum(axis=1) < (R + radii[js] + gap) ** 2):
                    continue
            if grid[tuple(c)] >= 0:
                continue  # cell taken (cannot happen with valid spacing)
            pos[idx, :dim] = p
            grid[tuple(c)] = idx
            placed = True
            break
        if not placed:
            raise RuntimeError("random sequential addition did not converge")
    return pos


def _finish(dim, nx, ny, nz, wall_y, tau, gs, rho_f, e, radius, density, pos, vel, name,
            k_n=None, storage="f64", balance=True, substeps=1):
    n = len(radius)
    cfg = SuspensionConfig(
        dim=dim, nx=nx, ny=ny, nz=nz if dim == 3 else 1, wall_y=wall_y, tau=tau,
        body_force=np.zeros(3), gravity=np.asarray(gs, dtype=np.float64), rho_fluid=rho_f,
        k_n=0.0, restitution=e, dem_substeps=substeps, pos=pos, vel=vel, omega=np.zeros((n, 3)),
        radius=np.asarray(radius, dtype=np.float64), density=np.asarray(density, dtype=np.float64),
        storage=storage, name=name)
    m = cfg.masses()
    if k_n is None:
        k_n = stiffness_for_contact_time(float(np.max(m)) / 2.0 if n else 1.0, e)
    cfg.k_n = float(k_n)
    if wall_y:
        cfg.body_force = np.asarray(gs, dtype=np.float64).copy()
    elif balance and n:
        cfg.body_force = -np.asarray(gs, dtype=np.float64) * float(m.sum()) / (rho_f * cfg.n_nodes)
    return cfg


def channel_config(nx=128, ny=256, n_particles=20, radius=6.0, density_ratio=10.0, g=1e-6, tau=0.6,
                   seed=1, e=0.9, storage="f64", name="D2Q9 channel") -> SuspensionConfig:
    """2D channel suspension: periodic in x, walls in y, gravity -y on both
    phases, disks at rest placed by RSA with >= 1 lu gaps; fluid at rest."""
    rng = np.random.default_rng(seed)
    radii = np.full(n_particles, float(radius))
    pos = rsa_place(rng, radii, (nx, ny, 1), 2, (True, False, True)) if n_particles else np.zeros((0, 3))
    return _finish(2, nx, ny, 1, 1, tau, (0.0, -g, 0.0), 1.0, e, radii, np.full(n_particles, density_ratio),
                   pos, np.zeros((n_particles, 3)), name, storage=storage)


def config1(**kw) -> SuspensionConfig:
    """D2Q9 FP64 128x256, tau 0.6, 20 disks R=6, density ratio 10, g=1e-6."""
    return channel_config(name="cfg1 D2Q9 128x256 channel, 20 disks R=6", **kw)


def periodic2d_config(nx=8192, ny=32768, phi=0.05, radius=4.0, tau=0.55, seed=2, gs=1.176e-7, v0=5e-3,
                      e=0.9, storage="f64", density_ratio=None, name="") -> SuspensionConfig:
    """2D periodic gravity-driven suspension (paper 2D case, scaled): disks of
    radius R at area fraction phi by RSA, density ratio drawn log-uniform in
    [2.5, 1500] once per run, initial speed v0 in random directions."""
    rng = np.random.default_rng(seed)
    n = int(round(phi * nx * ny / (math.pi * radius * radius)))
    if density_ratio is None:
        density_ratio = float(math.exp(rng.uniform(math.log(2.5), math.log(1500.0))))
    radii = np.full(n, float(radius))
    pos = rsa_place(rng, radii, (nx, ny, 1), 2, (True, True, True))
    vel = v0 * random_directions(rng, n, 2)
    return _finish(2, nx, ny, 1, 0, tau, (0.0, -gs, 0.0), 1.0, e, radii, np.full(n, density_ratio), pos, vel,
                   name or f"D2Q9 periodic {nx}x{ny}, {n} disks R={radius}", storage=storage)


def config2(scale: float = 1.0, **kw) -> SuspensionConfig:
    """D2Q9 FP64 8192x32768 (scale<1 shrinks both sides), phi=0.05, R=4."""
    nx = max(32, int(round(8192 * scale)))
    ny = max(64, int(round(32768 * scale)))
    return periodic2d_config(nx=nx, ny=ny, **kw)


def channel3d_config(nx=384, ny=1512, nz=384, phi=None, n_particles=129024, radius=3.75, density_ratio=1000.0,
                     g=4.704e-7, tau=0.6, seed=3, v0=5e-3, e=0.9, storage="f64", name="") -> SuspensionConfig:
    """3D suspension between walls in y (periodic x/z), spheres by RSA,
    gravity -y on both phases, initial speed v0 in random directions."""
    rng = np.random.default_rng(seed)
    if phi is not None:
        n_particles = int(round(phi * nx * ny * nz / (4.0 / 3.0 * math.pi * radius ** 3)))
    radii = np.full(n_particles, float(radius))
    pos = rsa_place(rng, radii, (nx, ny, nz), 3, (True, False, True)) if n_particles else np.zeros((0, 3))
    vel = v0 * random_directions(rng, n_particles, 3) if n_particles else np.zeros((0, 3))
    return _finish(3, nx, ny, nz, 1, tau, (0.0, -g, 0.0), 1.0, e, radii, np.full(n_particles, density_ratio),
                   pos, vel, name or f"D3Q19 channel {nx}x{ny}x{nz}, {n_particles} spheres R={radius}",
                   storage=storage)


def config3(**kw) -> SuspensionConfig:
    """D3Q19 FP64 384x1512x384, walls in y, 129,024 spheres R=3.75, ratio 1000."""
    return channel3d_config(**kw)


def config3_scaled(nx=64, ny=96, nz=64, storage="f64", seed=3, **kw) -> SuspensionConfig:
    """A cut-down config 3 at the same solid volume fraction (~0.1278)."""
    phi = 129024 * (4.0 / 3.0) * math.pi * 3.75 ** 3 / (384 * 1512 * 384)
    return channel3d_config(nx=nx, ny=ny, nz=nz, phi=phi, storage=storage, seed=seed, **kw)


def periodic3d_config(nx=64, ny=64, nz=64, phi=0.1, radius=3.75, density_ratio=1000.0, gs=4.704e-7, tau=0.6,
                      seed=5, v0=5e-3, e=0.9, storage="f64", name="") -> SuspensionConfig:
    """3D fully periodic gravity-driven suspension (the paper's 3D setup)."""
    rng = np.random.default_rng(seed)
    n = int(round(phi * nx * ny * nz / (4.0 / 3.0 * math.pi * radius ** 3)))
    radii = np.full(n, float(radius))
    pos = rsa_place(rng, radii, (nx, ny, nz), 3, (True, True, True))
    vel = v0 * random_directions(rng, n, 3)
    return _finish(3, nx, ny, nz, 0, tau, (0.0, -gs, 0.0), 1.0, e, radii, np.full(n, density_ratio), pos, vel,
                   name or f"D3Q19 periodic {nx}x{ny}x{nz}, {n} spheres", storage=storage)


def random_populations(rng: np.random.Generator, cfg: SuspensionConfig, amp: float = 0.05) -> np.ndarray:
    """Positive non-equilibrium populations for parity tests: rho_f/Q times
    (1 + amp * noise), shape (Q, nz, ny, nx).  Far from equilibrium on
    purpose, so that every term of the collision is exercised."""
    Q = 9 if cfg.dim == 2 else 19
    nz = cfg.nz if cfg.dim == 3 else 1
    return cfg.rho_fluid / Q * (1.0 + amp * rng.standard_normal((Q, nz, cfg.ny, cfg.nx)))


def batch_configs(n: int = 32, seed: int = 4, nx_range=(256, 1024), ny_range=(512, 4096), np_range=(10, 2000),
                  r_range=(4.0, 8.0), ratio_range=(2.5, 1500.0), phi_max=0.25, tau=0.6, gs=1.176e-7, v0=5e-3,
                  e=0.9, storage="f64"):
    """Independent 2D periodic gravity-driven suspensions of uneven sizes:
    nx and ny drawn log-uniformly in their ranges (ny >= nx), particle count
    log-uniform in np_range (capped at solid fraction phi_max), radii uniform
    in r_range, one density ratio per lattice log-uniform in ratio_range."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n):
        nx = int(round(math.exp(rng.uniform(math.log(nx_range[0]), math.log(nx_range[1])))))
        ny = int(round(math.exp(rng.uniform(math.log(max(ny_range[0], nx)), math.log(ny_range[1])))))
        ratio = float(math.exp(rng.uniform(math.log(ratio_range[0]), math.log(ratio_range[1]))))
        k = int(round(math.exp(rng.uniform(math.log(np_range[0]), math.log(np_range[1])))))
        radii = rng.uniform(r_range[0], r_range[1], k)
        area = math.pi * (radii ** 2)
        while area.sum() > phi_max * nx * ny and k > 1:
            k -= 1
            area = area[:k]
        radii = radii[:k]
        pos = rsa_place(rng, radii, (nx, ny, 1), 2, (True, True, True))
        vel = v0 * random_directions(rng, k, 2)
        out.append(_finish(2, nx, ny, 1, 0, tau, (0.0, -gs, 0.0), 1.0, e, radii, np.full(k, ratio), pos, vel,
                           f"batch member {i}: D2Q9 {nx}x{ny}, {k} disks R in [{r_range[0]}, {r_range[1]}], "
                           f"ratio {ratio:.1f}", storage=storage))
    return out


def jittered_lattice_place(rng: np.random.Generator, n: int, R: float, box, gap: float = 0.2) -> np.ndarray:
    """n non-overlapping spheres of radius R in a fully periodic box: the
    sites of the coarsest cubic lattice that holds n spheres, a random subset
    of n of them, each displaced uniformly by up to half the free spacing.
    (Random sequential addition jams near solid fraction 0.38; this reaches
    denser suspensions.)"""
    L = np.array(box, dtype=np.float64)
    m = np.maximum(1, np.floor(L / (2 * R + gap)).astype(int))
    while m.prod() < n:
        raise RuntimeError("box too small for the requested number of spheres")
    a = L / m
    sites = np.stack(np.meshgrid(*[np.arange(k) for k in m], indexing="ij"), -1).reshape(-1, 3)
    pick = rng.choice(len(sites), size=n, replace=False)
    jit = np.maximum(0.0, (a - 2 * R - gap) / 2)
    pos = (sites[pick] + 0.5) * a + rng.uniform(-1, 1, (n, 3)) * jit
    return np.mod(pos, L)


def closure_config(phi: float, seed: int, n: int = 128, radius: float = 3.75, density_ratio: float = 1000.0,
                   gs: float = 4.704e-7, tau: float = 0.6, v0: float = 5e-3, e: float = 0.9,
                   storage: str = "f32dev") -> SuspensionConfig:
    """A fully periodic D3Q19 gravity-driven suspension of solid fraction phi
    for drag sampling (RSA below phi = 0.25, jittered lattice above)."""
    rng = np.random.default_rng(seed)
    k = int(round(phi * n ** 3 / (4.0 / 3.0 * math.pi * radius ** 3)))
    radii = np.full(k, float(radius))
    if phi < 0.25:
        pos = rsa_place(rng, radii, (n, n, n), 3, (True, True, True), gap=0.5)
    else:
        pos = jittered_lattice_place(rng, k, radius, (n, n, n))
    vel = v0 * random_directions(rng, k, 3)
    return _finish(3, n, n, n, 0, tau, (0.0, -gs, 0.0), 1.0, e, radii, np.full(k, density_ratio), pos, vel,
                   f"closure D3Q19 {n}^3 periodic, phi={phi}, {k} spheres, seed {seed}", storage=storage)


def fixed_sphere_config(R: float, phi: float, tau: float = 1.0, re_p: float = 0.2, storage: str = "f64",
                        offset=(0.1, 0.2, 0.3)) -> SuspensionConfig:
    """Gravity-driven flow through a simple cubic array of fixed spheres: one
    sphere of radius R in a periodic cube of side L = round(R (4 pi/(3 phi))^(1/3)),
    held in place by a solid/gas density ratio of 1e12 and no gravity of its
    own; the gas is driven by a body force along x sized for the particle
    Reynolds number re_p (Stokes estimate).  The centre sits near the cube
    centre, shifted by ``offset`` so that it is not node-aligned."""
    L = int(round(R * (4.0 * math.pi / (3.0 * phi)) ** (1.0 / 3.0)))
    nu = (tau - 0.5) / 3.0
    u_target = re_p * nu / (2.0 * R)
    g = 6.0 * math.pi * nu * R * u_target / L ** 3  # Stokes drag of one sphere per cube volume
    pos = np.array([[L / 2 + offset[0], L / 2 + offset[1], L / 2 + offset[2]]])
    return SuspensionConfig(
        dim=3, nx=L, ny=L, nz=L, wall_y=0, tau=tau, body_force=np.array([g, 0.0, 0.0]), gravity=np.zeros(3),
        rho_fluid=1.0, k_n=0.0, restitution=1.0, dem_substeps=1, pos=pos, vel=np.zeros((1, 3)),
        omega=np.zeros((1, 3)), radius=np.array([float(R)]), density=np.array([1e12]), storage=storage,
        name=f"fixed sphere R={R} in a periodic {L}^3 cube, phi={4 / 3 * math.pi * R ** 3 / L ** 3:.4f}")
