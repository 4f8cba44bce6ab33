"""Validation workload: drag on a fixed sphere in a simple cubic array.

A sphere held fixed in a periodic cube is driven by a uniform body force on
the gas until the flow is steady; the dimensionless drag
K = F / (6 pi rho nu R U), with F the hydrodynamic force on the sphere (Eq. 3)
and U the mean gas velocity over the cube, is compared with the dilute
simple-cubic-array result of Hasimoto (1959),
1/K = 1 - 1.7601 phi^(1/3) + phi - 1.5593 phi^2 + O(phi^(7/3)).
The error falls as the sphere spans more lattice cells, the trend of the
paper's fixed-sphere validation (Table 1)."""
from __future__ import annotations

import math

import numpy as np

from . import inputs as I
from .lbm import Simulation


def hasimoto_K(phi: float) -> float:
    """Drag factor of a simple cubic array of spheres at solid fraction phi
    (Hasimoto 1959, terms through phi^2)."""
    return 1.0 / (1.0 - 1.7601 * phi ** (1.0 / 3.0) + phi - 1.5593 * phi ** 2)


def fixed_sphere_drag(R: float, phi: float = 0.008, tau: float = 1.0, re_p: float = 0.2, storage: str = "f64",
                      eps_method: int = 0, relax: float = 10.0) -> dict:
    """Run the fixed-sphere array from rest to steady state and return the
    measured and Hasimoto drag factors.  The gas spins up with the time
    constant L^3 / (6 pi nu R K) (its momentum over the array's drag
    coefficient); the run lasts ``relax`` of them, and at least 14 e-folding
    times L^2 / (4 pi^2 nu) of the slowest diffusive mode."""
    cfg = I.fixed_sphere_config(R, phi, tau=tau, re_p=re_p, storage=storage).replace(eps_method=eps_method)
    L = cfg.nx
    nu = (tau - 0.5) / 3.0
    kh = hasimoto_K(4.0 / 3.0 * math.pi * R ** 3 / L ** 3)
    t_drag = L ** 3 / (6.0 * math.pi * nu * R * kh)
    steps = int(math.ceil(max(relax * t_drag, 14.0 * L * L / (4.0 * math.pi ** 2 * nu))))
    sim = Simulation(cfg)
    sim.step(steps - 1)
    sim.sync()
    f_prev = sim.particles()["force"][0, 0]
    sim.step(1)
    sim.sync()
    p = sim.particles()
    rho, u, eps = sim.fields()
    sim.close()
    F = float(p["force"][0, 0])
    U = float(u[0].mean())
    rho_m = float(rho.mean())
    phi_eff = 4.0 / 3.0 * math.pi * R ** 3 / L ** 3
    K = F / (6.0 * math.pi * rho_m * nu * R * U)
    Kh = hasimoto_K(phi_eff)
    return {"R": R, "L": L, "phi": phi_eff, "steps": steps, "K": K, "K_hasimoto": Kh,
            "rel_error": K / Kh - 1.0, "re_p": 2.0 * R * U / nu, "force": F,
            "force_balance": F / (rho_m * cfg.body_force[0] * L ** 3) - 1.0,
            "steady": abs(F - f_prev) / abs(F), "eps_volume": float(np.sum(eps)) / (4 / 3 * math.pi * R ** 3) - 1.0}
