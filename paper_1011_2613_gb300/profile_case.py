"""A fixed, small case for profiling one kernel family under ncu:
``python -m paper_1011_2613_gb300.profile_case --workload cfg3s --storage f64
--variant 5 [--no-particles] [--steps 3]``.  Builds the workload, fixes the
collision form, runs 4 warm-up steps and ``--steps`` steps through
``lbm_imb_step_profiled`` (one launch per kernel family per step, no graph),
and prints the per-family device times."""
from __future__ import annotations

import argparse
import json

import numpy as np

from . import inputs as I
from . import lbm as L

CASES = {
    # config 3 at 1/16 of its nodes (same solid fraction and physics)
    "cfg3s": lambda: I.config3_scaled(nx=192, ny=384, nz=192),
    # config 2 at 1/32 of its nodes (same solid fraction and physics)
    "cfg2s": lambda: I.periodic2d_config(nx=2048, ny=4096),
}


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", default="cfg3s", choices=sorted(CASES))
    ap.add_argument("--storage", default="f64", choices=["f64", "f32dev", "f16dev", "dfdev"])
    ap.add_argument("--variant", type=int, default=0)
    ap.add_argument("--no-particles", action="store_true")
    ap.add_argument("--steps", type=int, default=3)
    a = ap.parse_args(argv)
    cfg = CASES[a.workload]().replace(storage=a.storage)
    if a.no_particles:
        z = np.zeros((0, 3))
        cfg = cfg.replace(pos=z, vel=z, omega=z, radius=np.zeros(0), density=np.zeros(0))
    sim = L.Simulation(cfg)
    sim.set_collide_variant(a.variant)
    sim.step(4)
    sim.sync()
    k, t = sim.step_profiled(a.steps)
    print(json.dumps({"workload": a.workload, "storage": a.storage, "variant": a.variant,
                      "particles": cfg.n_particles, "nodes": cfg.n_nodes,
                      "ms_per_step": {n: v / a.steps for n, v in k.items()}}))
    sim.close()


if __name__ == "__main__":
    main()
