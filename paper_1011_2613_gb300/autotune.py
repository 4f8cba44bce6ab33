"""Launch-shape autotuner for the batched persistent step.

Times each candidate (tile width, CTAs per SM) on the actual batch through
``lbm_imb_step_profiled`` and keeps the fastest; results are cached in a JSON
file keyed by the GPU, lattice type, storage and a coarse size signature, so a
later batch of the same shape starts with the tuned launch.  Timing advances
the batch it runs on (the steps are real steps).

Cache file: $LBM_IMB_AUTOTUNE_CACHE, else ~/.cache/lbm_imb/autotune.json.
"""
from __future__ import annotations

import json
import math
import os
import tempfile

CANDIDATES = [(tx, bps) for tx in (32, 64, 128) for bps in (1, 2, 4, 0)]


def cache_path() -> str:
    p = os.environ.get("LBM_IMB_AUTOTUNE_CACHE")
    if p:
        return p
    return os.path.join(os.path.expanduser("~"), ".cache", "lbm_imb", "autotune.json")


def signature(cfgs, device_name: str) -> str:
    """GPU, lattice, storage, member count and log2 buckets of the total node
    and particle counts."""
    c0 = cfgs[0]
    nodes = sum(c.n_nodes for c in cfgs)
    parts = sum(c.n_particles for c in cfgs)
    return "|".join([device_name, f"d{c0.dim}", str(c0.storage), f"m{len(cfgs)}",
                     f"n{int(math.log2(max(nodes, 1)))}", f"p{int(math.log2(max(parts, 1)))}"])


def load_cache(path: str | None = None) -> dict:
    path = path or cache_path()
    try:
        with open(path) as fh:
            d = json.load(fh)
        return d if isinstance(d, dict) else {}
    except (OSError, ValueError):
        return {}


def save_cache(cache: dict, path: str | None = None) -> None:
    path = path or cache_path()
    os.makedirs(os.path.dirname(path) or ".", exist_ok=True)
    fd, tmp = tempfile.mkstemp(dir=os.path.dirname(path) or ".", suffix=".tmp")
    with os.fdopen(fd, "w") as fh:
        json.dump(cache, fh, indent=1, sort_keys=True)
    os.replace(tmp, path)


def tune(batch, steps: int = 3, warmup: int = 1, candidates=None) -> dict:
    """Time every candidate on ``batch`` (an object with set_launch, step,
    sync, step_profiled(n) -> ms) and leave it on the fastest.  Returns
    {"tile_x", "blocks_per_sm", "ms_per_step", "table"}."""
    table = []
    for tx, bps in (candidates or CANDIDATES):
        try:
            batch.set_launch(tx, bps)
            if warmup:
                batch.step(warmup)
                batch.sync()
            ms = batch.step_profiled(steps) / steps
        except Exception as ex:  # a shape that does not fit is skipped
            table.append({"tile_x": tx, "blocks_per_sm": bps, "error": str(ex)})
            continue
        table.append({"tile_x": tx, "blocks_per_sm": bps, "ms_per_step": ms})
    ok = [r for r in table if "ms_per_step" in r]
    if not ok:
        raise RuntimeError("no launch shape could be timed")
    best = min(ok, key=lambda r: r["ms_per_step"])
    batch.set_launch(best["tile_x"], best["blocks_per_sm"])
    return {"tile_x": best["tile_x"], "blocks_per_sm": best["blocks_per_sm"],
            "ms_per_step": best["ms_per_step"], "table": table}


def tuned_batch(cfgs, device=None, path: str | None = None, steps: int = 3):
    """A Batch on the cached launch shape for this signature, tuning (and
    caching) first when there is none.  Returns (batch, record, from_cache)."""
    import torch

    from .lbm import Batch

    dev = torch.device(device if device is not None else "cuda")
    key = signature(cfgs, torch.cuda.get_device_name(dev))
    cache = load_cache(path)
    if key in cache:
        rec = cache[key]
        return Batch(cfgs, tile_x=rec["tile_x"], blocks_per_sm=rec["blocks_per_sm"], device=dev), rec, True
    batch = Batch(cfgs, device=dev)
    rec = tune(batch, steps=steps)
    cache[key] = {k: rec[k] for k in ("tile_x", "blocks_per_sm", "ms_per_step")}
    save_cache(cache, path)
    return batch, rec, False


COLLIDE_VARIANTS = (0, 1, 2, 3, 4, 5, 6, 7, 8, 9)
# the pair storage has the persistent fused forms, the TMA form and the
# split forms (6: covered nodes in FP64, 7: in pair arithmetic)
COLLIDE_VARIANTS_BY_STORAGE = {"dfdev": (0, 1, 2, 3, 4, 5, 6, 7, 8, 9)}


def collide_variants(storage) -> tuple:
    return COLLIDE_VARIANTS_BY_STORAGE.get(storage, COLLIDE_VARIANTS)


def collide_signature(cfg, device_name: str) -> str:
    return "|".join(["collide", device_name, f"d{cfg.dim}", str(cfg.storage),
                     f"n{int(math.log2(max(cfg.n_nodes, 1)))}", f"p{int(math.log2(max(cfg.n_particles, 1)))}"])


def _step_ms(sim, steps: int) -> float:
    """Whole-step time (graph-replayed steps, CUDA events on the simulation's
    stream): forms that change the rasteriser's work or overlap it with the
    collision are compared on what they change."""
    import torch
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(sim.stream)
    sim.step(steps)
    e1.record(sim.stream)
    e1.synchronize()
    return e0.elapsed_time(e1) / steps


def tune_collide(sim, steps: int = 2, variants=None) -> dict:
    """Time every collide kernel form on ``sim`` by its whole step (real
    steps: the simulation advances) and leave it on the fastest.  Returns
    {"variant", "table"}."""
    if variants is None:
        variants = collide_variants(sim.cfg.storage)
    table = []
    for var in variants:
        try:
            sim.set_collide_variant(var)
            sim.step(1)
            sim.sync()
            ms = _step_ms(sim, steps)
            sim.sync()
        except Exception as ex:
            table.append({"variant": var, "error": str(ex)})
            continue
        table.append({"variant": var, "step_ms": ms})
    ok = [r for r in table if "step_ms" in r]
    if not ok:
        raise RuntimeError("no collide variant could be timed")
    best = min(ok, key=lambda r: r["step_ms"])
    sim.set_collide_variant(best["variant"])
    return {"variant": best["variant"], "table": table}


def tuned_collide(sim, path: str | None = None, steps: int = 2) -> tuple[dict, bool]:
    """Apply the cached collide variant for this configuration, or tune and
    cache it.  Returns (record, from_cache)."""
    import torch

    key = collide_signature(sim.cfg, torch.cuda.get_device_name(sim.device))
    cache = load_cache(path)
    if key in cache:
        sim.set_collide_variant(cache[key]["variant"])
        return cache[key], True
    rec = tune_collide(sim, steps=steps)
    cache[key] = {"variant": rec["variant"], "table": rec["table"]}
    save_cache(cache, path)
    return rec, False
