"""Host logic of the launch-shape autotuner (no GPU): picks the fastest
candidate, skips shapes that fail, round-trips its JSON cache."""
import os

import pytest

from paper_1011_2613_gb300 import autotune as A
from paper_1011_2613_gb300 import inputs as I


class FakeBatch:
    def __init__(self, times):
        self.times = times
        self.shape = None
        self.steps = 0

    def set_launch(self, tx, bps):
        if (tx, bps) not in self.times:
            raise RuntimeError("does not fit")
        self.shape = (tx, bps)

    def step(self, n):
        self.steps += n

    def sync(self):
        pass

    def step_profiled(self, n):
        self.steps += n
        return self.times[self.shape] * n


def test_tune_picks_fastest_and_skips_failures():
    times = {(32, 1): 3.0, (64, 2): 1.5, (128, 0): 2.0}
    b = FakeBatch(times)
    rec = A.tune(b, steps=4, warmup=1, candidates=[(32, 1), (64, 2), (128, 0), (128, 4)])
    assert (rec["tile_x"], rec["blocks_per_sm"]) == (64, 2)
    assert b.shape == (64, 2)
    assert rec["ms_per_step"] == pytest.approx(1.5)
    assert any("error" in r for r in rec["table"])
    assert b.steps == 3 * (1 + 4)


def test_tune_raises_when_nothing_fits():
    with pytest.raises(RuntimeError):
        A.tune(FakeBatch({}), candidates=[(32, 1)])


def test_cache_roundtrip_and_signature(tmp_path):
    p = str(tmp_path / "sub" / "cache.json")
    cfgs = I.batch_configs(n=3, seed=2, nx_range=(40, 60), ny_range=(64, 80), np_range=(2, 5), r_range=(3, 4))
    key = A.signature(cfgs, "GPU X")
    assert key.startswith("GPU X|d2|f64|m3|")
    A.save_cache({key: {"tile_x": 64, "blocks_per_sm": 2, "ms_per_step": 1.0}}, p)
    assert A.load_cache(p)[key]["tile_x"] == 64
    assert A.load_cache(str(tmp_path / "missing.json")) == {}
    open(p, "w").write("not json")
    assert A.load_cache(p) == {}
