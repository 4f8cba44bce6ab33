"""GPU: the FP64 <-> FP32-pair conversions of the double-FP32 storage
(integer bit operations, no FP64 instructions) against exact arithmetic."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def pairs(rng, n):
    """Normalised pairs h = fl32(x), l = fl32(x - h) of doubles x over many
    binades, both signs, plus powers of two with neighbours of either sign."""
    x = rng.uniform(0.5, 1.0, n) * 2.0 ** rng.integers(-70, 20, n) * rng.choice([-1.0, 1.0], n)
    h = x.astype(np.float32)
    l = (x - h.astype(np.float64)).astype(np.float32)
    p2 = (2.0 ** rng.integers(-60, 10, 64)).astype(np.float32) * rng.choice([-1, 1], 64).astype(np.float32)
    lp = (p2.astype(np.float64) * rng.uniform(-2.0 ** -25, 2.0 ** -25, 64)).astype(np.float32)
    return np.concatenate([h, p2, [0.0, 1.0, -1.0]]).astype(np.float32), \
        np.concatenate([l, lp, [0.0, 0.0, 0.0]]).astype(np.float32)


def test_pair_to_double_is_the_rounded_sum():
    import torch
    from paper_1011_2613_gb300 import lbm as L
    rng = np.random.default_rng(3)
    h, l = pairs(rng, 200000)
    d = np.zeros(h.size)
    dev = torch.device("cuda")
    out, _ = L.probe_df(torch.from_numpy(h).to(dev), torch.from_numpy(l).to(dev), torch.from_numpy(d).to(dev))
    exact = h.astype(np.float64) + l.astype(np.float64)  # h + l needs at most 53 bits here
    assert np.array_equal(out.cpu().numpy(), exact)


def test_double_roundtrip_keeps_48_bits():
    import torch
    from paper_1011_2613_gb300 import lbm as L
    rng = np.random.default_rng(4)
    d = rng.standard_normal(200000) * 10.0 ** rng.uniform(-20, 1, 200000)
    d = np.concatenate([d, [0.0, -0.0, 1.0, -0.5, 2.0 ** -100, 1e-40, -1e-45]])
    z = torch.zeros(d.size, dtype=torch.float32, device="cuda")
    _, rt = L.probe_df(z, z, torch.from_numpy(d).cuda())
    rt = rt.cpu().numpy()
    big = np.abs(d) >= 2.0 ** -74
    assert np.all(np.abs(rt[big] - d[big]) <= 2.0 ** -47 * np.abs(d[big]))
    small = (np.abs(d) < 2.0 ** -74) & (np.abs(d) >= 2.0 ** -126)
    assert np.all(np.abs(rt[small] - d[small]) <= 2.0 ** -23 * np.abs(d[small]))
    assert np.all(rt[np.abs(d) < 2.0 ** -126] == 0.0)
