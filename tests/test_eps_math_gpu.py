"""GPU: the first-quadrant arctangent used by the FP64 exact-volume
rasterisation (arctangent addition formula on a 1/16 table + Taylor series)
against CUDA's atan2 and the host's libm (numpy.arctan2)."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def ulp_err(a, b):
    return np.abs(a - b) / np.spacing(np.maximum(np.abs(b), 1e-300))


def test_atan2_first_quadrant_within_two_ulp():
    import torch
    from paper_1011_2613_gb300 import lbm as L

    rng = np.random.default_rng(5)
    n = 1 << 20
    # magnitudes of the rasteriser's arguments (0 .. a few R^2), plus edges
    y = rng.uniform(0.0, 1.0, n) * 10.0 ** rng.uniform(-3, 2, n)
    x = rng.uniform(0.0, 1.0, n) * 10.0 ** rng.uniform(-3, 2, n)
    y[:64] = 0.0
    x[64:128] = 0.0
    y[128:192] = x[128:192]                      # t = 1 exactly
    y[192:256] = x[192:256] * (np.arange(64) % 17) / 16.0   # table points
    x[:64] += 1.0
    y[64:128] += 1.0
    fast, ref = L.probe_atan2q1(torch.from_numpy(y).cuda(), torch.from_numpy(x).cuda())
    fast = fast.cpu().numpy()
    ref = ref.cpu().numpy()
    host = np.arctan2(y, x)
    assert np.all(np.isfinite(fast))
    assert ulp_err(fast, ref).max() <= 2.0
    assert ulp_err(fast, host).max() <= 2.0
    assert np.all(fast[:64] == 0.0)
    assert np.allclose(fast[64:128], np.pi / 2, rtol=0, atol=4e-16)


@pytest.mark.parametrize("dim", [2, 3])
def test_fp32_rasteriser_close_to_fp64(dim):
    """The FP32 rasteriser (reduced-precision storages) evaluates the same
    closed forms as the FP64 one; its covered fractions stay within a few
    FP32 roundings of the corner terms (magnitude R^3 in 3D)."""
    from paper_1011_2613_gb300 import inputs as I
    from paper_1011_2613_gb300 import lbm as L
    if dim == 2:
        cfg = I.periodic2d_config(nx=96, ny=80, phi=0.2, radius=5.3, seed=4, density_ratio=3.0)
    else:
        cfg = I.periodic3d_config(nx=40, ny=36, nz=32, phi=0.15, radius=3.75, seed=4)
    _, _, e64 = L.Simulation(cfg).fields()
    _, _, e32 = L.Simulation(cfg.replace(storage="f32dev")).fields()
    d = float(np.max(np.abs(e32 - e64)))
    print(f"dim {dim}: max |eps32 - eps64| = {d:.2e}")
    assert d < 1e-4
