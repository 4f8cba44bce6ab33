"""The learned drag closure on the GPU: tcgen05 operand layout (one product
against numpy), network forward and gradients against the FP64 MLP oracle
with the same bfloat16 rounding points, one Adam step, convergence on a
smooth target, and the per-particle drag samples against their definition."""
import numpy as np
import pytest

from oracle import mlp_oracle as M
from oracle import oracle as O
from paper_1011_2613_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def bf16_bits(x):
    a = np.ascontiguousarray(np.asarray(x, dtype=np.float32))
    u = a.view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) >> 16
    return u.astype(np.uint16)


def bits_to_f64(b):
    return (b.astype(np.uint32) << 16).view(np.float32).astype(np.float64)


@pytest.mark.parametrize("N,K", [(16, 16), (128, 16), (16, 128), (128, 128), (64, 32)])
def test_tcgen05_product_layout(N, K):
    from paper_1011_2613_gb300 import closure as CL

    rng = np.random.default_rng(N * 1000 + K)
    a = bf16_bits(rng.standard_normal((128, K)))
    b = bf16_bits(rng.standard_normal((N, K)))
    ref = bits_to_f64(a) @ bits_to_f64(b).T
    d = CL.probe_gemm(a, b)
    assert np.max(np.abs(d - ref)) <= 1e-5 * max(1.0, np.abs(ref).max()) * K


def _net(seed=0, max_batch=4096):
    from paper_1011_2613_gb300 import closure as CL

    W, b = M.init_params(seed)
    rng = np.random.default_rng(seed + 1)
    b = [0.05 * rng.standard_normal(v.shape) for v in b]
    mlp = CL.MLP(max_batch=max_batch, seed=seed)
    mlp.set_params(CL.layers_to_flat(W, b))
    # the GPU holds FP32 masters: compare against the same FP32 values
    W, b = CL.flat_to_layers(mlp.get_params())
    return mlp, W, b


def test_forward_matches_oracle():
    """Element by element, within 1e-3 of the largest output, against the
    oracle with the same bfloat16 rounding points (x, W_l, every hidden
    activation), FP64 accumulation; and loosely against the unrounded FP64
    network."""
    import torch

    mlp, W, b = _net(3)
    x = np.random.default_rng(4).standard_normal((300, 6)).astype(np.float32)
    y = mlp.predict(torch.tensor(x, device="cuda")).cpu().numpy()
    yr, _ = M.forward(W, b, x.astype(np.float64), bf16=True)
    err = float(np.max(np.abs(y - yr)) / np.abs(yr).max())
    print(f"forward: max |y - oracle| / max |oracle| = {err:.2e}")
    assert err <= 1e-3
    y64, _ = M.forward(W, b, x.astype(np.float64), bf16=False)
    assert np.max(np.abs(y - y64)) <= 6e-2 * np.abs(y64).max()


@pytest.mark.parametrize("batch", [256, 1000, 4096])
def test_gradients_match_oracle(batch):
    """Every weight and bias gradient element by element within 1e-3 of its
    tensor's largest entry (the oracle rounds the same operands to bfloat16:
    x, W_l, the activations and the back-propagated gradients), for a batch
    of whole tiles, a ragged one and a large one."""
    import torch
    from paper_1011_2613_gb300 import closure as CL

    mlp, W, b = _net(5)
    rng = np.random.default_rng(6)
    x = rng.standard_normal((batch, 6)).astype(np.float32)
    t = rng.standard_normal((batch, 3)).astype(np.float32)
    g, loss = mlp.gradients(torch.tensor(x, device="cuda"), torch.tensor(t, device="cuda"))
    gW, gb = CL.flat_to_layers(g)
    rW, rb, rloss = M.gradients(W, b, x.astype(np.float64), t.astype(np.float64), bf16=True)
    assert abs(loss - rloss) <= 1e-3 * rloss
    worst = 0.0
    for l in range(5):
        ew = float(np.max(np.abs(gW[l] - rW[l])) / np.abs(rW[l]).max())
        eb = float(np.max(np.abs(gb[l] - rb[l])) / max(np.abs(rb[l]).max(), 1e-30))
        worst = max(worst, ew, eb)
        assert ew <= 1e-3, (l, ew)
        assert eb <= 1e-3, (l, eb)
    print(f"batch {batch}: worst gradient error {worst:.2e} of the tensor maximum")


def test_one_adam_step():
    import torch
    from paper_1011_2613_gb300 import closure as CL

    mlp, W, b = _net(7)
    rng = np.random.default_rng(8)
    x = torch.tensor(rng.standard_normal((128, 6)).astype(np.float32), device="cuda")
    t = torch.tensor(rng.standard_normal((128, 3)).astype(np.float32), device="cuda")
    p0 = mlp.get_params().astype(np.float64)
    g, _ = mlp.gradients(x, t)
    mlp.train(x, t, batch=128, steps=1, lr=1e-3)
    p1 = mlp.get_params().astype(np.float64)
    ref = [p0.copy()]
    M.Adam(ref).step(ref, [g.astype(np.float64)], 1e-3)
    assert np.max(np.abs(p1 - ref[0])) <= 1e-6


def test_training_fits_smooth_target():
    import torch
    from paper_1011_2613_gb300 import closure as CL

    rng = np.random.default_rng(9)
    x = rng.uniform(-1, 1, (8192, 6)).astype(np.float32)
    t = np.stack([np.sin(2 * x[:, 0]) + x[:, 1] * x[:, 2], np.cos(x[:, 3]) - x[:, 4] ** 2,
                  x[:, 5] * x[:, 0]], axis=1).astype(np.float32)
    mlp = CL.MLP(max_batch=1024, seed=1)
    xd, td = torch.tensor(x, device="cuda"), torch.tensor(t, device="cuda")
    _, l0 = mlp.gradients(xd[:1024], td[:1024])
    mlp.train(xd, td, batch=1024, steps=600, lr=2e-3)
    _, l1 = mlp.gradients(xd[:1024], td[:1024])
    assert l1 < 0.1 * l0


def test_drag_samples_match_definition():
    from paper_1011_2613_gb300 import closure as CL
    from paper_1011_2613_gb300 import lbm

    cfg = I.periodic3d_config(nx=28, ny=32, nz=26, phi=0.12, radius=3.75, seed=12, v0=0.02)
    sim = lbm.Simulation(cfg)
    ref = O.OracleSim(cfg)
    sim.step(6)
    ref.step(6)
    fg, tg = CL.drag_samples(sim, 5.0)
    fr, tr = M.drag_samples(ref, 5.0)
    fg, tg = fg.cpu().numpy(), tg.cpu().numpy()
    assert np.max(np.abs(fg - fr) / (np.abs(fr) + 1e-3 * np.abs(fr).max(axis=0))) < 1e-4
    assert np.max(np.abs(tg - tr)) < 1e-4 * np.abs(tr).max()
