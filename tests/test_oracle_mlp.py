"""Pins for the MLP oracle: analytic gradients against central finite
differences, the Adam update against a hand-computed step, bf16 rounding
against exact bfloat16 values."""
import numpy as np

from oracle import mlp_oracle as M


def test_gradients_match_finite_differences():
    sizes = (6, 8, 8, 8, 8, 3)
    W, b = M.init_params(3, sizes)
    rng = np.random.default_rng(0)
    for l in range(len(b)):
        b[l] = 0.1 * rng.standard_normal(b[l].shape)
    x = rng.standard_normal((7, 6))
    t = rng.standard_normal((7, 3))
    gW, gb, _ = M.gradients(W, b, x, t)
    h = 1e-6
    for l in range(len(W)):
        for (i, j) in [(0, 0), (W[l].shape[0] - 1, W[l].shape[1] - 1), (1, 2)]:
            Wp = [w.copy() for w in W]
            Wm = [w.copy() for w in W]
            Wp[l][i, j] += h
            Wm[l][i, j] -= h
            fd = (M.loss(Wp, b, x, t) - M.loss(Wm, b, x, t)) / (2 * h)
            assert abs(fd - gW[l][i, j]) <= 1e-6 * max(1.0, abs(fd))
        bp = [v.copy() for v in b]
        bm = [v.copy() for v in b]
        bp[l][0] += h
        bm[l][0] -= h
        fd = (M.loss(W, bp, x, t) - M.loss(W, bm, x, t)) / (2 * h)
        assert abs(fd - gb[l][0]) <= 1e-6 * max(1.0, abs(fd))


def test_linear_net_gradient_closed_form():
    """One layer y = W x + b: dL/dW = 2/(n m) (y - t)^T x."""
    W = [np.array([[0.5, -1.0], [2.0, 0.25]])]
    b = [np.array([0.1, -0.2])]
    x = np.array([[1.0, 2.0], [-1.0, 0.5], [0.0, 3.0]])
    t = np.array([[0.0, 1.0], [1.0, 0.0], [2.0, 2.0]])
    y = x @ W[0].T + b[0]
    gW, gb, _ = M.gradients(W, b, x, t)
    assert np.allclose(gW[0], 2 / 6 * (y - t).T @ x)
    assert np.allclose(gb[0], 2 / 6 * (y - t).sum(axis=0))


def test_adam_first_step_is_lr_sign():
    """After one step, m/c1 = g and v/c2 = g^2, so the update is lr*g/(|g|+eps)."""
    p = [np.array([1.0, -2.0, 0.5])]
    g = [np.array([0.3, -4.0, 0.0])]
    opt = M.Adam(p)
    opt.step(p, g, 0.01)
    expect = np.array([1.0 - 0.01 * 0.3 / (0.3 + 1e-8), -2.0 + 0.01 * 4.0 / (4.0 + 1e-8), 0.5])
    assert np.allclose(p[0], expect, rtol=0, atol=1e-15)


def test_bf16_rounding():
    vals = np.array([1.0, 1.00390625, 1.005859375, 3.0e-3, -7.5, 65504.0])
    r = M.bf16_round(vals)
    assert r[0] == 1.0
    assert r[1] == 1.0  # halfway between 1 and 1+2^-7: ties to even
    assert r[2] == 1.0078125
    assert abs(r[3] - 3.0e-3) <= 2 ** -8 * 3.0e-3  # half an ulp of an 8-bit significand
    assert r[4] == -7.5
    assert r[5] == 65536.0
