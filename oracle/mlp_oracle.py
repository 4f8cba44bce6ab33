"""FP64 reference of the learned drag closure (MLP) and of its drag samples.

TEST INFRASTRUCTURE ONLY: used by the tests to check the library's MLP
training/inference kernels and its per-particle drag-sample kernel.  Plain
numpy; no code shared with the CUDA path.

Network (normalised inputs -> normalised outputs):
    h1 = relu(W1 x + b1), h2 = relu(W2 h1 + b2), h3 = relu(W3 h2 + b3),
    h4 = relu(W4 h3 + b4), y = W5 h4 + b5
with sizes 6 -> 128 -> 128 -> 128 -> 128 -> 3, weights W_l stored [out][in].
Loss: mean over samples and outputs of (y - t)^2.  Optimiser: Adam
(beta1 0.9, beta2 0.999, eps 1e-8) on FP32-like master weights.

With ``bf16=True`` the forward/backward round to bfloat16 at the points where
the GPU kernels keep bfloat16 operands (inputs of every product: x, h_l,
W_l and the back-propagated gradients), accumulating in FP64.
"""
from __future__ import annotations

import numpy as np

SIZES = (6, 128, 128, 128, 128, 3)


def bf16_round(x):
    """Round to the nearest bfloat16 (ties to even), via float32."""
    a = np.ascontiguousarray(np.asarray(x, dtype=np.float32))
    bits = a.view(np.uint32).astype(np.uint64)
    lsb = (bits >> 16) & 1
    bits = (bits + 0x7FFF + lsb) & 0xFFFF0000
    return bits.astype(np.uint32).view(np.float32).astype(np.float64).reshape(np.shape(x))


def init_params(seed: int = 0, sizes=SIZES):
    """He-uniform weights, zero biases (float64)."""
    rng = np.random.default_rng(seed)
    W, b = [], []
    for i in range(len(sizes) - 1):
        lim = np.sqrt(6.0 / sizes[i])
        W.append(rng.uniform(-lim, lim, (sizes[i + 1], sizes[i])))
        b.append(np.zeros(sizes[i + 1]))
    return W, b


def forward(W, b, x, bf16=False):
    """x: (n, 6).  Returns (y (n, 3), cache of layer inputs)."""
    r = bf16_round if bf16 else (lambda a: a)
    acts = [r(np.asarray(x, dtype=np.float64))]
    L = len(W)
    for l in range(L):
        z = acts[-1] @ r(W[l]).T + b[l]
        if l < L - 1:
            acts.append(r(np.maximum(z, 0.0)))
        else:
            return z, acts
    raise AssertionError


def loss(W, b, x, t, bf16=False):
    y, _ = forward(W, b, x, bf16)
    return float(np.mean((y - t) ** 2))


def gradients(W, b, x, t, bf16=False):
    """Gradients of the mean squared error w.r.t. every W_l and b_l."""
    r = bf16_round if bf16 else (lambda a: a)
    y, acts = forward(W, b, x, bf16)
    n, m = y.shape
    d = 2.0 * (y - t) / (n * m)  # dL/dy
    gW = [None] * len(W)
    gb = [None] * len(W)
    for l in range(len(W) - 1, -1, -1):
        dr = r(d)
        gW[l] = dr.T @ acts[l]
        gb[l] = d.sum(axis=0)
        if l > 0:
            d = (dr @ r(W[l])) * (acts[l] > 0)
    return gW, gb, float(np.mean((y - t) ** 2))


class Adam:
    def __init__(self, params, beta1=0.9, beta2=0.999, eps=1e-8):
        self.m = [np.zeros_like(p) for p in params]
        self.v = [np.zeros_like(p) for p in params]
        self.t = 0
        self.beta1, self.beta2, self.eps = beta1, beta2, eps

    def step(self, params, grads, lr):
        self.t += 1
        c1 = 1.0 - self.beta1 ** self.t
        c2 = 1.0 - self.beta2 ** self.t
        for p, g, m, v in zip(params, grads, self.m, self.v):
            m *= self.beta1
            m += (1.0 - self.beta1) * g
            v *= self.beta2
            v += (1.0 - self.beta2) * g * g
            p -= lr * (m / c1) / (np.sqrt(v / c2) + self.eps)


def drag_samples(sim, shell: float = 5.0):
    """Features and targets of every particle of an OracleSim, by their
    definition (see the library header): nodes at distance (R, R + shell]
    from the centre (minimum image; outside walls skipped), mean eps,
    (1 - eps)-weighted mean fluid velocity, slip, Reynolds number, density
    ratio; target = force / Stokes scale."""
    rho, u, eps = sim.fields()
    p = sim.particles()
    m, _ = sim.masses()
    dim = sim.dim
    nx, ny, nz = sim.shape
    tau = sim.tau
    nu = (tau - 0.5) / 3.0
    rho0 = sim.rho0
    wall = sim.wall_y
    Z, Y, X = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    coords = [X, Y, Z]
    feats = np.zeros((sim.np, 6))
    tgt = np.zeros((sim.np, 3))
    for k in range(sim.np):
        R = float(sim.radius[k])
        c = p["pos"][k]
        d2 = np.zeros(X.shape)
        for d in range(dim):
            r = coords[d] - c[d]
            if not (d == 1 and wall):
                L = (nx, ny, nz)[d]
                r = np.where(r > L / 2, r - L, np.where(r < -L / 2, r + L, r))
            d2 += r * r
        sel = (d2 > R * R) & (d2 <= (R + shell) ** 2)
        e = eps[sel]
        wgt = 1.0 - e
        us = np.array([(wgt * u[d][sel]).sum() / wgt.sum() if wgt.sum() > 0 else 0.0 for d in range(dim)]
                      + [0.0] * (3 - dim))
        slip = us - p["vel"][k]
        vol = 4.0 / 3.0 * np.pi * R ** 3 if dim == 3 else np.pi * R * R
        scale = 6 * np.pi * rho0 * nu * R if dim == 3 else 4 * np.pi * rho0 * nu
        feats[k] = [e.mean() if e.size else 0.0, slip[0], slip[1], slip[2],
                    np.linalg.norm(slip) * 2 * R / nu, m[k] / vol / rho0]
        tgt[k] = p["force"][k] / scale
    return feats, tgt
