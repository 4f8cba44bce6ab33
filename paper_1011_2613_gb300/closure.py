"""ctypes binding of the learned drag closure (lbm_imb_drag_samples and
lbm_imb_mlp_* in the C ABI).  Marshalling only: the sample extraction and the
network's forward, backward and Adam steps run in the library's kernels
(tcgen05 BF16 products, FP32 accumulation).  PyTorch provides the device
buffers and the stream."""
from __future__ import annotations

import ctypes as C

import numpy as np

from . import lbm as _lbm

_dp = C.POINTER(C.c_double)
_fp = C.POINTER(C.c_float)
_configured = False


def _lib():
    global _configured
    L = _lbm.lib()
    if not _configured:
        L.lbm_imb_drag_samples.restype = C.c_int
        L.lbm_imb_drag_samples.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_double, C.c_void_p, C.c_void_p,
                                           C.c_int64]
        L.lbm_imb_mlp_required_bytes.restype = C.c_size_t
        L.lbm_imb_mlp_required_bytes.argtypes = [C.c_int64]
        L.lbm_imb_mlp_init.restype = C.c_int
        L.lbm_imb_mlp_init.argtypes = [C.c_void_p, C.c_size_t, C.c_int64, C.c_uint64, C.c_void_p,
                                       C.POINTER(C.c_void_p)]
        L.lbm_imb_mlp_num_params.restype = C.c_int
        L.lbm_imb_mlp_num_params.argtypes = [C.POINTER(C.c_int)]
        for nm in ("lbm_imb_mlp_set_params", "lbm_imb_mlp_get_params"):
            getattr(L, nm).restype = C.c_int
            getattr(L, nm).argtypes = [C.c_void_p, C.c_void_p]
        L.lbm_imb_mlp_set_normalization.restype = C.c_int
        L.lbm_imb_mlp_set_normalization.argtypes = [C.c_void_p, _fp, _fp, _fp, _fp]
        L.lbm_imb_mlp_predict.restype = C.c_int
        L.lbm_imb_mlp_predict.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int64]
        L.lbm_imb_mlp_gradients.restype = C.c_int
        L.lbm_imb_mlp_gradients.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p]
        L.lbm_imb_mlp_train_steps.restype = C.c_int
        L.lbm_imb_mlp_train_steps.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int64, C.c_int64, C.c_int64,
                                              C.c_float, C.c_void_p]
        L.lbm_imb_mlp_destroy.restype = C.c_int
        L.lbm_imb_mlp_destroy.argtypes = [C.c_void_p]
        L.lbm_imb_mlp_probe_gemm.restype = C.c_int
        L.lbm_imb_mlp_probe_gemm.argtypes = [C.c_void_p, C.c_void_p, C.c_int, C.c_int, C.c_void_p, C.c_void_p,
                                             C.c_size_t, C.c_void_p]
        _configured = True
    return L


def drag_samples(sim, shell: float = 5.0):
    """Features (np,6) and targets (np,3), float32 CUDA tensors, of every
    particle of ``sim`` (a lbm.Simulation) in its current state."""
    import torch

    dev = sim.device
    u = torch.empty(sim.dim * sim.N, dtype=torch.float64, device=dev)
    eps = torch.empty(sim.N, dtype=torch.float64, device=dev)
    sim.fields_device(None, u, eps)
    n = max(sim.np, 1)
    feats = torch.empty((n, 6), dtype=torch.float32, device=dev)
    tgt = torch.empty((n, 3), dtype=torch.float32, device=dev)
    _lbm._check(_lib().lbm_imb_drag_samples(sim.h, C.c_void_p(u.data_ptr()), C.c_void_p(eps.data_ptr()),
                                            float(shell), C.c_void_p(feats.data_ptr()), C.c_void_p(tgt.data_ptr()),
                                            n), "lbm_imb_drag_samples")
    sim.sync()
    return feats[: sim.np], tgt[: sim.np]


def probe_gemm(a_bits: np.ndarray, b_bits: np.ndarray, device=None) -> np.ndarray:
    """One tcgen05 product D = A B^T of raw bfloat16 bit patterns (test hook)."""
    import torch

    a = np.ascontiguousarray(a_bits, dtype=np.uint16)
    b = np.ascontiguousarray(b_bits, dtype=np.uint16)
    K = a.shape[1]
    N = b.shape[0]
    assert a.shape[0] == 128 and b.shape[1] == K
    scratch = torch.empty(128 * 1024 + 512, dtype=torch.uint8, device=device or "cuda")
    ptr = (scratch.data_ptr() + 255) // 256 * 256
    d = np.zeros((128, N), dtype=np.float32)
    s = torch.cuda.current_stream()
    _lbm._check(_lib().lbm_imb_mlp_probe_gemm(C.c_void_p(a.ctypes.data), C.c_void_p(b.ctypes.data), N, K,
                                              C.c_void_p(d.ctypes.data), C.c_void_p(ptr), 128 * 1024 + 256,
                                              C.c_void_p(s.cuda_stream)), "lbm_imb_mlp_probe_gemm")
    return d


class MLP:
    """The drag-closure network in a caller-owned device block."""

    def __init__(self, max_batch: int = 8192, seed: int = 0, device=None, stream=None):
        import torch

        L = _lib()
        self.device = torch.device(device if device is not None else "cuda")
        nb = int(L.lbm_imb_mlp_required_bytes(int(max_batch)))
        if nb == 0:
            raise _lbm.LbmImbError(_lbm.EINVAL, "lbm_imb_mlp_required_bytes")
        with torch.cuda.device(self.device):
            self.stream = stream if stream is not None else torch.cuda.Stream(self.device)
            self.buf = torch.empty(nb + 256, dtype=torch.uint8, device=self.device)
            ptr = (self.buf.data_ptr() + 255) // 256 * 256
            h = C.c_void_p()
            st = L.lbm_imb_mlp_init(C.c_void_p(ptr), nb, int(max_batch), int(seed),
                                    C.c_void_p(self.stream.cuda_stream), C.byref(h))
        _lbm._check(st, "lbm_imb_mlp_init")
        self.h = h
        n = C.c_int()
        L.lbm_imb_mlp_num_params(C.byref(n))
        self.n_params = int(n.value)
        self.max_batch = int(max_batch)

    def close(self):
        if getattr(self, "h", None):
            _lib().lbm_imb_mlp_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _sync_inputs(self):
        import torch
        torch.cuda.current_stream(self.device).synchronize()

    def set_params(self, flat):
        p = np.ascontiguousarray(np.asarray(flat, dtype=np.float32))
        assert p.size == self.n_params
        _lbm._check(_lib().lbm_imb_mlp_set_params(self.h, C.c_void_p(p.ctypes.data)), "lbm_imb_mlp_set_params")

    def get_params(self) -> np.ndarray:
        p = np.zeros(self.n_params, dtype=np.float32)
        _lbm._check(_lib().lbm_imb_mlp_get_params(self.h, C.c_void_p(p.ctypes.data)), "lbm_imb_mlp_get_params")
        return p

    def set_normalization(self, x_mean, x_std, y_mean, y_std):
        a = [np.ascontiguousarray(np.asarray(v, dtype=np.float32)) for v in (x_mean, x_std, y_mean, y_std)]
        _lbm._check(_lib().lbm_imb_mlp_set_normalization(self.h, *[v.ctypes.data_as(_fp) for v in a]),
                    "lbm_imb_mlp_set_normalization")

    def predict(self, x):
        """x: float32 CUDA tensor (n,6) -> float32 CUDA tensor (n,3)."""
        import torch

        x = x.contiguous()
        y = torch.empty((x.shape[0], 3), dtype=torch.float32, device=x.device)
        self._sync_inputs()
        _lbm._check(_lib().lbm_imb_mlp_predict(self.h, C.c_void_p(x.data_ptr()), C.c_void_p(y.data_ptr()),
                                               x.shape[0]), "lbm_imb_mlp_predict")
        return y

    def gradients(self, x, t):
        g = np.zeros(self.n_params, dtype=np.float32)
        loss = np.zeros(1, dtype=np.float32)
        x, t = x.contiguous(), t.contiguous()
        self._sync_inputs()
        _lbm._check(_lib().lbm_imb_mlp_gradients(self.h, C.c_void_p(x.data_ptr()), C.c_void_p(t.data_ptr()),
                                                 x.shape[0], C.c_void_p(g.ctypes.data),
                                                 C.c_void_p(loss.ctypes.data)), "lbm_imb_mlp_gradients")
        return g, float(loss[0])

    def train(self, x, t, batch: int, steps: int, lr: float) -> float:
        loss = np.zeros(1, dtype=np.float32)
        x, t = x.contiguous(), t.contiguous()
        self._sync_inputs()
        _lbm._check(_lib().lbm_imb_mlp_train_steps(self.h, C.c_void_p(x.data_ptr()), C.c_void_p(t.data_ptr()),
                                                   x.shape[0], int(batch), int(steps), float(lr),
                                                   C.c_void_p(loss.ctypes.data)), "lbm_imb_mlp_train_steps")
        return float(loss[0])


def flat_to_layers(flat, sizes=(6, 128, 128, 128, 128, 3)):
    """Split the flat parameter vector into [W_l], [b_l] (float64)."""
    W, b = [], []
    k = 0
    for i in range(len(sizes) - 1):
        nw = sizes[i + 1] * sizes[i]
        W.append(np.asarray(flat[k:k + nw], dtype=np.float64).reshape(sizes[i + 1], sizes[i]))
        k += nw
        b.append(np.asarray(flat[k:k + sizes[i + 1]], dtype=np.float64))
        k += sizes[i + 1]
    return W, b


def layers_to_flat(W, b):
    return np.concatenate([np.concatenate([w.reshape(-1), bb]) for w, bb in zip(W, b)]).astype(np.float32)


# ---------------------------------------------------------------------------
# the closure experiment: samples from resolved runs, training, evaluation
# ---------------------------------------------------------------------------
def drag_dataset(phis, seeds, n=128, transient=2000, every=200, snapshots=10, shell=5.0, storage="f32dev"):
    """Resolved D3Q19 periodic suspensions at each solid fraction and seed;
    after ``transient`` steps, drag samples of every particle every ``every``
    steps, ``snapshots`` times.  Returns (features (S,6), targets (S,3),
    seed label (S,), phi label (S,)) as CUDA tensors / numpy labels, and the
    resolved cost in seconds per particle-step."""
    import time

    import torch

    from . import inputs as I
    from .lbm import Simulation

    feats, tgts, sl, pl = [], [], [], []
    t_steps = 0.0
    particle_steps = 0
    for phi in phis:
        for sd in seeds:
            cfg = I.closure_config(phi, sd, n=n, storage=storage)
            sim = Simulation(cfg)
            sim.step(transient)
            for _ in range(snapshots):
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                sim.step(every)
                sim.sync()
                t_steps += time.perf_counter() - t0
                particle_steps += every * cfg.n_particles
                f, t = drag_samples(sim, shell)
                feats.append(f.clone())
                tgts.append(t.clone())
                sl.append(np.full(cfg.n_particles, sd))
                pl.append(np.full(cfg.n_particles, phi))
            sim.close()
            del sim
    return (torch.cat(feats), torch.cat(tgts), np.concatenate(sl), np.concatenate(pl),
            t_steps / max(particle_steps, 1))


def wen_yu_fit(x, t):
    """Least-squares fit of a Wen-Yu-form drag law to the samples:
    F / (6 pi mu R) = s (1 - phi)^(-k) (1 + 0.15 Re^0.687) + c,
    with s the slip vector, fitting the voidage exponent k by a scan and the
    constant vector c (pressure-gradient part) by least squares.  Returns a
    predictor f(x) -> (n,3)."""
    x = np.asarray(x, dtype=np.float64)
    t = np.asarray(t, dtype=np.float64)
    phi, s, re = x[:, 0], x[:, 1:4], x[:, 4]
    base = (1.0 + 0.15 * np.power(np.maximum(re, 0.0), 0.687))[:, None] * s
    best = None
    for k in np.linspace(0.0, 6.0, 121):
        g = base * np.power(np.clip(1.0 - phi, 1e-3, 1.0), -k)[:, None]
        c = (t - g).mean(axis=0)
        err = np.sum((t - g - c) ** 2)
        if best is None or err < best[0]:
            best = (err, k, c)
    _, k, c = best

    def predict(xx):
        xx = np.asarray(xx, dtype=np.float64)
        gg = (1.0 + 0.15 * np.power(np.maximum(xx[:, 4], 0.0), 0.687))[:, None] * xx[:, 1:4]
        return gg * np.power(np.clip(1.0 - xx[:, 0], 1e-3, 1.0), -k)[:, None] + c

    predict.k = k
    predict.c = c
    return predict


def rel_error(pred, t) -> float:
    """|| pred - t || / || t || over all samples and components."""
    pred = np.asarray(pred, dtype=np.float64)
    t = np.asarray(t, dtype=np.float64)
    return float(np.linalg.norm(pred - t) / np.linalg.norm(t))


def train_closure(x, t, batch=8192, epochs=30, lr=1e-3, seed=0, max_batch=None):
    """Train the network on CUDA tensors x (S,6), t (S,3): normalisation from
    the training set (zero spreads replaced by 1), shuffled once, then
    consecutive minibatches.  Returns (mlp, seconds, last loss)."""
    import time

    import torch

    S = x.shape[0]
    g = torch.Generator(device="cpu").manual_seed(seed)
    perm = torch.randperm(S, generator=g).to(x.device)
    xs, ts = x[perm].contiguous(), t[perm].contiguous()
    xm, xsd = xs.mean(0).cpu().numpy(), xs.std(0).cpu().numpy()
    ym, ysd = ts.mean(0).cpu().numpy(), ts.std(0).cpu().numpy()
    xsd[xsd <= 1e-12] = 1.0
    ysd[ysd <= 1e-12] = 1.0
    mlp = MLP(max_batch=max_batch or batch, seed=seed)
    mlp.set_normalization(xm, xsd, ym, ysd)
    steps = max(1, epochs * S // batch)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    loss = mlp.train(xs, ts, batch=min(batch, S), steps=steps, lr=lr)
    torch.cuda.synchronize()
    return mlp, time.perf_counter() - t0, loss
