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
