"""Thin ctypes binding over liblbm_imb.so (the C ABI in include/lbm_imb.h).

Argument marshalling only: every step of the method runs in the library's
CUDA kernels.  PyTorch supplies the device memory block (one uint8 tensor per
simulation) and the CUDA stream.  There is no CPU fallback: if the compiled
library is missing the first call raises.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

from . import inputs as _inputs

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "liblbm_imb.so")
_lock = threading.Lock()
_lib = None

_dp = C.POINTER(C.c_double)

OK, EINVAL, ENOMEM, ECUDA, ETIMEOUT, ENONFINITE, EUNSUPPORTED, EOWNERS, EBIN = 0, -1, -2, -3, -4, -5, -6, -7, -8
MAX_OWNERS = 4
# kernel families of one step, in the order of lbm_imb_step_profiled's array
KERNEL_FAMILIES = ("eps_clear", "eps_raster", "collide", "dem")


class LbmImbError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        msg = lib().lbm_imb_strerror(status).decode() if _lib is not None else str(status)
        super().__init__(f"{where}: {msg} (status {status})")


class Config(C.Structure):
    """Mirror of ``lbm_imb_config``."""

    _fields_ = [
        ("struct_size", C.c_uint32), ("dim", C.c_int32), ("nx", C.c_int32), ("ny", C.c_int32),
        ("nz", C.c_int32), ("wall_y", C.c_int32), ("storage", C.c_int32), ("tau", C.c_double),
        ("body_force", C.c_double * 3), ("gravity", C.c_double * 3), ("rho_fluid", C.c_double),
        ("k_n", C.c_double), ("restitution", C.c_double), ("dem_substeps", C.c_int32),
        ("eps_method", C.c_int32), ("n_particles", C.c_int64), ("pos", _dp), ("vel", _dp),
        ("omega", _dp), ("radius", _dp), ("density", _dp), ("dem_skin", C.c_double),
    ]


def lib():
    """Load liblbm_imb.so (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(
                    "liblbm_imb.so is not built; run `python -c \"import __graft_entry__ as g; g.build()\"`")
            L = C.CDLL(LIB_PATH)
            L.lbm_imb_required_bytes.restype = C.c_size_t
            L.lbm_imb_required_bytes.argtypes = [C.POINTER(Config)]
            L.lbm_imb_init.restype = C.c_int
            L.lbm_imb_init.argtypes = [C.POINTER(Config), C.c_void_p, C.c_size_t, C.c_void_p, C.POINTER(C.c_void_p)]
            L.lbm_imb_step.restype = C.c_int
            L.lbm_imb_step.argtypes = [C.c_void_p, C.c_int64]
            L.lbm_imb_step_profiled.restype = C.c_int
            L.lbm_imb_step_profiled.argtypes = [C.c_void_p, C.c_int64, _dp, _dp]
            L.lbm_imb_slabs_required_bytes.restype = C.c_size_t
            L.lbm_imb_slabs_required_bytes.argtypes = [C.POINTER(Config), C.c_int]
            L.lbm_imb_slabs_init.restype = C.c_int
            L.lbm_imb_slabs_init.argtypes = [C.POINTER(Config), C.c_int, C.c_void_p, C.c_size_t, C.c_void_p,
                                             C.POINTER(C.c_void_p)]
            L.lbm_imb_slab_member.restype = C.c_int
            L.lbm_imb_slab_member.argtypes = [C.c_void_p, C.c_int, C.POINTER(C.c_void_p)]
            L.lbm_imb_dem_rebuilds.restype = C.c_int
            L.lbm_imb_dem_rebuilds.argtypes = [C.c_void_p, C.POINTER(C.c_int64)]
            L.lbm_imb_launches_per_step.restype = C.c_int
            L.lbm_imb_launches_per_step.argtypes = [C.c_void_p, C.POINTER(C.c_int)]
            L.lbm_imb_set_collide_variant.restype = C.c_int
            L.lbm_imb_set_collide_variant.argtypes = [C.c_void_p, C.c_int]
            L.lbm_imb_sync.restype = C.c_int
            L.lbm_imb_sync.argtypes = [C.c_void_p]
            L.lbm_imb_particles.restype = C.c_int
            L.lbm_imb_particles.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                            C.c_int64]
            L.lbm_imb_set_particles.restype = C.c_int
            L.lbm_imb_set_particles.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int64]
            L.lbm_imb_fields.restype = C.c_int
            L.lbm_imb_fields.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int64, C.c_int]
            L.lbm_imb_get_populations.restype = C.c_int
            L.lbm_imb_get_populations.argtypes = [C.c_void_p, C.c_void_p, C.c_int64, C.c_int]
            L.lbm_imb_set_populations.restype = C.c_int
            L.lbm_imb_set_populations.argtypes = [C.c_void_p, C.c_void_p, C.c_int64, C.c_int]
            L.lbm_imb_totals.restype = C.c_int
            L.lbm_imb_totals.argtypes = [C.c_void_p, _dp, _dp, _dp]
            L.lbm_imb_set_health_check.restype = C.c_int
            L.lbm_imb_set_health_check.argtypes = [C.c_void_p, C.c_int64]
            L.lbm_imb_check_health.restype = C.c_int
            L.lbm_imb_check_health.argtypes = [C.c_void_p]
            L.lbm_imb_save.restype = C.c_int
            L.lbm_imb_save.argtypes = [C.c_void_p, C.c_char_p]
            L.lbm_imb_load.restype = C.c_int
            L.lbm_imb_load.argtypes = [C.c_void_p, C.c_char_p]
            L.lbm_imb_steps_done.restype = C.c_int
            L.lbm_imb_steps_done.argtypes = [C.c_void_p, C.POINTER(C.c_int64)]
            L.lbm_imb_dem_workspace_bytes.restype = C.c_size_t
            L.lbm_imb_dem_workspace_bytes.argtypes = [C.c_int32, C.POINTER(C.c_int32), C.c_int32, C.c_int64,
                                                      C.c_double]
            L.lbm_imb_dem_forces.restype = C.c_int
            L.lbm_imb_dem_forces.argtypes = [C.c_int32, C.POINTER(C.c_int32), C.c_int32, C.c_int64, C.c_double,
                                             C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_double,
                                             C.c_double, C.c_void_p, C.c_void_p, C.c_size_t, C.c_void_p]
            L.lbm_imb_dem_forces_static.restype = C.c_int
            L.lbm_imb_dem_forces_static.argtypes = [C.c_int32, C.POINTER(C.c_int32), C.c_int32, C.c_int64,
                                                    C.c_double, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                                    C.c_double, C.c_double, C.c_void_p, C.c_void_p]
            L.lbm_imb_batch_required_bytes.restype = C.c_size_t
            L.lbm_imb_batch_required_bytes.argtypes = [C.POINTER(Config), C.c_int]
            L.lbm_imb_batch_init.restype = C.c_int
            L.lbm_imb_batch_init.argtypes = [C.POINTER(Config), C.c_int, C.c_int, C.c_int, C.c_void_p, C.c_size_t,
                                             C.c_void_p, C.POINTER(C.c_void_p)]
            L.lbm_imb_batch_member.restype = C.c_int
            L.lbm_imb_batch_member.argtypes = [C.c_void_p, C.c_int, C.POINTER(C.c_void_p)]
            L.lbm_imb_batch_size.restype = C.c_int
            L.lbm_imb_batch_size.argtypes = [C.c_void_p, C.POINTER(C.c_int)]
            L.lbm_imb_batch_set_launch.restype = C.c_int
            L.lbm_imb_batch_set_launch.argtypes = [C.c_void_p, C.c_int, C.c_int]
            L.lbm_imb_batch_get_launch.restype = C.c_int
            L.lbm_imb_batch_get_launch.argtypes = [C.c_void_p, C.POINTER(C.c_int), C.POINTER(C.c_int)]
            L.lbm_imb_batch_set_barrier_test.restype = C.c_int
            L.lbm_imb_batch_set_barrier_test.argtypes = [C.c_void_p, C.c_int64, C.c_int]
            L.lbm_imb_probe_fp64_rate.restype = C.c_int
            L.lbm_imb_probe_fp64_rate.argtypes = [C.c_void_p, C.c_int64, C.c_int64, C.c_int, _dp, _dp, C.c_void_p]
            L.lbm_imb_probe_df.restype = C.c_int
            L.lbm_imb_probe_df.argtypes = [C.c_void_p] * 5 + [C.c_int64, C.c_void_p]
            L.lbm_imb_probe_atan2q1.restype = C.c_int
            L.lbm_imb_probe_atan2q1.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int64,
                                                C.c_void_p]
            L.lbm_imb_destroy.restype = C.c_int
            L.lbm_imb_destroy.argtypes = [C.c_void_p]
            L.lbm_imb_strerror.restype = C.c_char_p
            L.lbm_imb_strerror.argtypes = [C.c_int]
            L.lbm_imb_version.restype = C.c_char_p
            L.lbm_imb_version.argtypes = []
            _lib = L
    return _lib


def _check(status: int, where: str):
    if status != OK:
        raise LbmImbError(status, where)


def _arr(x, n3=False):
    a = np.ascontiguousarray(np.asarray(x, dtype=np.float64))
    return a


def make_config(cfg) -> tuple[Config, list]:
    """Build the C struct from a SuspensionConfig-like object.  Returns the
    struct and the list of numpy arrays it points into (keep it alive)."""
    keep = []
    np_ = int(len(cfg.radius))

    def ptr(a):
        a = np.ascontiguousarray(np.asarray(a, dtype=np.float64).reshape(-1))
        keep.append(a)
        return a.ctypes.data_as(_dp)

    c = Config()
    c.struct_size = C.sizeof(Config)
    c.dim = int(cfg.dim)
    c.nx, c.ny = int(cfg.nx), int(cfg.ny)
    c.nz = int(cfg.nz) if int(cfg.dim) == 3 else 1
    c.wall_y = int(cfg.wall_y)
    st = getattr(cfg, "storage", "f64")
    c.storage = _inputs.STORAGE[st] if isinstance(st, str) else int(st)
    c.tau = float(cfg.tau)
    for d in range(3):
        c.body_force[d] = float(np.asarray(cfg.body_force, dtype=np.float64)[d])
        c.gravity[d] = float(np.asarray(cfg.gravity, dtype=np.float64)[d])
    c.rho_fluid = float(cfg.rho_fluid)
    c.k_n = float(cfg.k_n)
    c.restitution = float(cfg.restitution)
    c.dem_substeps = int(cfg.dem_substeps)
    c.eps_method = int(getattr(cfg, "eps_method", 0))
    c.dem_skin = float(getattr(cfg, "dem_skin", 0.0))
    c.n_particles = np_
    if np_:
        c.pos = ptr(cfg.pos)
        c.vel = ptr(cfg.vel)
        c.omega = ptr(cfg.omega)
        c.radius = ptr(cfg.radius)
        c.density = ptr(cfg.density)
    return c, keep


def required_bytes(cfg) -> int:
    c, _keep = make_config(cfg)
    return int(lib().lbm_imb_required_bytes(C.byref(c)))


class Simulation:
    """One suspension advanced on the GPU by liblbm_imb (or a member view of
    a :class:`Batch`).

    ``cfg``: :class:`paper_1011_2613_gb300.inputs.SuspensionConfig`.
    ``stream``: a ``torch.cuda.Stream`` (a new one by default; its graphs are
    captured on it)."""

    def __init__(self, cfg, device=None, stream=None):
        import torch

        L = lib()
        self.cfg = cfg
        self.dim = int(cfg.dim)
        self.shape = (int(cfg.nx), int(cfg.ny), int(cfg.nz) if self.dim == 3 else 1)
        self.N = self.shape[0] * self.shape[1] * self.shape[2]
        self.Q = 9 if self.dim == 2 else 19
        self.np = int(len(cfg.radius))
        self.device = torch.device(device if device is not None else "cuda")
        c, keep = make_config(cfg)
        nbytes = int(L.lbm_imb_required_bytes(C.byref(c)))
        if nbytes == 0:  # the configuration is rejected: report why
            h0 = C.c_void_p()
            _check(L.lbm_imb_init(C.byref(c), None, 0, None, C.byref(h0)), "lbm_imb_init")
            raise LbmImbError(EINVAL, "lbm_imb_required_bytes")
        self.nbytes = nbytes
        with torch.cuda.device(self.device):
            self.stream = stream if stream is not None else torch.cuda.Stream(self.device)
            self.buf = torch.empty(nbytes + 256, dtype=torch.uint8, device=self.device)
            base = self.buf.data_ptr()
            ptr = (base + 255) // 256 * 256
            h = C.c_void_p()
            st = L.lbm_imb_init(C.byref(c), C.c_void_p(ptr), nbytes, C.c_void_p(self.stream.cuda_stream),
                                C.byref(h))
        del keep
        _check(st, "lbm_imb_init")
        self.h = h

    # ------------------------------------------------------------------
    @classmethod
    def _member(cls, batch, i, cfg, accessor="lbm_imb_batch_member"):
        self = cls.__new__(cls)
        self.cfg = cfg
        self.dim = int(cfg.dim)
        self.shape = (int(cfg.nx), int(cfg.ny), int(cfg.nz) if self.dim == 3 else 1)
        self.N = self.shape[0] * self.shape[1] * self.shape[2]
        self.Q = 9 if self.dim == 2 else 19
        self.np = int(len(cfg.radius))
        self.device = batch.device
        self.stream = batch.stream
        self.batch = batch  # keeps the batch (and its memory) alive
        h = C.c_void_p()
        _check(getattr(lib(), accessor)(batch.h, i, C.byref(h)), accessor)
        self.h = h
        self._member_of = batch
        return self

    def close(self):
        if getattr(self, "_member_of", None) is not None:
            self.h = None
            return
        if getattr(self, "h", None):
            lib().lbm_imb_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def step(self, n: int = 1):
        _check(lib().lbm_imb_step(self.h, int(n)), "lbm_imb_step")

    def step_profiled(self, n: int):
        """Run n steps with CUDA events between kernel families; returns
        (per-family ms dict, total ms)."""
        k = (C.c_double * len(KERNEL_FAMILIES))()
        t = C.c_double()
        _check(lib().lbm_imb_step_profiled(self.h, int(n), k, C.byref(t)), "lbm_imb_step_profiled")
        names = KERNEL_FAMILIES
        return {nm: float(k[i]) for i, nm in enumerate(names)}, float(t.value)

    def set_collide_variant(self, variant: int):
        _check(lib().lbm_imb_set_collide_variant(self.h, int(variant)), "lbm_imb_set_collide_variant")

    def dem_rebuilds(self) -> int:
        """Verlet-list builds so far (dem_skin > 0)."""
        b = C.c_int64()
        _check(lib().lbm_imb_dem_rebuilds(self.h, C.byref(b)), "lbm_imb_dem_rebuilds")
        return int(b.value)

    def launches_per_step(self) -> int:
        x = C.c_int()
        _check(lib().lbm_imb_launches_per_step(self.h, C.byref(x)), "lbm_imb_launches_per_step")
        return int(x.value)

    def sync(self):
        _check(lib().lbm_imb_sync(self.h), "lbm_imb_sync")

    def set_health_check(self, every: int):
        """Steps between the health checks of step() (0: off)."""
        _check(lib().lbm_imb_set_health_check(self.h, int(every)), "lbm_imb_set_health_check")

    def check_health(self):
        """Scan the stored state for NaN/Inf now (raises LbmImbError with
        status ENONFINITE if found)."""
        _check(lib().lbm_imb_check_health(self.h), "lbm_imb_check_health")

    def save(self, path):
        """Checkpoint the simulation to a file (lbm_imb_save)."""
        _check(lib().lbm_imb_save(self.h, os.fsencode(path)), "lbm_imb_save")

    def load(self, path):
        """Resume from a checkpoint of the same configuration (lbm_imb_load)."""
        _check(lib().lbm_imb_load(self.h, os.fsencode(path)), "lbm_imb_load")

    def steps_done(self) -> int:
        s = C.c_int64()
        _check(lib().lbm_imb_steps_done(self.h, C.byref(s)), "lbm_imb_steps_done")
        return int(s.value)

    def particles(self, out=None):
        """dict of (np,3) float64 arrays: pos, vel, omega, force, torque
        (force/torque = hydrodynamic, Eq. 3, of the last step)."""
        n3 = 3 * max(self.np, 1)
        a = out if out is not None else {k: np.zeros(n3) for k in ("pos", "vel", "omega", "force", "torque")}
        p = [a[k].ctypes.data if a.get(k) is not None else None for k in ("pos", "vel", "omega", "force", "torque")]
        _check(lib().lbm_imb_particles(self.h, *[C.c_void_p(x) if x else None for x in p], max(self.np, 1)),
               "lbm_imb_particles")
        if out is not None:
            return out
        return {k: v[: 3 * self.np].reshape(self.np, 3) for k, v in a.items()}

    def set_particles(self, pos=None, vel=None, omega=None):
        arrs = [None if x is None else np.ascontiguousarray(np.asarray(x, dtype=np.float64).reshape(-1))
                for x in (pos, vel, omega)]
        _check(lib().lbm_imb_set_particles(self.h, *[None if a is None else C.c_void_p(a.ctypes.data) for a in arrs],
                                           self.np), "lbm_imb_set_particles")

    def fields(self):
        """(rho (nz,ny,nx), u (dim,nz,ny,nx), eps (nz,ny,nx)) as numpy."""
        rho = np.zeros(self.N)
        u = np.zeros(self.dim * self.N)
        eps = np.zeros(self.N)
        _check(lib().lbm_imb_fields(self.h, C.c_void_p(rho.ctypes.data), C.c_void_p(u.ctypes.data),
                                    C.c_void_p(eps.ctypes.data), self.N, 0), "lbm_imb_fields")
        nx, ny, nz = self.shape
        return rho.reshape(nz, ny, nx), u.reshape(self.dim, nz, ny, nx), eps.reshape(nz, ny, nx)

    def fields_device(self, rho, u, eps):
        """Write the fields into caller-owned float64 CUDA tensors (any may be None)."""
        ptrs = [C.c_void_p(t.data_ptr()) if t is not None else None for t in (rho, u, eps)]
        _check(lib().lbm_imb_fields(self.h, *ptrs, self.N, 1), "lbm_imb_fields")

    def populations(self) -> np.ndarray:
        """Stored post-collision populations as FP64, shape (Q, nz, ny, nx)."""
        f = np.zeros(self.Q * self.N)
        _check(lib().lbm_imb_get_populations(self.h, C.c_void_p(f.ctypes.data), f.size, 0),
               "lbm_imb_get_populations")
        nx, ny, nz = self.shape
        return f.reshape(self.Q, nz, ny, nx)

    def set_populations(self, f):
        f = np.ascontiguousarray(np.asarray(f, dtype=np.float64).reshape(-1))
        assert f.size == self.Q * self.N
        _check(lib().lbm_imb_set_populations(self.h, C.c_void_p(f.ctypes.data), f.size, 0),
               "lbm_imb_set_populations")

    def totals(self):
        m = C.c_double()
        jf = (C.c_double * 3)()
        jp = (C.c_double * 3)()
        _check(lib().lbm_imb_totals(self.h, C.byref(m), jf, jp), "lbm_imb_totals")
        return float(m.value), np.array(list(jf)), np.array(list(jp))


def dem_forces(dim, extent, wall_y, pos, vel, radius, mass, k_n, restitution, rmax=None, stream=None):
    """Contact forces (Eqs. 4-5) of particles held in float64 CUDA tensors
    (pos/vel (n,3), radius/mass (n,)); returns a new (n,3) CUDA tensor.  The
    workspace is a torch uint8 tensor sized by lbm_imb_dem_workspace_bytes."""
    import torch

    n = int(radius.numel())
    rmax = float(radius.max().item()) if rmax is None else float(rmax)
    ext = (C.c_int32 * 3)(*[int(x) for x in (list(extent) + [1, 1])[:3]])
    nb = int(lib().lbm_imb_dem_workspace_bytes(int(dim), ext, int(wall_y), n, rmax))
    if nb == 0:
        raise LbmImbError(EINVAL, "lbm_imb_dem_workspace_bytes")
    ws = torch.empty(nb + 256, dtype=torch.uint8, device=radius.device)
    wp = (ws.data_ptr() + 255) // 256 * 256
    fc = torch.empty((n, 3), dtype=torch.float64, device=radius.device)
    s = stream if stream is not None else torch.cuda.current_stream(radius.device)
    st = lib().lbm_imb_dem_forces(int(dim), ext, int(wall_y), n, rmax, C.c_void_p(pos.data_ptr()),
                                  C.c_void_p(vel.data_ptr()), C.c_void_p(radius.data_ptr()),
                                  C.c_void_p(mass.data_ptr()), float(k_n), float(restitution),
                                  C.c_void_p(fc.data_ptr()), C.c_void_p(wp), nb, C.c_void_p(s.cuda_stream))
    _check(st, "lbm_imb_dem_forces")
    return fc


class Batch:
    """Many independent suspensions advanced by one persistent kernel launch
    per step (lbm_imb_batch_* in the C ABI).  ``members[i]`` gives the
    accessors of suspension i."""

    def __init__(self, cfgs, tile_x=0, blocks_per_sm=0, device=None, stream=None):
        import torch

        L = lib()
        self.cfgs = list(cfgs)
        n = len(self.cfgs)
        arr = (Config * n)()
        keeps = []
        for i, cfg in enumerate(self.cfgs):
            c, keep = make_config(cfg)
            arr[i] = c
            keeps.append(keep)
        nbytes = int(L.lbm_imb_batch_required_bytes(arr, n))
        if nbytes == 0:  # a configuration is rejected: report why
            h0 = C.c_void_p()
            _check(L.lbm_imb_batch_init(arr, n, 0, 0, None, 0, None, C.byref(h0)), "lbm_imb_batch_init")
            raise LbmImbError(EINVAL, "lbm_imb_batch_required_bytes")
        self.nbytes = nbytes
        self.device = torch.device(device if device is not None else "cuda")
        with torch.cuda.device(self.device):
            self.stream = stream if stream is not None else torch.cuda.Stream(self.device)
            self.buf = torch.empty(nbytes + 256, dtype=torch.uint8, device=self.device)
            ptr = (self.buf.data_ptr() + 255) // 256 * 256
            h = C.c_void_p()
            st = L.lbm_imb_batch_init(arr, n, int(tile_x), int(blocks_per_sm), C.c_void_p(ptr), nbytes,
                                      C.c_void_p(self.stream.cuda_stream), C.byref(h))
        del keeps
        _check(st, "lbm_imb_batch_init")
        self.h = h
        self.members = [Simulation._member(self, i, cfg) for i, cfg in enumerate(self.cfgs)]
        self.n_nodes = sum(m.N for m in self.members)

    def close(self):
        if getattr(self, "h", None):
            for m in self.members:
                m.h = None
            lib().lbm_imb_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def step(self, n: int = 1):
        _check(lib().lbm_imb_step(self.h, int(n)), "lbm_imb_step")

    def sync(self):
        _check(lib().lbm_imb_sync(self.h), "lbm_imb_sync")

    def step_profiled(self, n: int):
        k = (C.c_double * len(KERNEL_FAMILIES))()
        t = C.c_double()
        _check(lib().lbm_imb_step_profiled(self.h, int(n), k, C.byref(t)), "lbm_imb_step_profiled")
        return float(t.value)

    def set_launch(self, tile_x: int, blocks_per_sm: int):
        _check(lib().lbm_imb_batch_set_launch(self.h, int(tile_x), int(blocks_per_sm)), "lbm_imb_batch_set_launch")

    def launch(self):
        tx = C.c_int()
        g = C.c_int()
        _check(lib().lbm_imb_batch_get_launch(self.h, C.byref(tx), C.byref(g)), "lbm_imb_batch_get_launch")
        return int(tx.value), int(g.value)

    def set_barrier_test(self, spin_limit: int, phantom: int):
        _check(lib().lbm_imb_batch_set_barrier_test(self.h, int(spin_limit), int(phantom)),
               "lbm_imb_batch_set_barrier_test")


def probe_atan2q1(y, x):
    """The library's first-quadrant atan2 (FP64 rasterisation) and CUDA's
    atan2 on device tensors y, x (float64, same shape); returns (fast, ref)."""
    import torch
    y = y.contiguous()
    x = x.contiguous()
    fast = torch.empty_like(y)
    ref = torch.empty_like(y)
    s = torch.cuda.current_stream(y.device)
    _check(lib().lbm_imb_probe_atan2q1(y.data_ptr(), x.data_ptr(), fast.data_ptr(), ref.data_ptr(), y.numel(),
                                        s.cuda_stream), "lbm_imb_probe_atan2q1")
    return fast, ref


def probe_df(h, l, d):
    """FP64 <-> FP32-pair conversions of the double-FP32 storage on device
    tensors: h, l float32 (the pairs), d float64 (same length); returns
    (FP64 value of each pair, d split and converted back)."""
    import torch
    h, l, d = h.contiguous(), l.contiguous(), d.contiguous()
    to_double = torch.empty(h.numel(), dtype=torch.float64, device=h.device)
    roundtrip = torch.empty(d.numel(), dtype=torch.float64, device=d.device)
    if h.numel() != d.numel() or l.numel() != h.numel():
        raise ValueError("h, l and d must have the same length")
    s = torch.cuda.current_stream(h.device)
    _check(lib().lbm_imb_probe_df(h.data_ptr(), l.data_ptr(), d.data_ptr(), to_double.data_ptr(),
                                  roundtrip.data_ptr(), h.numel(), s.cuda_stream), "lbm_imb_probe_df")
    return to_double, roundtrip


FP64_KINDS = {"fma": 0, "add": 1, "mul": 2}


def probe_fp64_rate(kind: str = "fma", trips: int = 2400, blocks_per_sm: int = 8, device=None):
    """Measured FP64 throughput of this GPU for one instruction kind ("fma",
    "add", "mul"; G instructions/s) and the timed launch's ms (test hook)."""
    import torch
    dev = torch.device(device if device is not None else "cuda")
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    n = sms * blocks_per_sm * 256
    sink = torch.empty(n, dtype=torch.float64, device=dev)
    g, ms = C.c_double(), C.c_double()
    s = torch.cuda.current_stream(dev)
    _check(lib().lbm_imb_probe_fp64_rate(C.c_void_p(sink.data_ptr()), n, int(trips), FP64_KINDS[kind], C.byref(g),
                                         C.byref(ms), C.c_void_p(s.cuda_stream)), "lbm_imb_probe_fp64_rate")
    return float(g.value), float(ms.value)


def slab_rows(ny: int, nslabs: int):
    """(first global row, computed rows) of each y slab: ny split as evenly as
    possible, the first ny % nslabs slabs one row more."""
    base, rem = divmod(int(ny), int(nslabs))
    out, y = [], 0
    for k in range(nslabs):
        n = base + (1 if k < rem else 0)
        out.append((y, n))
        y += n
    return out


class Slabs:
    """One suspension decomposed along y into ``nslabs`` slabs with halo
    exchange after every collision (lbm_imb_slabs_* in the C ABI).  The
    particles are shared; ``members[k]`` gives slab k's local lattice (its
    computed rows between two halo rows)."""

    def __init__(self, cfg, nslabs: int, device=None, stream=None):
        import torch

        L = lib()
        self.cfg = cfg
        self.nslabs = int(nslabs)
        c, keep = make_config(cfg)
        nbytes = int(L.lbm_imb_slabs_required_bytes(C.byref(c), self.nslabs))
        if nbytes == 0:  # the configuration is rejected: report why
            h0 = C.c_void_p()
            _check(L.lbm_imb_slabs_init(C.byref(c), self.nslabs, None, 0, None, C.byref(h0)), "lbm_imb_slabs_init")
            raise LbmImbError(EINVAL, "lbm_imb_slabs_required_bytes")
        self.nbytes = nbytes
        self.device = torch.device(device if device is not None else "cuda")
        with torch.cuda.device(self.device):
            self.stream = stream if stream is not None else torch.cuda.Stream(self.device)
            self.buf = torch.empty(nbytes + 256, dtype=torch.uint8, device=self.device)
            ptr = (self.buf.data_ptr() + 255) // 256 * 256
            h = C.c_void_p()
            st = L.lbm_imb_slabs_init(C.byref(c), self.nslabs, C.c_void_p(ptr), nbytes,
                                      C.c_void_p(self.stream.cuda_stream), C.byref(h))
        del keep
        _check(st, "lbm_imb_slabs_init")
        self.h = h
        self.dim = int(cfg.dim)
        self.np = int(len(cfg.radius))
        self.Q = 9 if self.dim == 2 else 19
        self.shape = (int(cfg.nx), int(cfg.ny), int(cfg.nz) if self.dim == 3 else 1)
        self.N = self.shape[0] * self.shape[1] * self.shape[2]
        self.rows = slab_rows(cfg.ny, self.nslabs)
        self.members = [Simulation._member(self, k, cfg.replace(ny=n + 2), "lbm_imb_slab_member")
                        for k, (_, n) in enumerate(self.rows)]

    def close(self):
        if getattr(self, "h", None):
            for m in self.members:
                m.h = None
            lib().lbm_imb_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def step(self, n: int = 1):
        _check(lib().lbm_imb_step(self.h, int(n)), "lbm_imb_step")

    def sync(self):
        _check(lib().lbm_imb_sync(self.h), "lbm_imb_sync")

    particles = Simulation.particles

    def populations(self) -> np.ndarray:
        """The whole lattice's populations (Q, nz, ny, nx), assembled from the
        slabs' computed rows."""
        parts = [m.populations()[:, :, 1:n + 1, :] for m, (_, n) in zip(self.members, self.rows)]
        return np.concatenate(parts, axis=2)
