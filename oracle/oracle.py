"""ctypes wrapper around the FP64 CPU oracle (``lbm_oracle.c``).

TEST INFRASTRUCTURE ONLY: tests, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` use this module to check and time the CUDA
library.  The product package never imports it.

``OracleSim`` mirrors the call shape of the CUDA binding (``step``,
``particles``, ``fields``, ``populations``) so that a test can drive both with
the same seeded inputs.  Each function states the part of the method it
follows (Xiong et al., section "Numerical scheme", Eqs. 1-5).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lbm_oracle.c")
_LIB = os.path.join(_HERE, "liblbm_oracle.so")
# timing build: the same source with OpenMP (loops over nodes and particles
# on all host cores; forces summed atomically), used only to time the oracle
_LIB_OMP = os.path.join(_HERE, "liblbm_oracle_omp.so")
_lock = threading.Lock()
_lib = None
_lib_omp = None

# -ffp-contract=off: no fused multiply-add contraction, so that the oracle's
# rounding is the plain IEEE sequence of the source on x86 and on Arm alike.
CFLAGS = ["-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared"]


def build(force: bool = False) -> str:
    """Compile the oracle shared library next to its source (gcc)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", *CFLAGS, "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def build_timing(force: bool = False):
    """Compile the OpenMP timing build of the oracle; returns its path, or
    None if the compiler has no OpenMP (the timing then uses one core)."""
    if force or not os.path.exists(_LIB_OMP) or os.path.getmtime(_LIB_OMP) < os.path.getmtime(_SRC):
        tmp = _LIB_OMP + ".tmp%d" % os.getpid()
        try:
            subprocess.check_call(["gcc", *CFLAGS, "-fopenmp", "-o", tmp, _SRC, "-lm"],
                                  stdout=subprocess.DEVNULL, stderr=subprocess.DEVNULL)
        except (subprocess.CalledProcessError, OSError):
            return None
        os.replace(tmp, _LIB_OMP)
    return _LIB_OMP


def timing_threads() -> int:
    """Threads the OpenMP timing build uses (OMP_NUM_THREADS, else the
    host's cores), or 1 without that build."""
    if build_timing() is None:
        return 1
    n = os.environ.get("OMP_NUM_THREADS")
    return int(n) if n and n.isdigit() else (os.cpu_count() or 1)


_dp = C.POINTER(C.c_double)
_ip = C.POINTER(C.c_int)


def _load(timing: bool = False):
    """The parity build (default) or the OpenMP timing build."""
    global _lib, _lib_omp
    with _lock:
        if timing:
            if _lib_omp is None:
                path = build_timing()
                _lib_omp = _declare(C.CDLL(path)) if path else None
            if _lib_omp is not None:
                return _lib_omp
        if _lib is None:
            _lib = _declare(C.CDLL(build()))
    return _lib


def _declare(lib):
    """Argument and result types of the oracle's C functions."""
    lib.oracle_area_disk_rect.restype = C.c_double
    lib.oracle_area_disk_rect.argtypes = [C.c_double] * 7
    lib.oracle_volume_ball_box.restype = C.c_double
    lib.oracle_volume_ball_box.argtypes = [C.c_double] * 10
    lib.oracle_cell_fraction.restype = C.c_double
    lib.oracle_cell_fraction.argtypes = [C.c_int] + [C.c_double] * 7
    lib.oracle_set_eps_table.restype = C.c_int
    lib.oracle_set_eps_table.argtypes = [C.c_void_p]
    lib.oracle_eps_table_value.restype = C.c_double
    lib.oracle_eps_table_value.argtypes = [C.c_void_p, C.c_double, C.c_double, C.c_double]
    lib.oracle_collide_node.restype = C.c_double
    lib.oracle_collide_node.argtypes = [C.c_int, C.c_double, _dp, _dp, C.c_int, _dp, _dp, _dp, _dp]
    lib.oracle_dem_advance.restype = None
    lib.oracle_dem_advance.argtypes = [C.c_int, _ip, C.c_int, C.c_int, _dp, _dp, _dp, _dp, _dp, _dp,
                                       _dp, _dp, _dp, C.c_double, C.c_double, C.c_int, _dp]
    lib.oracle_dem_contacts.restype = None
    lib.oracle_dem_contacts.argtypes = [C.c_int, _ip, C.c_int, C.c_int, _dp, _dp, _dp, _dp, C.c_double,
                                        C.c_double, _dp]
    lib.oracle_create.restype = C.c_void_p
    lib.oracle_create.argtypes = [C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, C.c_double, _dp, _dp,
                                  C.c_double, C.c_double, C.c_double, C.c_int, C.c_int,
                                  _dp, _dp, _dp, _dp, _dp]
    lib.oracle_destroy.argtypes = [C.c_void_p]
    lib.oracle_step.restype = C.c_int
    lib.oracle_step.argtypes = [C.c_void_p, C.c_int]
    lib.oracle_rasterize.restype = C.c_int
    lib.oracle_rasterize.argtypes = [C.c_void_p]
    lib.oracle_num_nodes.restype = C.c_long
    lib.oracle_num_nodes.argtypes = [C.c_void_p]
    lib.oracle_num_dirs.restype = C.c_int
    lib.oracle_num_dirs.argtypes = [C.c_void_p]
    lib.oracle_get_populations.argtypes = [C.c_void_p, _dp]
    lib.oracle_set_populations.argtypes = [C.c_void_p, _dp]
    lib.oracle_get_particles.argtypes = [C.c_void_p, _dp, _dp, _dp, _dp, _dp, _dp]
    lib.oracle_get_mass.argtypes = [C.c_void_p, _dp, _dp]
    lib.oracle_fields.argtypes = [C.c_void_p, _dp, _dp, _dp]
    lib.oracle_get_owners.argtypes = [C.c_void_p, _ip, _ip, _dp, C.c_int]
    return lib


def _p(a):
    return a.ctypes.data_as(_dp)


def _f64(a, n=None):
    a = np.ascontiguousarray(np.asarray(a, dtype=np.float64))
    if n is not None:
        assert a.size == n
    return a


# ---------------------------------------------------------------------------
# eps: covered area / volume of a lattice cell (the definition of the solid
# fraction; text following the Omega^S equation).
# ---------------------------------------------------------------------------
def area_disk_rect(cx, cy, R, x0, x1, y0, y1) -> float:
    """Exact area of disk(cx, cy; R) n [x0,x1]x[y0,y1]."""
    return _load().oracle_area_disk_rect(cx, cy, R, x0, x1, y0, y1)


def volume_ball_box(cx, cy, cz, R, x0, x1, y0, y1, z0, z1) -> float:
    """Volume of ball(c; R) n box, integral of exact slice areas."""
    return _load().oracle_volume_ball_box(cx, cy, cz, R, x0, x1, y0, y1, z0, z1)


def cell_fraction(dim, center, R, node) -> float:
    """Covered fraction of the unit cell centred on integer node coordinates."""
    c = list(center) + [0.0] * (3 - len(center))
    n = list(node) + [0] * (3 - len(node))
    return _load().oracle_cell_fraction(dim, c[0], c[1], c[2], R, n[0], n[1], n[2])


# ---------------------------------------------------------------------------
# One-node IMB collision (Eqs. 1-2 and the Omega^S term).
# ---------------------------------------------------------------------------
def collide_node(dim, tau, g, ft, eps_list=(), vs_list=()):
    """Returns (f_out, m, beta): post-collision populations, the momentum
    beta * sum_i Omega_i^S c_i given to the fluid, and beta."""
    Q = 9 if dim == 2 else 19
    ft = _f64(ft, Q)
    g = _f64(list(g) + [0.0] * (3 - len(g)))
    e = _f64(list(eps_list) if len(eps_list) else [0.0])
    vs = _f64(np.asarray(vs_list, dtype=np.float64).reshape(-1) if len(vs_list) else np.zeros(3))
    fo = np.zeros(Q)
    m = np.zeros(3)
    beta = _load().oracle_collide_node(dim, tau, _p(g), _p(ft), len(eps_list), _p(e), _p(vs), _p(fo), _p(m))
    return fo, m, beta


def dem_advance(dim, n, wall_y, pos, vel, omg, rad, mass, inertia, ff, tf, gs, kn, e, substeps=1):
    """Advance particle state one lattice step (Eqs. 4-5 with reading R7); in place."""
    np_ = len(rad)
    Ld = (C.c_int * 3)(*(list(n) + [1] * (3 - len(n))))
    fc = np.zeros(3 * max(np_, 1))
    _load().oracle_dem_advance(dim, Ld, int(wall_y), np_, _p(pos), _p(vel), _p(omg), _p(_f64(rad)),
                               _p(_f64(mass)), _p(_f64(inertia)), _p(_f64(ff)), _p(_f64(tf)),
                               _p(_f64(gs)), kn, e, substeps, _p(fc))
    return fc[: 3 * np_].reshape(np_, 3)


def dem_contacts(dim, n, wall_y, pos, vel, rad, mass, kn, e):
    """Contact forces (np,3) of the given state (Eqs. 4-5 with reading R7)."""
    np_ = len(rad)
    Ld = (C.c_int * 3)(*(list(n) + [1] * (3 - len(n))))
    fc = np.zeros(3 * max(np_, 1))
    _load().oracle_dem_contacts(dim, Ld, int(wall_y), np_, _p(_f64(pos)), _p(_f64(vel)), _p(_f64(rad)),
                                _p(_f64(mass)), kn, e, _p(fc))
    return fc[: 3 * np_].reshape(np_, 3)


# ---------------------------------------------------------------------------
# Whole simulation.
# ---------------------------------------------------------------------------
class OracleSim:
    """FP64 CPU LB-IMB-DEM simulation with the library's call shape.

    ``cfg`` is a :class:`paper_1011_2613_gb300.inputs.SuspensionConfig`-like
    object (attributes dim, nx, ny, nz, wall_y, tau, body_force, gravity,
    rho_fluid, k_n, restitution, dem_substeps, pos, vel, omega, radius,
    density)."""

    def __init__(self, cfg, timing: bool = False):
        """timing = True: the OpenMP timing build (all host cores, forces
        summed atomically; for timing only, never for parity)."""
        lib = _load(timing)
        self._lib = lib
        self.dim = int(cfg.dim)
        self.shape = (int(cfg.nx), int(cfg.ny), int(cfg.nz) if self.dim == 3 else 1)
        self.np = len(cfg.radius)
        npa = max(self.np, 1)
        self._keep = [
            _f64(cfg.body_force), _f64(cfg.gravity),
            _f64(np.asarray(cfg.pos).reshape(-1) if self.np else np.zeros(3)),
            _f64(np.asarray(cfg.vel).reshape(-1) if self.np else np.zeros(3)),
            _f64(np.asarray(cfg.omega).reshape(-1) if self.np else np.zeros(3)),
            _f64(cfg.radius if self.np else np.zeros(1)),
            _f64(cfg.density if self.np else np.zeros(1)),
        ]
        gf, gs, pos, vel, omg, rad, rhos = self._keep
        self.h = lib.oracle_create(self.dim, self.shape[0], self.shape[1], self.shape[2], int(cfg.wall_y),
                                   float(cfg.tau), _p(gf), _p(gs), float(cfg.rho_fluid), float(cfg.k_n),
                                   float(cfg.restitution), int(cfg.dem_substeps), self.np,
                                   _p(pos), _p(vel), _p(omg), _p(rad), _p(rhos))
        self.N = lib.oracle_num_nodes(self.h)
        self.Q = lib.oracle_num_dirs(self.h)
        self.tau = float(cfg.tau)
        self.rho0 = float(cfg.rho_fluid)
        self.wall_y = int(cfg.wall_y)
        self.radius = np.asarray(cfg.radius, dtype=np.float64).copy()
        self.steps_done = 0
        self.eps_method = int(getattr(cfg, "eps_method", 0))
        if self.eps_method == 1 and lib.oracle_set_eps_table(self.h) != 0:
            raise ValueError("the Eq. 6 table needs all radii equal and > 1")
        del npa

    def eps_table_value(self, offset) -> float:
        """Eq. 6 table value for a cell centred at ``offset`` from the particle
        centre (before the inside/outside classification and the clamp)."""
        o = [float(x) for x in offset] + [0.0] * (3 - len(offset))
        return self._lib.oracle_eps_table_value(self.h, o[0], o[1], o[2])

    def close(self):
        if getattr(self, "h", None):
            self._lib.oracle_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def step(self, n: int = 1) -> int:
        st = self._lib.oracle_step(self.h, int(n))
        self.steps_done += int(n)
        if st != 0:
            raise RuntimeError("oracle: a node exceeded the owner limit")
        return st

    def populations(self) -> np.ndarray:
        """Stored post-collision populations, shape (Q, nz, ny, nx)."""
        f = np.zeros(self.Q * self.N)
        self._lib.oracle_get_populations(self.h, _p(f))
        nx, ny, nz = self.shape
        return f.reshape(self.Q, nz, ny, nx)

    def set_populations(self, f):
        f = _f64(f, self.Q * self.N)
        self._lib.oracle_set_populations(self.h, _p(f))

    def particles(self):
        """dict of (np,3) arrays: pos, vel, omega, force (hydrodynamic, last
        step), torque (hydrodynamic, last step), contact (last sub-step)."""
        n3 = 3 * max(self.np, 1)
        a = [np.zeros(n3) for _ in range(6)]
        self._lib.oracle_get_particles(self.h, *[_p(x) for x in a])
        keys = ["pos", "vel", "omega", "force", "torque", "contact"]
        return {k: v[: 3 * self.np].reshape(self.np, 3) for k, v in zip(keys, a)}

    def masses(self):
        m = np.zeros(max(self.np, 1))
        I = np.zeros(max(self.np, 1))
        self._lib.oracle_get_mass(self.h, _p(m), _p(I))
        return m[: self.np], I[: self.np]

    def fields(self):
        """rho (nz,ny,nx), u (dim,nz,ny,nx) of the streamed state, eps (nz,ny,nx)."""
        rho = np.zeros(self.N)
        u = np.zeros(self.dim * self.N)
        eps = np.zeros(self.N)
        self._lib.oracle_fields(self.h, _p(rho), _p(u), _p(eps))
        nx, ny, nz = self.shape
        return rho.reshape(nz, ny, nx), u.reshape(self.dim, nz, ny, nx), eps.reshape(nz, ny, nx)

    def owners(self, maxo: int = 4):
        cnt = np.zeros(self.N, dtype=np.int32)
        ids = np.zeros(self.N * maxo, dtype=np.int32)
        e = np.zeros(self.N * maxo)
        self._lib.oracle_get_owners(self.h, cnt.ctypes.data_as(_ip), ids.ctypes.data_as(_ip), _p(e), maxo)
        return cnt, ids.reshape(self.N, maxo), e.reshape(self.N, maxo)
