"""lbm_imb_dem_forces_static: the DEM contact-force call for callers that
cannot allocate device memory (its bins live in a fixed array inside the
library).  Its forces must equal those of lbm_imb_dem_forces (the same
kernels with a caller workspace) on two calls in a row, the second with a
different particle set, so that nothing left in the shared array from the
first call leaks into the second.  Collected last so that a failing run
stops after every other test has run."""
import ctypes as C

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

TOL = 1e-15  # relative to the largest force, as in the DEM parity tests


def state(dim, n_side, R, seed, wall):
    rng = np.random.default_rng(seed)
    sp = 2 * R * 0.97
    ext = [int(np.ceil(n_side * sp)) + (2 if wall else 0)] * dim + [1] * (3 - dim)
    g = np.stack(np.meshgrid(*([np.arange(n_side)] * dim), indexing="ij"), -1).reshape(-1, dim)
    pos = np.zeros((len(g), 3))
    pos[:, :dim] = (g + 0.5) * sp + rng.uniform(-0.08, 0.08, (len(g), dim)) * R
    if wall:
        pos[:, 1] -= 0.5
    vel = 0.01 * rng.standard_normal((len(g), 3))
    if dim == 2:
        vel[:, 2] = 0
    rad = R * (1 + 0.05 * rng.random(len(g)))
    mass = 100 * rad ** dim
    return ext, pos, vel, rad, mass


def call_static(dim, ext, wall, pos, vel, rad, mass, kn, e, rmax):
    import torch
    from paper_1011_2613_gb300 import lbm

    n = rad.numel()
    fc = torch.full((n, 3), float("nan"), dtype=torch.float64, device="cuda")
    ex = (C.c_int32 * 3)(*ext)
    st = lbm.lib().lbm_imb_dem_forces_static(
        dim, ex, wall, n, rmax, C.c_void_p(pos.data_ptr()), C.c_void_p(vel.data_ptr()),
        C.c_void_p(rad.data_ptr()), C.c_void_p(mass.data_ptr()), kn, e, C.c_void_p(fc.data_ptr()),
        C.c_void_p(torch.cuda.current_stream().cuda_stream))
    return st, fc


def test_static_scratch_matches_workspace_call_twice():
    import torch
    from paper_1011_2613_gb300 import lbm

    t = lambda a: torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")
    cases = [(3, state(3, 6, 3.0, 21, 1), 40.0, 0.85), (2, state(2, 14, 2.5, 22, 0), 25.0, 0.9)]
    for dim, (ext, pos, vel, rad, mass), kn, e in cases:
        args = (t(pos), t(vel), t(rad), t(mass))
        rmax = float(rad.max())
        ref = lbm.dem_forces(dim, ext, 0 if dim == 2 else 1, *args, kn, e, rmax=rmax).cpu().numpy()
        st, fc = call_static(dim, ext, 0 if dim == 2 else 1, *args, kn, e, rmax)
        assert st == 0
        fc = fc.cpu().numpy()
        assert np.count_nonzero(np.abs(ref).sum(axis=1)) > len(rad) // 2
        assert np.max(np.abs(fc - ref)) <= TOL * np.max(np.abs(ref))


def test_static_scratch_rejects_oversize_problem():
    import torch
    from paper_1011_2613_gb300 import lbm

    # 4096^2 lattice, rmax 2: 1024^2 bins * 68 B > the fixed 8 MiB
    pos = torch.zeros((1, 3), dtype=torch.float64, device="cuda")
    r = torch.full((1,), 2.0, dtype=torch.float64, device="cuda")
    st, _ = call_static(2, [4096, 4096, 1], 0, pos, pos, r, r, 10.0, 0.9, 2.0)
    assert st == lbm.EUNSUPPORTED


def test_static_scratch_allocates_nothing():
    """The call's defining property: once the library is loaded (the first
    call also looks up the array's address), further calls leave the
    device's free memory unchanged.  Every buffer is made before the
    measurement, so the only allocation that could show is the library's."""
    import torch

    dim, (ext, pos, vel, rad, mass), kn, e = 3, state(3, 5, 3.0, 31, 1), 40.0, 0.85
    t = lambda a: torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")
    args = (t(pos), t(vel), t(rad), t(mass))
    rmax = float(rad.max())
    st, fc0 = call_static(dim, ext, 1, *args, kn, e, rmax)  # warm-up: loads the module and its array
    assert st == 0
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(3):
        st = _call_into(dim, ext, 1, *args, kn, e, rmax, fc0)
        assert st == 0
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0, f"free device memory changed by {free0 - free1} bytes"


def _call_into(dim, ext, wall, pos, vel, rad, mass, kn, e, rmax, fc):
    import torch
    from paper_1011_2613_gb300 import lbm

    ex = (C.c_int32 * 3)(*ext)
    return lbm.lib().lbm_imb_dem_forces_static(
        dim, ex, wall, rad.numel(), rmax, C.c_void_p(pos.data_ptr()), C.c_void_p(vel.data_ptr()),
        C.c_void_p(rad.data_ptr()), C.c_void_p(mass.data_ptr()), kn, e, C.c_void_p(fc.data_ptr()),
        C.c_void_p(torch.cuda.current_stream().cuda_stream))


def test_static_scratch_no_particles_is_ok_like_workspace_call():
    """n = 0: nothing to do, so neither call checks the layout (an oversized
    bin grid is not an error without particles)."""
    from paper_1011_2613_gb300 import lbm

    ex = (C.c_int32 * 3)(4096, 4096, 1)
    assert lbm.lib().lbm_imb_dem_forces_static(2, ex, 0, 0, 2.0, None, None, None, None, 10.0, 0.9, None,
                                                None) == 0
