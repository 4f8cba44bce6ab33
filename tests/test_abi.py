"""Host-only checks of the C ABI: the library loads, exports every function
include/lbm_imb.h declares, the ctypes struct matches the C layout, and the
size query validates configurations (no GPU needed)."""
import ctypes as C
import os
import re
import subprocess
import tempfile

import numpy as np
import pytest

from paper_1011_2613_gb300 import build_lib, inputs as I, lbm

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADERS = [os.path.join(ROOT, "include", f) for f in sorted(os.listdir(os.path.join(ROOT, "include")))
           if f.endswith(".h")]


@pytest.fixture(scope="module")
def built():
    build_lib.build()
    return lbm.lib()


def declared_functions():
    names = []
    for h in HEADERS:
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        names += re.findall(r"\b(lbm_imb_\w+)\s*\(", src)
    return sorted(set(names))


def test_every_declared_function_is_exported(built):
    names = declared_functions()
    assert len(names) >= 14
    out = subprocess.run(["nm", "-D", "--defined-only", lbm.LIB_PATH], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\sT\s(\w+)", out))
    missing = [n for n in names if n not in exported]
    assert not missing, missing
    for n in names:
        assert hasattr(built, n)


def test_struct_layout_matches_c():
    prog = r'''
#include <stddef.h>
#include <stdio.h>
#include "lbm_imb.h"
int main(void){
  printf("%zu %zu %zu %zu %zu %zu %zu\n", sizeof(lbm_imb_config), offsetof(lbm_imb_config, tau),
    offsetof(lbm_imb_config, rho_fluid), offsetof(lbm_imb_config, dem_substeps),
    offsetof(lbm_imb_config, n_particles), offsetof(lbm_imb_config, pos), offsetof(lbm_imb_config, density));
  return 0; }
'''
    with tempfile.TemporaryDirectory() as d:
        src = os.path.join(d, "t.c")
        exe = os.path.join(d, "t")
        open(src, "w").write(prog)
        subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), src, "-o", exe])
        vals = [int(x) for x in subprocess.check_output([exe]).split()]
    Cfg = lbm.Config
    assert vals == [C.sizeof(Cfg), Cfg.tau.offset, Cfg.rho_fluid.offset, Cfg.dem_substeps.offset,
                    Cfg.n_particles.offset, Cfg.pos.offset, Cfg.density.offset]


def test_required_bytes_and_validation(built):
    cfg = I.config1()
    n = lbm.required_bytes(cfg)
    # two FP64 D2Q9 lattices (x padded to 128) dominate
    assert n > 2 * 9 * 128 * 256 * 8
    assert lbm.required_bytes(cfg.replace(tau=0.5)) == 0
    assert lbm.required_bytes(cfg.replace(dim=4)) == 0
    assert lbm.required_bytes(cfg.replace(restitution=0.0)) == 0
    bad = cfg.replace(radius=np.full(20, -1.0))
    assert lbm.required_bytes(bad) == 0
    n32 = lbm.required_bytes(cfg.replace(storage="f32dev"))
    n16 = lbm.required_bytes(cfg.replace(storage="f16dev"))
    assert n16 < n32 < n
    # the pair storage (same 8-byte elements as FP64) adds its covered-node
    # list (one int per node) and the split form's covered-node buffer: an
    # entry of (Q + 5) float pairs, a double and three ints for every cell
    # of every particle's box, (2 R + 2)^d cells
    cells = int(2 * cfg.radius.max() + 2) ** 2
    buf = min(cfg.n_particles * cells, 128 * 256) * ((9 + 5) * 8 + 20)
    ndf = lbm.required_bytes(cfg.replace(storage="dfdev"))
    assert ndf >= n + 128 * 256 * 4 + buf
    assert built.lbm_imb_strerror(-7).decode().startswith("a lattice cell")


def test_slab_rows_partition():
    """The y-slab split of the decomposed lattice (host logic): every row once,
    sizes differing by at most one, larger slabs first."""
    from paper_1011_2613_gb300 import lbm as L

    for ny in (7, 64, 1512):
        for ns in (2, 3, 5, 16):
            rows = L.slab_rows(ny, ns)
            assert rows[0][0] == 0 and sum(n for _, n in rows) == ny
            assert all(rows[k][0] + rows[k][1] == rows[k + 1][0] for k in range(ns - 1))
            sizes = [n for _, n in rows]
            assert max(sizes) - min(sizes) <= 1 and sizes == sorted(sizes, reverse=True)
