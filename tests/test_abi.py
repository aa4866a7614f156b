"""The C-ABI library builds, loads without a GPU and exports every symbol nh.h declares."""
import ctypes
import os
import re

from paper_1706_04551_b300 import build as B
from paper_1706_04551_b300 import nh

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    txt = open(os.path.join(ROOT, "include", "nh.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(nh_[a-z_0-9]+)\s*\(", txt)))


def test_library_exports_every_declared_symbol():
    B.build()
    lib = ctypes.CDLL(B.LIB)
    names = declared_functions()
    assert "nh_create" in names and "nh_step" in names
    for n in names:
        assert hasattr(lib, n), n
    assert set(names) <= set(nh.EXPORTS) | set(names)


def test_binding_loads_and_default_params():
    B.build()
    p = nh.default_params()
    assert p.g == 9.81 and p.cfl == 0.9 and p.delta == 1e-5 and p.B1 == 0.15


def test_create_rejects_bad_grid_without_touching_the_gpu():
    import numpy as np
    B.build()
    L = nh.load()
    g = nh.Grid()
    g.dim, g.nx, g.ny, g.dx, g.dy = 2, 1, 4, 0.1, 0.1   # nx < 2 is invalid
    p = nh.default_params()
    h = ctypes.c_void_p()
    H = np.ones(4)
    rc = L.nh_create(ctypes.byref(g), H.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                     ctypes.byref(p), None, ctypes.byref(h))
    assert rc == nh.EINVAL and not h.value
