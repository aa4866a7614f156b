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
    # q = 0 in dry cells by default (Sec. 4.5 literal form: dry_zero = 0); default wait limit
    assert p.dry_zero == 1 and p.wait_polls == 0
    # steps captured as graphs; small batched fallback solves in one block each
    assert p.capture == 1 and p.fallback_block_nodes == 70000
    # the cyclic form of the Chebyshev pass
    assert p.cheb_cyclic == 1


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


def test_cheb_forms_and_bad_form_rejected_without_touching_the_gpu():
    import numpy as np
    B.build()
    L = nh.load()
    assert nh.cheb_forms("fp32") == 8 and nh.cheb_forms("fp64") == 4
    assert nh.cheb_cyclic_forms("fp32") == 3 and nh.cheb_cyclic_forms("fp64") == 1
    assert L.nh_cheb_forms(7) == nh.EINVAL and L.nh_cheb_cyclic_forms(7) == nh.EINVAL
    p = nh.default_params()
    assert p.cheb_form == -1
    g = nh.Grid()
    g.dim, g.nx, g.ny, g.dx, g.dy = 2, 8, 8, 0.1, 0.1
    H = np.ones(64)
    # past the Jacobi forms come the cyclic ones (FP32 8-10, FP64 4)
    for prec, bad in ((nh.FP32, 11), (nh.FP64, 5), (nh.FP32, -2)):
        p.precision, p.cheb_form = prec, bad
        h = ctypes.c_void_p()
        rc = L.nh_create(ctypes.byref(g), H.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                         ctypes.byref(p), None, ctypes.byref(h))
        assert rc == nh.EINVAL and not h.value
    # the cyclic form is a switch (the form number nh_cheb_forms reports it under is not a
    # value of cheb_form)
    p.cheb_form, p.cheb_cyclic = -1, 2
    h = ctypes.c_void_p()
    rc = L.nh_create(ctypes.byref(g), H.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                     ctypes.byref(p), None, ctypes.byref(h))
    assert rc == nh.EINVAL and not h.value


def test_periodic_only_on_both_ends_of_1d_channels():
    import numpy as np
    B.build()
    L = nh.load()
    p = nh.default_params()
    H = np.ones(64)
    for dim, bc in ((2, (2, 2, 0, 0)), (1, (2, 0, 0, 0)), (1, (0, 2, 0, 0)), (1, (0, 0, 2, 2))):
        g = nh.Grid()
        g.dim, g.nx, g.ny, g.dx, g.dy = dim, 8, 8, 0.1, 0.1
        for k in range(4):
            g.bc[k] = bc[k]
        h = ctypes.c_void_p()
        rc = L.nh_create(ctypes.byref(g), H.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                         ctypes.byref(p), None, ctypes.byref(h))
        assert rc == nh.EINVAL and not h.value, (dim, bc)


def test_create_batch_rejects_bad_input_without_touching_the_gpu():
    import numpy as np
    B.build()
    L = nh.load()
    grids = (nh.Grid * 2)()
    for g in grids:
        g.dim, g.nx, g.ny, g.dx, g.dy = 2, 8, 8, 0.1, 0.1
    H = [np.ones(64), np.ones(64)]
    ptrs = (ctypes.c_void_p * 2)(*[h.ctypes.data for h in H])
    p = nh.default_params()
    h = ctypes.c_void_p()
    # the batched form solves with the Chebyshev-scheduled Jacobi only
    p.solver = nh.BICGSTAB
    assert L.nh_create_batch(2, grids, ptrs, ctypes.byref(p), None, 0, ctypes.byref(h)) == nh.EINVAL
    p.solver = nh.CHEBYSHEV
    grids[1].dim = 1   # 2D domains only
    assert L.nh_create_batch(2, grids, ptrs, ctypes.byref(p), None, 0, ctypes.byref(h)) == nh.EINVAL
    assert L.nh_create_batch(0, grids, ptrs, ctypes.byref(p), None, 0, ctypes.byref(h)) == nh.EINVAL
    assert not h.value


def test_batch_candidates_listed():
    B.build()
    for prec in ("fp32", "fp64"):
        c = nh.batch_candidates(prec)
        assert all(len(c[k]) >= 2 for k in ("hyp", "assembly", "cheb"))
        for tx, ty, th in c["cheb"]:
            assert tx > 16 and ty > 16 and th in (256, 512, 1024)


def test_w_equation_default_and_bad_value_rejected_without_touching_the_gpu():
    import numpy as np
    B.build()
    L = nh.load()
    p = nh.default_params()
    assert p.w_equation == nh.W_YAMAZAKI
    g = nh.Grid()
    g.dim, g.nx, g.ny, g.dx, g.dy = 2, 8, 8, 0.1, 0.1
    H = np.ones(64)
    for bad in (2, -1):
        p.w_equation = bad
        h = ctypes.c_void_p()
        rc = L.nh_create(ctypes.byref(g), H.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                         ctypes.byref(p), None, ctypes.byref(h))
        assert rc == nh.EINVAL and not h.value


def test_relaxation_zone_rules_without_touching_the_gpu():
    import numpy as np
    B.build()
    L = nh.load()
    p0 = nh.default_params()
    assert list(p0.relax_width) == [0.0] * 4
    H = np.ones(64)
    cases = (  # (dim, bc, widths) that nh_create must reject before any device work
        (1, (2, 2, 0, 0), (0.2, 0, 0, 0)),     # zone on a periodic side
        (1, (0, 0, 0, 0), (0, 0, 0.2, 0)),     # south zone of a 1D channel
        (2, (0, 0, 0, 0), (-0.1, 0, 0, 0)),    # negative width
        (2, (0, 0, 0, 0), (0, 0.9, 0, 0)),     # wider than the domain (8 x 0.1)
    )
    for dim, bc, wd in cases:
        g = nh.Grid()
        g.dim, g.nx, g.ny, g.dx, g.dy = dim, 8, 8, 0.1, 0.1
        for k in range(4):
            g.bc[k] = bc[k]
        p = nh.default_params()
        for k in range(4):
            p.relax_width[k] = wd[k]
        h = ctypes.c_void_p()
        rc = L.nh_create(ctypes.byref(g), H.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                         ctypes.byref(p), None, ctypes.byref(h))
        assert rc == nh.EINVAL and not h.value
