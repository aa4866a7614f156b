"""Steps captured as CUDA graphs (nh_params.capture = 1: one graph per step, the pressure
solve as conditional WHILE nodes whose condition kernels read the solve's control block)
against the same steps launched eagerly with the host polling the solve (capture = 0): the
same kernels with the same arguments, so the states agree bit for bit, and so do the
solver statistics.
"""
import numpy as np
import pytest

from paper_1706_04551_b300 import inputs, nh

pytestmark = pytest.mark.gpu

FIELDS = ("eta", "q1", "q2", "w", "p")


def island(n=128):
    return inputs.island_2d(n=n, L=6.4 * n / 128, center=(5.0 * n / 128, None),
                            x0=2.0 * n / 128)


def run(wl, capture, steps, precision="fp32", **kw):
    dt_np = np.float32 if precision == "fp32" else np.float64
    sim = nh.Sim(wl.H, wl.dx, wl.dy, bc=wl.bc, precision=precision, capture=capture, **kw)
    sim.set_state(wl.eta.astype(dt_np), wl.q1.astype(dt_np), wl.q2.astype(dt_np))
    dts = [sim.step() for _ in range(steps)]
    g = sim.get_state()
    st = sim.stats()
    sim.close()
    return g, st, dts


def same(a, b):
    for k in FIELDS:
        assert np.array_equal(a[k], b[k]), k
    assert a["t"] == b["t"]


@pytest.mark.parametrize("precision,form", [("fp32", 7), ("fp32", 5), ("fp32", 0),
                                            ("fp64", 3), ("fp64", 0)])
def test_captured_steps_equal_eager_steps_bitwise(precision, form):
    wl = island()
    kw = dict(manning_n=0.015, breaking=1, cheb_form=form,
              tol=1e-5 if precision == "fp32" else 1e-12)
    ge, se, de = run(wl, 0, 12, precision, **kw)
    gg, sg, dg = run(wl, 1, 12, precision, **kw)
    same(ge, gg)
    assert de == dg
    for k in ("solver_iters", "last_iters", "fallbacks", "fallback_iters", "steps"):
        assert se[k] == sg[k], k
    assert se["last_resid"] == sg["last_resid"]


def test_captured_fallback_to_bicgstab_equals_eager():
    """The Sec. 7.7 dam-break: rows near the dam fail the Gershgorin test, so every solve
    goes on with BiCGStab (stopped by criterion (32)) -- inside the graph, the second
    WHILE node."""
    wl = inputs.dambreak_2d(96)
    kw = dict(cfl=0.9, tol=1e-12, eps_dp=1e-6, cheb_form=1, max_iter=20000)
    ge, se, _ = run(wl, 0, 6, "fp64", **kw)
    gg, sg, _ = run(wl, 1, 6, "fp64", **kw)
    assert se["fallbacks"] > 0
    same(ge, gg)
    for k in ("solver_iters", "fallbacks", "fallback_iters", "last_iters"):
        assert se[k] == sg[k], k


def test_captured_options_equal_eager():
    """The energy-consistent w equation and absorbing relaxation zones inside the graph."""
    wl = island(96)
    kw = dict(manning_n=0.015, breaking=1, cheb_form=7, tol=1e-5, w_equation=nh.W_TRANSPORT,
              relax_width=(0.3, 0.3, 0.3, 0.3))
    ge, se, _ = run(wl, 0, 8, "fp32", **kw)
    gg, sg, _ = run(wl, 1, 8, "fp32", **kw)
    same(ge, gg)


def test_captured_hydrostatic_step_equals_eager():
    wl = inputs.dambreak_2d(96)
    ge, _, _ = run(wl, 0, 10, "fp64", nonhydrostatic=0)
    gg, _, _ = run(wl, 1, 10, "fp64", nonhydrostatic=0)
    same(ge, gg)


def test_captured_profile_counts_the_passes():
    """Profiling a captured step times each kernel class between event nodes; the
    Chebyshev class counts the passes the WHILE node launched (pairs, so at most one per
    solve more than the sweeps need)."""
    wl = island()
    sim = nh.Sim(wl.H, wl.dx, wl.dy, bc=wl.bc, precision="fp32", cheb_form=7, tol=1e-5,
                 manning_n=0.015, breaking=1)
    sim.set_state(wl.eta.astype(np.float32), wl.q1.astype(np.float32), wl.q2.astype(np.float32))
    sim.step()   # eager (one-time set-up), then captured
    it0 = sim.stats()["solver_iters"]
    sim.profile(True)
    steps = 5
    for _ in range(steps):
        sim.step()
    pr = sim.profile_read()
    sim.profile(False)
    sweeps = sim.stats()["solver_iters"] - it0
    sim.close()
    n_pass, ms_pass = pr["cheb_pass"]
    assert sweeps / 8 <= n_pass <= sweeps / 8 + 2 * steps
    for k in ("hyperbolic", "assembly", "correction"):
        assert pr[k][0] == 2 * steps and pr[k][1] > 0, k
    assert ms_pass > 0
