"""FP64 pressure solves by defect correction with FP32 inner solves (nh_params.refine_fp32):
the residual of every round is taken in FP64 with the FP64 rows and decides convergence, so
the step meets the FP64 parity bars while its sweeps run in FP32."""
import numpy as np
import pytest

import oracle as O
from paper_1706_04551_b300 import inputs, nh

pytestmark = pytest.mark.gpu


def rel(x, ref):
    s = np.abs(ref).max()
    return np.abs(np.asarray(x, np.float64) - ref).max() / (s if s > 0 else 1.0)


def rel_q(a, b, a_ref, b_ref):
    s = max(np.abs(a_ref).max(), np.abs(b_ref).max())
    e = max(np.abs(a - a_ref).max(), np.abs(b - b_ref).max())
    return e / (s if s > 0 else 1.0)


@pytest.mark.parametrize("which", ["shoals", "island"])
def test_refined_fp64_steps_match_the_oracle(which):
    if which == "shoals":
        wl = inputs.shoals_2d(n=64)
        kw, okw, steps = {}, {}, 20
    else:
        wl = inputs.island_2d(n=64, L=25.6, center=(12.8, None), x0=4.0)
        kw = dict(manning_n=0.015, breaking=1)
        okw = dict(manning=0.015, breaking=True)
        steps = 15
    sim = nh.Sim(wl.H, wl.dx, bc=wl.bc, precision="fp64", tol=1e-13, refine_fp32=1, **kw)
    sim.set_state(wl.eta, wl.q1, wl.q2)
    for _ in range(steps):
        sim.step()
    g = sim.get_state()
    st = sim.stats()
    sim.close()
    c = O.cfg(wl.nx, wl.ny, dx=wl.dx, bc=wl.bc, tol=1e-14, **okw)
    zn = np.zeros((wl.ny + 1, wl.nx + 1))
    h, q1, q2, w, p, t, s, it = O.run_2d(c, wl.H, wl.h, wl.q1, wl.q2, zn, zn, max_steps=steps)
    assert rel(g["eta"] + wl.H, h) < 1e-10
    assert rel_q(g["q1"], g["q2"], q1, q2) < 1e-10
    assert rel(g["p"], p) < 1e-10
    assert max(st["last_resid"]) <= 1e-13 and st["fallbacks"] == 0


def test_refined_lake_at_rest_exact():
    wl = inputs.island_2d(n=64, L=25.6, center=(12.8, None), x0=4.0)
    sim = nh.Sim(wl.H, wl.dx, bc=wl.bc, precision="fp64", refine_fp32=1)
    eta0 = np.where(wl.H > 0, 0.0, -wl.H)
    z = np.zeros_like(eta0)
    sim.set_state(eta0, z, z)
    for _ in range(10):
        sim.step()
    g = sim.get_state()
    sim.close()
    assert np.array_equal(g["eta"], eta0) and not g["p"].any() and not g["q1"].any()


def test_refined_solve_equals_fp64_sweeps_to_tolerance():
    """The 1024^2 shoals, 2 steps at tol 1e-12: the refined and the plain FP64 solves agree
    on eta, q and p to the tolerance's order."""
    wl = inputs.shoals_2d()
    out = []
    for r in (0, 1):
        sim = nh.Sim(wl.H, wl.dx, bc=wl.bc, precision="fp64", tol=1e-12, refine_fp32=r)
        sim.set_state(wl.eta, wl.q1, wl.q2)
        for _ in range(2):
            sim.step()
        out.append((sim.get_state(), sim.stats()))
        sim.close()
    (a, sa), (b, sb) = out
    assert rel(b["eta"], a["eta"]) < 1e-9 and rel(b["p"], a["p"]) < 1e-9
    assert max(sb["last_resid"]) <= 1e-12
