"""Kernel forms of the Chebyshev-scheduled Jacobi pass (the scheduled-relaxation Jacobi of
Sec. 5 with Chebyshev weights) forced one by one through nh_params.cheb_form.

Every form sweeps the same nodes with the same arithmetic, so a step taken with any form
equals, bit for bit, the step taken with form 0 whenever the two solves stop after the same
number of sweeps (the block sums of the convergence test are added in form-dependent order,
so a solve sitting exactly at the tolerance could stop one pass apart; the iteration counts
are compared first).  The register forms are also checked against the FP64 oracle.
"""
import numpy as np
import pytest

from paper_1706_04551_b300 import inputs, nh
from test_gpu_parity import _run_both, developed, make, rel, rel_q

pytestmark = pytest.mark.gpu


def island(n):
    # ragged: n + 1 nodes per side is no multiple of any form's tile; outflow walls mirror
    return inputs.island_2d(n=n, L=25.6 * n / 64, center=(12.8 * n / 64, None), x0=4.0)


def _run_form(wl, precision, form, steps, state, tol):
    sim, _ = make(wl, precision, cheb_form=form, tol=tol)
    eta, q1, q2 = state
    sim.set_state(eta.astype(sim.dtype), q1.astype(sim.dtype), q2.astype(sim.dtype))
    for _ in range(steps):
        sim.step()
    g = sim.get_state()
    st = sim.stats()
    sim.close()
    return g, (st["solver_iters"], st["fallbacks"])


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
@pytest.mark.parametrize("which", ["island", "shoals"])
def test_every_pass_form_gives_the_same_step(precision, which):
    """Bitwise equal to form 0 when both took the same sweeps and no BiCGStab hand-over
    (tolerances above the FP32 / FP64 stall floors); else p within the tolerance."""
    wl = island(150) if which == "island" else inputs.shoals_2d(n=203)
    state = developed(wl, seed=3)
    tol = 1e-4 if precision == "fp32" else 1e-10
    nf = nh.cheb_forms(precision)
    assert nf >= 4
    runs = [_run_form(wl, precision, f, 4, state, tol) for f in range(nf)]
    g0, c0 = runs[0]
    assert c0[0] > 0
    report = []
    for f, (g, c) in enumerate(runs[1:], start=1):
        d = max(float(np.abs(g[k].astype(np.float64) - g0[k]).max()) for k in g0 if k != "t")
        report.append((f, c, d))
    for f, c, d in report:
        if c == c0 and c[1] == 0:
            assert d == 0.0, (report, c0)
        else:
            assert rel(runs[f][0]["p"], g0["p"]) < 10 * tol, (report, c0)


def test_register_form_fp64_against_oracle():
    """The FP64 register form (3) through 12 steps of the wet/dry breaking island against
    the FP64 oracle (1e-10 relative L-infinity on h, the discharge and p)."""
    wl = island(100)
    sim, g, (h, q1, q2, w, p, t, s, it) = _run_both(wl, 12, cheb_form=3)
    assert rel(g["eta"] + wl.H, h) < 1e-10
    assert rel_q(g["q1"], g["q2"], q1, q2) < 1e-10
    assert rel(g["p"], p) < 1e-10


@pytest.mark.parametrize("form", [5, 6, 7])
def test_register_forms_fp32_against_oracle(form):
    """FP32 register forms on the shoals workload (walls, ragged 203^2): eta within 1e-4 of
    the FP64 oracle after 6 steps."""
    wl = inputs.shoals_2d(n=203)
    sim, g, (h, q1, q2, w, p, t, s, it) = _run_both(wl, 6, "fp32", tol=1e-5, cheb_form=form)
    assert rel(g["eta"], h - wl.H) < 1e-4
