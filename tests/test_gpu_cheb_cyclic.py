"""The cyclic form of the Chebyshev-scheduled Jacobi pass (nh_params.cheb_cyclic, the
default for single-domain 2D handles): each step updates the nodes of one colour (I + J) mod 2 in place,
half the node updates of a Jacobi sweep, and every node takes the values of the full
iteration at the steps of its colour.  Checked against the FP64 oracle, against the Jacobi
forms of the pass, graph against eager, and at rest."""
import numpy as np
import pytest

from paper_1706_04551_b300 import inputs, nh
from test_gpu_parity import _run_both, developed, make, rel, rel_q

pytestmark = pytest.mark.gpu


def island(n):
    # ragged: n + 1 nodes per side is no multiple of the region's interior (48 x 80 FP32,
    # 56 x 24 FP64); outflow sides mirror
    return inputs.island_2d(n=n, L=25.6 * n / 64, center=(12.8 * n / 64, None), x0=4.0)


def _steps(wl, precision, steps, state, **kw):
    kw.setdefault("cheb_cyclic", 1)
    sim, _ = make(wl, precision, **kw)
    eta, q1, q2 = state
    sim.set_state(eta.astype(sim.dtype), q1.astype(sim.dtype), q2.astype(sim.dtype))
    iters = []
    for _ in range(steps):
        sim.step()
        iters.append(tuple(sim.stats()["last_iters"]))
    g, st = sim.get_state(), sim.stats()
    sim.close()
    return g, st, iters


def cyclic_form(s, precision):
    nf = nh.cheb_forms(precision)
    return nf <= s["cheb_form"] < nf + nh.cheb_cyclic_forms(precision)


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_cyclic_form_is_the_default_where_it_applies(precision):
    """After the timing of the first solves (16 here) a cyclic form is in use."""
    wl = inputs.shoals_2d(n=96)
    nf = nh.cheb_forms(precision)
    st = developed(wl, seed=1)
    _, s, _ = _steps(wl, precision, 8, st, cheb_cyclic=nh.default_params().cheb_cyclic)
    assert cyclic_form(s, precision), s["cheb_form"]
    # switched off, or under criterion (32), or with a form named: the Jacobi forms
    _, s, _ = _steps(wl, precision, 1, st, cheb_cyclic=0)
    assert -1 <= s["cheb_form"] < nf
    _, s, _ = _steps(wl, precision, 1, st, eps_dp=1e-6, max_iter=20000)
    assert -1 <= s["cheb_form"] < nf
    _, s, _ = _steps(wl, precision, 1, st, cheb_form=nf - 1)
    assert s["cheb_form"] == nf - 1


@pytest.mark.parametrize("n,steps", [(100, 12), (150, 4)])
def test_cyclic_fp64_against_oracle(n, steps):
    """FP64 wet/dry breaking island (ragged sizes, regions crossing every side) against the
    FP64 oracle: h, the discharge and p within 1e-10 relative L-infinity."""
    wl = island(n)
    sim, g, (h, q1, q2, w, p, t, s, it) = _run_both(wl, steps)
    assert cyclic_form(sim.stats(), "fp64")
    assert rel(g["eta"] + wl.H, h) < 1e-10
    assert rel_q(g["q1"], g["q2"], q1, q2) < 1e-10
    assert rel(g["p"], p) < 1e-10
    assert abs(g["t"] - t) < 1e-12 * t


def test_cyclic_fp64_shoals_against_oracle():
    wl = inputs.shoals_2d(n=203)
    sim, g, (h, q1, q2, w, p, t, s, it) = _run_both(wl, 6)
    assert rel(g["eta"] + wl.H, h) < 1e-10
    assert rel_q(g["q1"], g["q2"], q1, q2) < 1e-10
    assert rel(g["p"], p) < 1e-10


@pytest.mark.parametrize("which", ["shoals", "island"])
def test_cyclic_fp32_against_oracle(which):
    """FP32 (tol 1e-5): eta within 1e-4 of the FP64 oracle after 6 steps."""
    wl = inputs.shoals_2d(n=203) if which == "shoals" else island(150)
    sim, g, (h, q1, q2, w, p, t, s, it) = _run_both(wl, 6, "fp32", tol=1e-5, cheb_cyclic=1)
    assert cyclic_form(sim.stats(), "fp32")
    assert rel(g["eta"], h - wl.H) < 1e-4


@pytest.mark.parametrize("precision,tol,form", [("fp64", 1e-11, 3), ("fp32", 1e-5, 7)])
def test_cyclic_against_the_jacobi_form(precision, tol, form):
    """The same steps as the Jacobi register form within the solver tolerance, and no more
    steps per stage than that form's sweeps plus one pass (both converge at the Chebyshev
    rate; their stopping tests measure slightly different vectors)."""
    wl = island(150)
    state = developed(wl, seed=3)
    K = 8 if precision == "fp32" else 4
    gc, sc, ic = _steps(wl, precision, 4, state, tol=tol)
    gj, sj, ij = _steps(wl, precision, 4, state, tol=tol, cheb_form=form)
    assert rel(gc["p"], gj["p"].astype(np.float64)) < 100 * tol
    assert rel(gc["eta"] + wl.H, (gj["eta"] + wl.H).astype(np.float64)) < 20 * tol
    if sc["fallbacks"] == 0 and sj["fallbacks"] == 0:
        for a, b in zip(ic, ij):
            assert a[0] <= b[0] + K and a[1] <= b[1] + K, (ic, ij)


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_every_cyclic_form_gives_the_same_steps(precision):
    """The cyclic forms (region shapes, forced one by one through cheb_form) update every
    node with the same arithmetic: equal, bit for bit, to the first cyclic form whenever both
    solves stop after the same number of steps (the block sums of the stopping test are
    added in form-dependent order); else p within the tolerance."""
    wl = island(150)
    state = developed(wl, seed=7)
    tol = 1e-5 if precision == "fp32" else 1e-11
    nf, nc = nh.cheb_forms(precision), nh.cheb_cyclic_forms(precision)
    runs = [_steps(wl, precision, 4, state, tol=tol, cheb_form=nf + k) for k in range(nc)]
    g0, s0, _ = runs[0]
    assert s0["cheb_form"] == nf
    for k, (g, s, _) in enumerate(runs[1:], start=1):
        assert s["cheb_form"] == nf + k
        if (s["solver_iters"], s["fallbacks"]) == (s0["solver_iters"], s0["fallbacks"]) \
                and s0["fallbacks"] == 0:
            for key in ("eta", "q1", "q2", "w", "p"):
                assert np.array_equal(g[key], g0[key]), (k, key)
        else:
            assert rel(g["p"], g0["p"].astype(np.float64)) < 100 * tol, k


def test_cyclic_graph_equals_eager():
    """Captured steps (conditional WHILE solve loop) give the eager steps' bits."""
    wl = island(150)
    state = developed(wl, seed=5)
    ge, se, ie = _steps(wl, "fp32", 6, state, tol=1e-5, capture=0)
    gg, sg, ig = _steps(wl, "fp32", 6, state, tol=1e-5, capture=1)
    assert ie == ig
    for k in ("eta", "q1", "q2", "w", "p"):
        assert np.array_equal(ge[k], gg[k]), k
    assert ge["t"] == gg["t"]


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_cyclic_lake_at_rest_exact(precision):
    wl = island(150)
    sim, _ = make(wl, precision, cheb_cyclic=1)
    eta0 = np.where(wl.H > 0, 0.0, -wl.H).astype(sim.dtype)
    z = np.zeros_like(eta0)
    sim.set_state(eta0, z, z)
    for _ in range(10):
        sim.step()
    g = sim.get_state()
    sim.close()
    assert np.array_equal(g["eta"], eta0)
    assert not g["q1"].any() and not g["q2"].any() and not g["p"].any()
