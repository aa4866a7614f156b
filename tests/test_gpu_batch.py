"""Batched ensemble form (nh_create_batch ...) against the FP64 oracle, the single-domain
handle, and itself across launch forms (graph / eager, kernel-shape candidates).

Bars as for one domain: FP64 within 1e-10 relative L-infinity on h, (hu, hv) and p; FP32
within 1e-4 on eta; lake at rest exact.  Every domain of a batch has its own grid, time
step and solver convergence, so each is compared with its own oracle run.
"""
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
    e = max(np.abs(np.asarray(a, np.float64) - a_ref).max(),
            np.abs(np.asarray(b, np.float64) - b_ref).max())
    return e / (s if s > 0 else 1.0)


def small_members():
    """Five uneven domains (one rectangular) of the ensemble recipe at small sizes; the
    steep small-domain bathymetry makes some pressure systems fail the Gershgorin test, so
    the BiCGStab fallback is exercised too."""
    out = []
    for i, side in enumerate((24, 40, 56, 33, 48)):
        wl = inputs.ensemble_member(i, sides=(side,))
        if i == 3:   # rectangular: crop columns
            k = 21
            wl.H, wl.eta, wl.q1, wl.q2 = (a[:, :k].copy() for a in (wl.H, wl.eta, wl.q1, wl.q2))
            wl.nx = k
        out.append(wl)
    return out


def make_batch(wls, precision="fp64", **kw):
    kw.setdefault("tol", 1e-13 if precision == "fp64" else 1e-5)
    b = nh.Batch([w.H for w in wls], dx=wls[0].dx, precision=precision, **kw)
    for d, w in enumerate(wls):
        b.set_state(d, w.eta.astype(b.dtype), w.q1.astype(b.dtype), w.q2.astype(b.dtype))
    return b


def oracle_run(w, steps):
    c = O.cfg(w.nx, w.ny, dx=w.dx, dy=w.dy, bc=w.bc, tol=1e-14)
    zn = np.zeros((w.ny + 1, w.nx + 1))
    return O.run_2d(c, w.H, np.maximum(w.eta + w.H, 0), w.q1, w.q2, zn, zn, max_steps=steps)


def test_batch_fp64_matches_oracle_per_domain():
    wls = small_members()
    b = make_batch(wls)
    b.run(8)
    for d, w in enumerate(wls):
        g = b.get_state(d)
        h, q1, q2, _, p, t, steps, _ = oracle_run(w, 8)
        assert rel(g["eta"] + w.H, h) < 1e-10, d
        assert rel_q(g["q1"], g["q2"], q1, q2) < 1e-10, d
        assert rel(g["p"], p) < 1e-10, d
        assert abs(g["t"] - t) <= 1e-12 * t and b.stats(d)["steps"] == 8
    # the steep small-domain systems fail the Gershgorin test: BiCGStab finished those
    assert sum(b.stats(d)["fallbacks"] for d in range(len(wls))) > 0


@pytest.mark.parametrize("block_nodes", [70000, 0])
def test_batch_fallback_forms_match_oracle(block_nodes):
    """The BiCGStab solves of the domains whose rows fail the Gershgorin test: in one thread
    block each, beside the Chebyshev passes of the others (the default), or by the
    grid-wide BiCGStab after the passes (fallback_block_nodes = 0); captured steps, FP64,
    each domain against the oracle at 1e-10."""
    wls = small_members()
    b = make_batch(wls, graph=True, fallback_block_nodes=block_nodes)
    b.run(4)
    assert b.tuning()["graph"] == 1
    for d, w in enumerate(wls):
        g = b.get_state(d)
        h, q1, q2, _, p, t, steps, _ = oracle_run(w, 4)
        assert rel(g["eta"] + w.H, h) < 1e-10, d
        assert rel_q(g["q1"], g["q2"], q1, q2) < 1e-10, d
        assert rel(g["p"], p) < 1e-10, d
    assert sum(b.stats(d)["fallbacks"] for d in range(len(wls))) > 0


def test_batch_profile_counts_launches():
    wls = small_members()
    b = make_batch(wls, "fp32", graph=True)
    b.profile(True)
    b.run(1)
    pr = b.profile_read()
    b.profile(False)
    assert pr["hyperbolic"][0] == 2 and pr["assembly"][0] == 2 and pr["correction"][0] == 2
    assert pr["cheb_pass"][0] >= 2 and all(v[1] >= 0 for v in pr.values())
    # the fallback solves of the small steep members: one block launch per stage
    assert pr["bicg_block"][0] == 2


def test_batch_fp32_matches_oracle_and_single_domain():
    wls = small_members()
    b = make_batch(wls, "fp32")
    b.run(8)
    for d, w in enumerate(wls):
        g = b.get_state(d)
        h, q1, q2, _, p, t, steps, _ = oracle_run(w, 8)
        assert rel(g["eta"], h - w.H) < 1e-4, d
        sim = nh.Sim(w.H, w.dx, precision="fp32", tol=1e-5)
        sim.set_state(w.eta.astype(np.float32), w.q1.astype(np.float32),
                      w.q2.astype(np.float32))
        for _ in range(8):
            sim.step()
        s = sim.get_state()
        assert rel(g["eta"], s["eta"].astype(np.float64)) < 1e-5, d
        assert sim.stats()["t"] == pytest.approx(g["t"], rel=1e-6)


def test_batch_graph_equals_eager():
    wls = small_members()
    a = make_batch(wls, "fp32", graph=False)
    b = make_batch(wls, "fp32", graph=True)
    a.run(6)
    b.run(3)
    b.run(3)
    assert b.tuning()["graph"] == 1
    for d in range(len(wls)):
        ga, gb = a.get_state(d), b.get_state(d)
        for k in ("eta", "q1", "q2", "w", "p"):
            assert np.array_equal(ga[k], gb[k]), (d, k)
        assert ga["t"] == gb["t"]
        assert a.stats(d)["solver_iters"] == b.stats(d)["solver_iters"]


def test_batch_every_kernel_shape_gives_the_same_result():
    wls = small_members()
    ref = make_batch(wls)
    ref.run(4)
    want = [ref.get_state(d) for d in range(len(wls))]
    cands = nh.batch_candidates("fp64")
    combos = [(k, 0, 0, 0) for k in range(len(cands["hyp"]))]
    combos += [(0, k, 0, 15) for k in range(len(cands["assembly"]))]
    combos += [(0, 0, k, 5) for k in range(len(cands["cheb"]))]
    for hyp, asm, cheb, pers in combos:
        b = make_batch(wls)
        b.set_tuning(hyp=hyp, assembly=asm, cheb=cheb, persistent=pers)
        b.run(4)
        for d in range(len(wls)):
            g = b.get_state(d)
            assert rel(g["eta"], want[d]["eta"]) < 1e-11, (hyp, asm, cheb, pers, d)
            assert rel(g["p"], want[d]["p"]) < 1e-9, (hyp, asm, cheb, pers, d)


def test_batch_autotune_with_graph():
    wls = small_members()
    b = make_batch(wls, "fp32", autotune=True, graph=True)
    b.run(4)
    t = b.tuning()
    assert t["tuned"] == 1 and t["graph"] == 1 and min(t["ms"]) > 0
    ref = make_batch(wls, "fp32")
    ref.run(4)
    for d in range(len(wls)):
        assert rel(b.get_state(d)["eta"], ref.get_state(d)["eta"]) < 1e-5


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_batch_lake_at_rest_exact(precision):
    wls = small_members()
    b = nh.Batch([w.H for w in wls], dx=0.1, precision=precision, graph=True)
    before = [b.get_state(d) for d in range(len(wls))]
    b.run(20)
    for d in range(len(wls)):
        g = b.get_state(d)
        assert np.array_equal(g["eta"], before[d]["eta"])
        assert not g["q1"].any() and not g["q2"].any() and not g["p"].any()


def test_batch_mass_and_time_steps():
    """All-wet basins of different sizes and cell sizes (walls): mass to round-off, and each
    domain's next step is the Eq. (23) step of its own state."""
    wls = [inputs.shoals_2d(n=n, seed=2 + n) for n in (24, 40, 56)]
    b = nh.Batch([w.H for w in wls], dxs=[w.dx for w in wls], precision="fp64", tol=1e-13)
    for d, w in enumerate(wls):
        b.set_state(d, w.eta, w.q1, w.q2)
    m0 = [b.stats(d)["mass"] for d in range(len(wls))]
    b.run(10)
    for d, w in enumerate(wls):
        st = b.stats(d)
        assert abs(st["mass"] - m0[d]) <= 1e-13 * m0[d]
        g = b.get_state(d)
        c = O.cfg(w.nx, w.ny, dx=w.dx, dy=w.dy, bc=w.bc)
        assert st["dt_next"] == pytest.approx(
            O.cfl_dt_2d(c, w.H, np.maximum(g["eta"] + w.H, 0), g["q1"], g["q2"]), rel=1e-12)
        h, q1, q2, _, p, t, steps, _ = oracle_run(w, 10)
        assert rel(g["eta"] + w.H, h) < 1e-10 and abs(g["t"] - t) <= 1e-12 * t


def test_full_ensemble_sampled_against_oracle():
    """The 256-domain ensemble (sides 128..1024) in FP32 with the autotuned kernels and the
    graph, two steps; two sampled domains (one 128^2, one 256^2) against the oracle."""
    wls = [inputs.ensemble_member(i) for i in range(256)]
    b = make_batch(wls, "fp32", autotune=True, graph=True)
    b.run(2)
    picked = [next(d for d, w in enumerate(wls) if w.nx == s) for s in (128, 256)]
    for d in picked:
        w = wls[d]
        h, q1, q2, _, p, t, steps, _ = oracle_run(w, 2)
        g = b.get_state(d)
        assert rel(g["eta"], h - w.H) < 1e-4, d
        assert g["t"] == pytest.approx(t, rel=1e-6)
    for d in range(0, 256, 17):
        st = b.stats(d)
        assert st["steps"] == 2 and not st["nonfinite"]


def test_batch_literal_wet_dry_form_matches_oracle():
    """dry_zero = 0 (the second step as Sec. 4.5 states it, no truncation in dry cells) on
    the batched form, against the oracle in the same mode, over 2 steps.  The device holds
    eta, so a depth h is known there only to ulp(H) / h relative, and the literal form keeps
    q in such cells and divides fluxes by h: the two sides agree to 1e-10 only while every
    wet depth stays above 1e6 ulps of H (1.1e-10 m here).  These members form thinner
    films within 2 steps (one reaches 2.5e-44 m, below any eta); a step is compared on the
    domains whose oracle depths all stay above that bound, at least three per step."""
    wls = small_members()
    b = make_batch(wls, dry_zero=0)
    for steps in (1, 2):
        b.run(1)
        compared = 0
        for d, w in enumerate(wls):
            c = O.cfg(w.nx, w.ny, dx=w.dx, dy=w.dy, bc=w.bc, tol=1e-14, dry_zero=False)
            zn = np.zeros((w.ny + 1, w.nx + 1))
            h, q1, q2, _, p, t, _, _ = O.run_2d(c, w.H, np.maximum(w.eta + w.H, 0), w.q1,
                                                w.q2, zn, zn, max_steps=steps)
            if h[h > 0].min() < 1e6 * np.spacing(np.abs(w.H).max()):
                continue
            g = b.get_state(d)
            assert rel(g["eta"] + w.H, h) < 1e-10, (steps, d)
            assert rel_q(g["q1"], g["q2"], q1, q2) < 1e-10, (steps, d)
            assert rel(g["p"], p) < 1e-10, (steps, d)
            compared += 1
        assert compared >= 3, steps
