"""The breaking terms (Sec. 3 with q_x -> div q, u_x -> div u, Eq. (9) switch), which run
inside the assembly kernels, on a state whose converging flow switches breaking on:
single-domain and batched paths against the FP64 oracle with breaking and Manning
friction, and against the same run without breaking (the terms must act).
"""
import numpy as np
import pytest

import oracle as O
from paper_1706_04551_b300 import inputs, nh

pytestmark = pytest.mark.gpu

KW = dict(breaking=1, manning_n=0.015)


def rel(x, ref):
    s = np.abs(ref).max()
    return np.abs(np.asarray(x, np.float64) - ref).max() / (s if s > 0 else 1.0)


def converging(n, seed, ny=None):
    """Shoals bathymetry (walls, all wet) with a discharge field of strong divergence:
    |div q| reaches several times B1 sqrt(g h), so the Eq. (9) switch is on where the flow
    converges."""
    wl = inputs.shoals_2d(n=n, L=0.1 * n, seed=seed, nshoal=2)
    if ny is not None:
        wl.H, wl.eta, wl.q1, wl.q2 = (a[:ny].copy() for a in (wl.H, wl.eta, wl.q1, wl.q2))
        wl.ny = ny
    rng = np.random.default_rng(seed)
    y, x = np.mgrid[0:wl.ny, 0:wl.nx] * wl.dx
    L = wl.nx * wl.dx
    h = wl.eta + wl.H
    ph = rng.uniform(0, 2 * np.pi, 2)
    wl.q1 = 0.5 * h * np.sin(2 * np.pi * 2 * x / L + ph[0])
    wl.q2 = 0.5 * h * np.cos(2 * np.pi * 3 * y / L + ph[1])
    return wl


def oracle(wl, steps):
    c = O.cfg(wl.nx, wl.ny, dx=wl.dx, dy=wl.dy, bc=wl.bc, manning=KW["manning_n"],
              breaking=True, tol=1e-14)
    zn = np.zeros((wl.ny + 1, wl.nx + 1))
    return O.run_2d(c, wl.H, np.maximum(wl.eta + wl.H, 0), wl.q1, wl.q2, zn, zn,
                    max_steps=steps)


def sim_run(wl, steps, precision="fp64", **kw):
    sim = nh.Sim(wl.H, wl.dx, wl.dy, bc=wl.bc, precision=precision,
                 tol=1e-13 if precision == "fp64" else 1e-5, **kw)
    dt = np.float64 if precision == "fp64" else np.float32
    sim.set_state(wl.eta.astype(dt), wl.q1.astype(dt), wl.q2.astype(dt))
    for _ in range(steps):
        sim.step()
    g = sim.get_state()
    sim.close()
    return g


def test_breaking_acts_and_matches_oracle_fp64():
    wl = converging(72, 11, ny=61)
    g = sim_run(wl, 6, **KW)
    h, q1, q2, w, p, t, s, it = oracle(wl, 6)
    assert rel(g["eta"] + wl.H, h) < 1e-10
    assert rel(g["q1"], q1) < 1e-10 and rel(g["q2"], q2) < 1e-10
    assert rel(g["p"], p) < 1e-10
    g0 = sim_run(wl, 6, manning_n=KW["manning_n"])   # same run without the breaking terms
    assert rel(g0["q1"], q1) > 1e-6   # the breaking terms changed the discharge


def test_breaking_fp32_within_1e4_of_oracle():
    wl = converging(72, 11, ny=61)
    g = sim_run(wl, 6, "fp32", **KW)
    h, *_ = oracle(wl, 6)
    assert rel(g["eta"], h - wl.H) < 1e-4


def test_batch_breaking_matches_oracle_fp64():
    wls = [converging(n, 20 + n) for n in (40, 57, 33)]
    b = nh.Batch([w.H for w in wls], dx=wls[0].dx, precision="fp64", tol=1e-13, **KW)
    for d, w in enumerate(wls):
        b.set_state(d, w.eta, w.q1, w.q2)
    b.run(5)
    for d, w in enumerate(wls):
        g = b.get_state(d)
        h, q1, q2, _, p, t, steps, _ = oracle(w, 5)
        assert rel(g["eta"] + w.H, h) < 1e-10, d
        assert max(rel(g["q1"], q1), rel(g["q2"], q2)) < 1e-10, d
        assert rel(g["p"], p) < 1e-10, d
    b.close()
