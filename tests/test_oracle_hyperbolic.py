"""Pins of the oracle's hyperbolic step and of whole-step invariants (CPU, no GPU).

The exact Riemann solutions of the shallow-water equations (Stoker's wet dam break,
Ritter's dry dam break) pin the PVM-HLL fluxes in the hydrostatic limit; lake at rest
(Remark 2, Sec. 4.5), mass conservation and mirror / transpose symmetries pin the source
terms, boundary treatment and the 2D assembly.
"""
import numpy as np
import pytest
from scipy.optimize import brentq

import oracle as O
from paper_1706_04551_b300 import inputs

G = 9.81


def _stoker(hl, hr, x, t, g=G):
    """Exact dam-break solution of the SWE on a flat bed (Stoker; Ritter when hr = 0)."""
    cl = np.sqrt(g * hl)
    rare = ((2.0 * cl - x / t) / 3.0) ** 2 / g
    if hr == 0.0:
        return np.where(x < -cl * t, hl, np.where(x < 2.0 * cl * t, rare, 0.0))
    f = lambda hm: 2.0 * (cl - np.sqrt(g * hm)) - (hm - hr) * np.sqrt(g * (hm + hr) / (2 * hm * hr))
    hm = brentq(f, hr, hl)
    um = 2.0 * (cl - np.sqrt(g * hm))
    s = hm * um / (hm - hr)
    return np.where(x < -cl * t, hl,
                    np.where(x < (um - np.sqrt(g * hm)) * t, rare, np.where(x < s * t, hm, hr)))


@pytest.mark.parametrize("hr", [0.3, 0.0])
def test_dam_break_converges_to_exact_riemann_solution(hr):
    errs = []
    L = 50.0
    for n in (400, 1600):
        dx = L / n
        x = (np.arange(n) + 0.5) * dx - L / 2
        c = O.cfg(n, dx=dx, nonhydro=False)
        h, q, w, p, t, s = O.run_1d(c, np.ones(n), np.where(x < 0.0, 1.0, hr), np.zeros(n),
                                    np.zeros(n + 1), np.zeros(n + 1), t_end=2.0)
        assert h.min() >= 0.0
        errs.append(np.abs(h - _stoker(1.0, hr, x, t)).sum() * dx)
    assert errs[1] < 0.025               # L1 error of h over the 50 m channel
    assert errs[1] < 0.35 * errs[0]      # first-order convergence through the shock/front


def test_lake_at_rest_1d_wet_dry_bitwise():
    """Remark 2 / Sec. 4.5: still water over an emerging island stays exactly at rest,
    with friction and breaking switched on."""
    n, L = 300, 60.0
    dx = L / n
    x = (np.arange(n) + 0.5) * dx
    H = 1.0 - 1.4 * np.exp(-((x - 30.0) / 6.0) ** 2) + 0.2 * np.sin(x / 3.0)
    h = np.maximum(H, 0.0)
    assert (h == 0.0).any()
    c = O.cfg(n, dx=dx, manning=0.02, breaking=True)
    ho, qo, wo, po, t, s = O.run_1d(c, H, h, np.zeros(n), np.zeros(n + 1), np.zeros(n + 1),
                                    max_steps=300)
    assert s == 300
    assert np.array_equal(ho, h) and not qo.any() and not wo.any() and not po.any()


@pytest.mark.parametrize("which", ["shoals", "island"])
def test_lake_at_rest_2d_bitwise(which):
    if which == "shoals":
        wl = inputs.shoals_2d(n=32)
        kw = {}
    else:
        wl = inputs.island_2d(n=48, L=19.2, center=(9.6, None), x0=3.0)
        kw = dict(manning=0.015, breaking=True)
    H = wl.H
    h = np.maximum(H, 0.0)
    c = O.cfg(wl.nx, wl.ny, dx=wl.dx, bc=wl.bc, **kw)
    z = np.zeros_like(h)
    zn = np.zeros((wl.ny + 1, wl.nx + 1))
    ho, q1, q2, w, p, t, s, it = O.run_2d(c, H, h, z, z, zn, zn, max_steps=20)
    assert s == 20
    assert np.array_equal(ho, h) and not q1.any() and not q2.any() and not w.any()
    assert not p.any()


def test_uniform_flow_is_steady_periodic():
    n = 64
    c = O.cfg(n, dx=0.5, bc=(O.PERIODIC, O.PERIODIC, 0, 0))
    H = np.full(n, 2.0)
    h = H.copy()
    q = np.full(n, 0.7)
    ho, qo, wo, po, t, s = O.run_1d(c, H, h, q, np.zeros(n + 1), np.zeros(n + 1), max_steps=50)
    assert np.array_equal(ho, h) and np.array_equal(qo, q)


def test_mass_conservation_1d_and_2d():
    wl = inputs.solitary_1d(n=400, L=80.0, x0=20.0)
    n = wl.nx
    x = (np.arange(n) + 0.5) * wl.dx
    H = wl.H - 0.4 * np.exp(-((x - 50.0) / 5.0) ** 2)
    h = wl.eta + H
    c = O.cfg(n, dx=wl.dx)
    ho, *_ = O.run_1d(c, H, h, wl.q1, np.zeros(n + 1), np.zeros(n + 1), max_steps=400)
    assert abs(ho.sum() - h.sum()) <= 1e-13 * h.sum()

    w2 = inputs.shoals_2d(n=32)
    c2 = O.cfg(32, 32, dx=w2.dx)
    zn = np.zeros((33, 33))
    ho2, *_ = O.run_2d(c2, w2.H, w2.h, w2.q1, w2.q2, zn, zn, max_steps=40)
    assert abs(ho2.sum() - w2.h.sum()) <= 1e-13 * w2.h.sum()


def test_wall_equals_mirrored_double_domain():
    """Reflection by a wall is the head-on collision with the mirror image (Sec. 7.2):
    the walled run equals the left half of the doubled, mirrored domain."""
    n, L = 150, 30.0
    dx = L / n
    x = (np.arange(n) + 0.5) * dx
    H = 1.0 - 0.3 * np.exp(-((x - 12.0) / 3.0) ** 2)
    eta = 0.15 / np.cosh(0.35 * (x - 20.0)) ** 2
    h = H + eta
    q = -np.sqrt(G * 1.15) * eta
    c = O.cfg(n, dx=dx)
    dt = 0.02
    hw, qw, ww, pw, *_ = O.run_1d(c, H, h, q, np.zeros(n + 1), np.zeros(n + 1), max_steps=120,
                                  fixed_dt=dt)
    c2 = O.cfg(2 * n, dx=dx)
    H2 = np.concatenate([H, H[::-1]])
    h2 = np.concatenate([h, h[::-1]])
    q2 = np.concatenate([q, -q[::-1]])
    hd, qd, wd, pd, *_ = O.run_1d(c2, H2, h2, q2, np.zeros(2 * n + 1), np.zeros(2 * n + 1),
                                  max_steps=120, fixed_dt=dt)
    assert np.abs(hd[:n] - hw).max() <= 1e-12
    assert np.abs(qd[:n] - qw).max() <= 1e-11
    assert np.abs(pd[: n + 1] - pw).max() <= 1e-11 * np.abs(pw).max()


def test_2d_run_on_y_invariant_data_equals_1d_run():
    n, ny = 120, 3
    dx = 0.25
    x = (np.arange(n) + 0.5) * dx
    H = 1.0 - 0.3 * np.exp(-((x - 18.0) / 3.0) ** 2)
    eta = 0.2 / np.cosh(0.387 * (x - 10.0)) ** 2
    h = H + eta
    q = h * np.sqrt(G * 1.2) * eta / (1.0 + eta)
    dt = 0.03
    c1 = O.cfg(n, dx=dx)
    h1, q1, w1, p1, *_ = O.run_1d(c1, H, h, q, np.zeros(n + 1), np.zeros(n + 1), max_steps=30,
                                  fixed_dt=dt)
    c2 = O.cfg(n, ny, dx=dx, tol=1e-14)
    T = lambda v: np.tile(v, (ny, 1))
    zn = np.zeros((ny + 1, n + 1))
    h2, a2, b2, w2, p2, *_ = O.run_2d(c2, T(H), T(h), T(q), np.zeros((ny, n)), zn, zn,
                                      max_steps=30, fixed_dt=dt)
    assert not b2.any()
    for j in range(ny):
        assert np.abs(h2[j] - h1).max() <= 1e-13
        assert np.abs(a2[j] - q1).max() <= 1e-12 * np.abs(q1).max()
    for J in range(ny + 1):
        assert np.abs(p2[J] - p1).max() <= 1e-11 * np.abs(p1).max()


def test_2d_run_transpose_symmetry():
    wl = inputs.shoals_2d(n=24)
    X = np.arange(24)[None, :] * np.ones((24, 1))
    eta = wl.eta * (1.0 + 0.3 * X / 24)              # break the x/y symmetry
    h = wl.H + eta
    c = O.cfg(24, 24, dx=wl.dx, tol=1e-14)
    zn = np.zeros((25, 25))
    z = np.zeros_like(h)
    dt = 0.05
    r = O.run_2d(c, wl.H, h, z + 0.01 * X / 24, z, zn, zn, max_steps=10, fixed_dt=dt)
    rt = O.run_2d(c, wl.H.T.copy(), h.T.copy(), z, (z + 0.01 * X / 24).T.copy(), zn, zn,
                  max_steps=10, fixed_dt=dt)
    assert np.abs(r[0] - rt[0].T).max() <= 1e-13
    assert np.abs(r[1] - rt[2].T).max() <= 1e-12 * np.abs(r[1]).max()
    assert np.abs(r[2] - rt[1].T).max() <= 1e-12 * np.abs(r[2]).max()
    assert np.abs(r[4] - rt[4].T).max() <= 1e-11 * np.abs(r[4]).max()
