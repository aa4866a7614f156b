"""Pins of the oracle's generating / absorbing relaxation zones (Sec. 4.4).

The paper defines the zone by its width L_Rel, the first k with k dx >= L_Rel, the blend
U <- m U + (1 - m) U* (w, p at nodes with the node mean of m) and m = sqrt(1 - (d / L_Rel)^2);
an absorbing zone has the still state as its target.  Checked from outside the oracle:
cells and nodes outside the zones are untouched; the inner zone cell is untouched and the
boundary cell takes the target; the target is a fixed point; an absorbing zone takes the
energy of an outgoing solitary wave where a wall reflects it; a generating zone driven by a
progressive long wave puts a wave of the target's amplitude into the channel.
"""
import numpy as np
import pytest

import oracle as O

G = 9.81


def _state2d(nx, ny, seed):
    rng = np.random.default_rng(seed)
    H = 1.0 + 0.1 * rng.random((ny, nx))
    h = H + 0.05 * rng.standard_normal((ny, nx))
    q1, q2 = 0.1 * rng.standard_normal((2, ny, nx))
    w, p = 0.01 * rng.standard_normal((2, ny + 1, nx + 1))
    return H, h, q1, q2, w, p


def test_zone_extent_and_end_values_2d():
    nx, ny, dx, dy = 40, 30, 0.1, 0.2
    relax = (0.45, 0.3, 0.0, 1.0)          # k = 5, 3, -, 5
    H, h, q1, q2, w, p = _state2d(nx, ny, 1)
    c = O.cfg(nx, ny, dx=dx, dy=dy, relax=relax)
    eta_t = 0.3 * np.ones((ny, nx))
    q1_t, q2_t = 0.2 * np.ones((2, ny, nx))
    w_t, p_t = 0.4 * np.ones((2, ny + 1, nx + 1))
    ho, ao, bo, wo, po = O.relax_2d(c, H, h, q1, q2, w, p, eta_t, q1_t, q2_t, w_t, p_t)
    kw, ke, kn = 5, 3, 5
    inside = np.zeros((ny, nx), bool)
    inside[:ny - 1 - kn, kw:nx - 1 - ke + 1] = True        # m = 1 (the zones' inner cells too)
    for a, b in ((ho, h), (ao, q1), (bo, q2)):
        assert np.array_equal(a[inside], b[inside])
        assert not np.allclose(a[~inside], b[~inside])
    # boundary cells of a zone take the target exactly (m = 0 there)
    assert np.array_equal(ho[:, 0], eta_t[:, 0] + H[:, 0])
    assert np.array_equal(ao[:, nx - 1], q1_t[:, nx - 1])
    assert np.array_equal(bo[ny - 1, :], q2_t[ny - 1, :])
    # nodes: untouched where both neighbouring cell columns / rows have m = 1
    node_in = np.zeros((ny + 1, nx + 1), bool)
    node_in[:ny - kn, kw + 1:nx - ke] = True
    assert np.array_equal(wo[node_in], w[node_in]) and np.array_equal(po[node_in], p[node_in])
    assert not np.allclose(wo[~node_in], w[~node_in])
    # the corner node of two zones: both node means are 0 (end cells and their images)
    assert wo[0, 0] == w_t[0, 0] and po[ny, nx] == p_t[ny, nx]


def test_target_is_a_fixed_point_and_blend_is_convex():
    nx, ny = 32, 24
    H, h, q1, q2, w, p = _state2d(nx, ny, 2)
    c = O.cfg(nx, ny, dx=0.1, relax=(0.6, 0.6, 0.6, 0.6))
    out = O.relax_2d(c, H, h, q1, q2, w, p, h - H, q1, q2, w, p)
    for a, b in zip(out, (h, q1, q2, w, p)):
        assert np.max(np.abs(a - b)) < 1e-15
    H2, h2, a2, b2, w2, p2 = _state2d(nx, ny, 3)
    out = O.relax_2d(c, H, h, q1, q2, w, p, h2 - H, a2, b2, w2, p2)
    for a, x, y in zip(out, (h, q1, q2, w, p), (h2, a2, b2, w2, p2)):
        lo, hi = np.minimum(x, y), np.maximum(x, y)
        assert (a >= lo - 1e-15).all() and (a <= hi + 1e-15).all()


def test_absorbing_target_is_the_lake_at_rest():
    """No target: dry cells of the zone stay dry (h* = max(H, 0)), wet ones relax to H."""
    nx, ny = 20, 10
    H = np.linspace(-0.2, 1.0, nx)[None, :].repeat(ny, 0)
    h = np.maximum(H, 0) + 0.05
    z = np.zeros((ny, nx))
    zn = np.zeros((ny + 1, nx + 1))
    c = O.cfg(nx, ny, dx=0.1, relax=(0.5, 0.0, 0.0, 0.0))
    ho, *_ = O.relax_2d(c, H, h, z, z, zn, zn)
    assert ho[0, 0] == 0.0 and (ho >= 0).all()


def _energy(H, h, q, dx):
    eta = h - H
    return float(np.sum(0.5 * G * eta ** 2 + 0.5 * q ** 2 / np.maximum(h, 1e-12)) * dx)


def test_absorbing_zone_takes_an_outgoing_solitary_wave():
    """1D channel, Eq. (33) wave running east.  A wall sends it back (> 80 % of its energy
    stays in the channel); an absorbing zone 1.5 wave widths wide in front of the same wall
    leaves < 0.5 % (plain outflow ghosts alone leave about 2 %)."""
    n, Lc, h0, A = 600, 120.0, 1.0, 0.1
    dx = Lc / n
    x = (np.arange(n) + 0.5) * dx
    k = np.sqrt(3 * A / (4 * h0 ** 3))
    c0 = np.sqrt(G * (h0 + A))
    eta = A / np.cosh(k * (x - 40.0)) ** 2
    H = np.full(n, h0)
    h = H + eta
    q = h * c0 * eta / (h0 + eta)
    E0 = _energy(H, h, q, dx)
    lam = 2 * 3.0 / k                        # the wave's width (eta > 1 % of A)
    res = {}
    for name, bc, relax in (("wall", (O.WALL,) * 4, (0, 0, 0, 0)),
                            ("absorb", (O.WALL,) * 4, (0, 1.5 * lam, 0, 0))):
        c = O.cfg(n, dx=dx, cfl=0.9, bc=bc, relax=relax)
        ho, qo, w, p, t, s = O.run_1d(c, H, h, q, np.zeros(n + 1), np.zeros(n + 1),
                                      t_end=(Lc - 40.0 + 20.0) / c0)
        res[name] = _energy(H, ho, qo, dx) / E0
    assert res["wall"] > 0.8
    assert res["absorb"] < 0.005


def test_generating_zone_drives_a_progressive_long_wave():
    """West zone, target eta* = A sin(k x - omega t), q* = c eta* (shallow-water wave,
    kh = 0.1), east absorbing zone: after the front has crossed, the crest-to-trough height
    in the middle of the channel is the target's 2A within 10 %."""
    n, h0, A = 800, 1.0, 0.01
    kk = 0.1 / h0
    lam = 2 * np.pi / kk
    Lc = 6 * lam
    dx = Lc / n
    x = (np.arange(n) + 0.5) * dx
    xn = np.arange(n + 1) * dx
    cph = np.sqrt(G * h0 / (1 + (kk * h0) ** 2 / 4))     # Yamazaki dispersion (Sec. 7.2)
    om = kk * cph
    H = np.full(n, h0)
    h = H.copy()
    q = np.zeros(n)
    w = np.zeros(n + 1)
    p = np.zeros(n + 1)
    c = O.cfg(n, dx=dx, cfl=0.8, bc=(O.OUTFLOW, O.OUTFLOW, 0, 0),
              relax=(1.0 * lam, 1.5 * lam, 0, 0))
    cz = O.cfg(n, dx=dx, cfl=0.8, bc=(O.OUTFLOW, O.OUTFLOW, 0, 0))
    cw = O.cfg(n, dx=dx, cfl=0.8, bc=(O.OUTFLOW, O.OUTFLOW, 0, 0), relax=(1.0 * lam, 0, 0, 0))
    ce = O.cfg(n, dx=dx, cfl=0.8, bc=(O.OUTFLOW, O.OUTFLOW, 0, 0), relax=(0, 1.5 * lam, 0, 0))
    t, T_end = 0.0, 4.5 * lam / cph
    mid = (x > 2.5 * lam) & (x < 3.5 * lam)
    hmax, hmin = -np.inf, np.inf
    while t < T_end:
        dt = O.cfl_dt_1d(cz, H, h, q)
        h, q, w, p = O.step_1d(cz, H, h, q, w, p, dt)
        t += dt
        eta_t = A * np.sin(kk * x - om * t)
        h, q, w, p = O.relax_1d(cw, H, h, q, w, p, eta_t, (h0 + eta_t) * cph * eta_t / h0,
                                np.zeros(n + 1), np.zeros(n + 1))
        h, q, w, p = O.relax_1d(ce, H, h, q, w, p)
        if t > 3.5 * lam / cph:
            hmax = max(hmax, (h - H)[mid].max())
            hmin = min(hmin, (h - H)[mid].min())
    assert c.relax[0] > 0
    assert abs((hmax - hmin) / (2 * A) - 1.0) < 0.1


def test_coefficients_at_special_distances():
    """Sec. 4.4's coefficients where they take exact values: L_Rel = 1, dx = 0.2 (k = 5);
    the cells 0.6 and 0.8 from the zone's inner cell have m = 0.8 and 0.6 (3-4-5 triangles),
    and the node between them the mean 0.7 (not the circle's value 0.714 at its own
    distance)."""
    n = 20
    H = np.full(n, 2.0)
    c = O.cfg(n, dx=0.2, relax=(1.0, 0.0, 0.0, 0.0))
    ho, qo, wo, po = O.relax_1d(c, H, H + 1.0, np.ones(n), np.ones(n + 1), np.ones(n + 1),
                                np.zeros(n), np.zeros(n), np.zeros(n + 1), np.zeros(n + 1))
    assert abs(ho[2] - H[2] - 0.8) < 1e-12 and abs(qo[1] - 0.6) < 1e-12
    assert abs(wo[2] - 0.7) < 1e-12 and abs(po[2] - 0.7) < 1e-12
    assert ho[0] == H[0] and ho[5] == H[5] + 1.0     # boundary cell: target; inner cell: kept
