"""Physics pins of the oracle's full step (CPU, no GPU).

- Linear dispersion: linearising Eq. (7) on a flat bottom (eta_t + h u_x = 0,
  u_t + g eta_x + p_x / 2 = 0, h w_t = p, h u_x + 2 w = 0) gives
  omega^2 = g h k^2 / (1 + (k h)^2 / 4); the measured standing-wave period must follow it
  (and not the hydrostatic omega = sqrt(g h) k), converging at second order.
- Solitary wave (Eq. 33, Sec. 7.1): travels at c = sqrt(g (h0 + A)) keeping its shape.
- Accuracy test of Sec. 7.1 / Table 1: the printed orders of accuracy.
- Breaking (Sec. 3, Eq. 12): switch-off limit and dissipation (the terms themselves are
  parity unpinned beyond these invariants).
"""
import json
import os

import numpy as np
import pytest

import oracle as O
from paper_1706_04551_b300 import inputs

G = 9.81
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _standing_wave_period(kh, ncell, nonhydro=True, h0=1.0, cfl=0.5):
    k = kh / h0
    L = 2.0 * np.pi / k                       # one wavelength between two walls
    dx = L / ncell
    x = (np.arange(ncell) + 0.5) * dx
    H = np.full(ncell, h0)
    h = H + 1e-4 * h0 * np.cos(k * x)
    q = np.zeros(ncell)
    w = np.zeros(ncell + 1)
    p = np.zeros(ncell + 1)
    c = O.cfg(ncell, dx=dx, nonhydro=nonhydro)
    om = np.sqrt(G * h0 * k * k / (1.0 + kh * kh / 4.0))
    T = 2.0 * np.pi / om
    nst = int(np.ceil(2.2 * T / (cfl * dx / np.sqrt(G * h0))))
    dt = 2.2 * T / nst
    ck = np.cos(k * x)
    amps, ts = [], []
    for s in range(nst + 1):
        amps.append(((h - H) * ck).sum() / (ck * ck).sum())
        ts.append(s * dt)
        h, q, w, p = O.step_1d(c, H, h, q, w, p, dt)
    a = np.array(amps)
    zc = [ts[i] - a[i] * (ts[i + 1] - ts[i]) / (a[i + 1] - a[i])
          for i in range(len(a) - 1) if a[i] * a[i + 1] < 0]
    return 2.0 * np.mean(np.diff(zc)), T, 2.0 * np.pi / (np.sqrt(G * h0) * k)


@pytest.mark.parametrize("kh", [0.5, 1.0, 2.0, 3.0])
def test_linear_dispersion_relation(kh):
    Tm, T_nh, T_swe = _standing_wave_period(kh, 64)
    assert abs(Tm / T_nh - 1.0) < 3e-3
    assert abs(Tm / T_swe - 1.0) > 2e-2      # discriminates from the hydrostatic relation


def test_dispersion_error_is_second_order():
    e64 = abs(_standing_wave_period(1.0, 64)[0] / _standing_wave_period(1.0, 64)[1] - 1)
    T128, T, _ = _standing_wave_period(1.0, 128)
    e128 = abs(T128 / T - 1)
    assert 3.0 < e64 / e128 < 5.0


def _crest(x, e):
    i = int(np.argmax(e))
    y0, y1, y2 = e[i - 1], e[i], e[i + 1]
    d = 0.5 * (y0 - y2) / (y0 - 2 * y1 + y2)
    return x[i] + d * (x[1] - x[0]), y1 - 0.25 * (y0 - y2) * d


def test_solitary_wave_1d_workload():
    """1000 cells, 200 m, A = 0.2, 20 s, CFL 0.9: celerity sqrt(g (h0 + A)), amplitude and
    mass kept; the hydrostatic model loses the wave's shape."""
    wl = inputs.solitary_1d()
    x = (np.arange(wl.nx) + 0.5) * wl.dx
    res = {}
    for nh in (True, False):
        c = O.cfg(wl.nx, dx=wl.dx, cfl=0.9, nonhydro=nh)
        h, q, w, p, t, s = O.run_1d(c, wl.H, wl.h, wl.q1, np.zeros(wl.nx + 1),
                                    np.zeros(wl.nx + 1), t_end=20.0)
        assert abs(t - 20.0) < 1e-12
        res[nh] = (h, t)
    h, t = res[True]
    x0, a0 = _crest(x, wl.eta)
    x1, a1 = _crest(x, h - wl.H)
    assert abs((x1 - x0) / t / np.sqrt(G * 1.2) - 1.0) < 5e-3
    assert 0.9 < a1 / a0 <= 1.0
    assert abs(h.sum() - wl.h.sum()) <= 1e-13 * wl.h.sum()
    _, a_swe = _crest(x, res[False][0] - wl.H)
    assert a_swe / a0 < 0.8


def test_table1_orders_of_accuracy():
    """Sec. 7.1 / Table 1 procedure (periodic 50 m channel, g = 1, H = 1, A = 0.1,
    t = 10 s, CFL 0.4, fine-grid reference): the orders match the printed ones."""
    ref = json.load(open(os.path.join(GOLDEN, "table1_convergence.json")))
    L, A, g = 50.0, 0.1, 1.0

    def run(n):
        dx = L / n
        x = (np.arange(n) + 0.5) * dx
        k = np.sqrt(3 * A / 4)
        eta = A / np.cosh(k * (x - 25.0)) ** 2
        H = np.ones(n)
        h = H + eta
        q = h * np.sqrt(g) * eta                    # u of Eq. (33) with H = 1
        c = O.cfg(n, dx=dx, g=g, cfl=0.4, bc=(O.PERIODIC, O.PERIODIC, 0, 0))
        ho, qo, *_ = O.run_1d(c, H, h, q, np.zeros(n + 1), np.zeros(n + 1), t_end=10.0)
        return ho, qo

    nref = 6400
    hr, qr = run(nref)
    errs = []
    for n in (100, 200, 400, 800):
        h, q = run(n)
        f = nref // n
        errs.append((np.abs(h - hr.reshape(n, f).mean(1)).sum() * L / n,
                     np.abs(q - qr.reshape(n, f).mean(1)).sum() * L / n))
    for i in range(1, 4):
        oh = np.log2(errs[i - 1][0] / errs[i][0])
        oq = np.log2(errs[i - 1][1] / errs[i][1])
        assert abs(oh - ref["order_h"][i]) < 0.2, (i, oh)
        assert abs(oq - ref["order_q"][i]) < 0.2, (i, oq)


def _beach(breaking, B1=0.15):
    """Solitary wave (A/H = 0.3) running up a 1:19.85 plane beach (Sec. 7.4 geometry)."""
    n, x0, x1 = 500, -10.0, 40.0
    dx = (x1 - x0) / n
    x = x0 + (np.arange(n) + 0.5) * dx
    H = np.minimum(1.0, x / 19.85)
    A = 0.3
    k = np.sqrt(3 * A / 4)
    eta_w = A / np.cosh(k * (x - 30.0)) ** 2
    wet = H > 0
    eta = np.where(x > 19.85, eta_w, np.where(wet, 0.0, -H))
    h = np.maximum(eta + H, 0.0)
    q = np.where(x > 19.85, -h * np.sqrt(G * 1.3) * eta_w / (1 + eta_w), 0.0)
    c = O.cfg(n, dx=dx, bc=(O.OUTFLOW, O.OUTFLOW, 0, 0), manning=0.01, breaking=breaking,
              B1=B1)
    w = np.zeros(n + 1)
    p = np.zeros(n + 1)
    emax = -np.inf
    t = 0.0
    while t < 6.0:
        dt = O.cfl_dt_1d(c, H, h, q)
        h, q, w, p = O.step_1d(c, H, h, q, w, p, dt)
        t += dt
        emax = max(emax, (h - H)[h > 1e-3].max())
    u = q / np.maximum(h, 1e-8)
    hn = 0.5 * (np.r_[h[0], h] + np.r_[h, h[-1]])
    E = (0.5 * q * u + 0.5 * G * (h - H) ** 2).sum() * dx + (0.5 * hn * w * w).sum() * dx
    return h, q, E, emax


def test_breaking_switch_off_limit_is_bitwise_no_breaking():
    h0, q0, _, _ = _beach(False)
    h1, q1, _, _ = _beach(True, B1=1e12)
    assert np.array_equal(h0, h1) and np.array_equal(q0, q1)


def test_breaking_dissipates():
    h0, q0, E0, m0 = _beach(False)
    h1, q1, E1, m1 = _beach(True)
    assert not np.array_equal(q0, q1)       # the mechanism was active
    assert E1 < E0
    assert m1 <= m0
