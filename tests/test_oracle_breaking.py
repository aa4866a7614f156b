"""Closed-form pins of the oracle's breaking terms (Sec. 3, Eq. 12; 2D with q_x -> div q and
u_x -> div u).

On a constant depth h0 with linear discharges and a linear bathymetry, every centred
difference the terms use is exact, so each interior cell and node must carry the paper's
formulas evaluated by hand: nu = B h |d| with d = q_x (div q), U1 = B1 sqrt(g h),
B = 1 - d / U1, active where |d| >= U1 and B > 0; cells q += dt 2 nu u_x H_x (and H_y);
nodes w += dt 2 nu u_x / h.  Both sides of the switch are checked: a converging flow with
d = -2 U1 (B = 3) and a diverging one with d = +2 U1 (B < 0: no term).
"""
import numpy as np
import pytest

import oracle as O

G = 9.81


@pytest.mark.parametrize("factor", [-2.0, -1.2, 2.0, -0.5])
def test_breaking_1d_closed_form(factor):
    n, dx, h0, B1, dt = 64, 0.1, 0.8, 0.15, 0.01
    U1 = B1 * np.sqrt(G * h0)
    a = factor * U1                         # q_x
    alpha = 0.05                            # H_x
    x = (np.arange(n) + 0.5) * dx
    H = 0.7 + alpha * x
    h = np.full(n, h0)
    q = 0.3 + a * x
    w = np.linspace(-0.01, 0.02, n + 1)
    c = O.cfg(n, dx=dx, B1=B1, breaking=True)
    qo, wo = O.breaking_1d(c, H, h, q, w, dt)
    B = 1.0 - a / U1
    on = abs(a) >= U1 and B > 0
    nu = B * h0 * abs(a) if on else 0.0
    ux = a / h0
    cells = slice(2, n - 2)                  # away from the wall ghosts
    assert np.allclose(qo[cells] - q[cells], dt * 2 * nu * ux * alpha, rtol=1e-10, atol=1e-15)
    nodes = slice(2, n - 1)
    assert np.allclose(wo[nodes] - w[nodes], dt * 2 * nu * ux / h0, rtol=1e-10, atol=1e-15)
    if on:
        assert np.all(np.abs(qo[cells] - q[cells]) > 0)


@pytest.mark.parametrize("fx,fy", [(-1.5, -1.0), (1.0, 1.5), (-0.3, 0.2)])
def test_breaking_2d_closed_form(fx, fy):
    nx, ny, dx, dy, h0, B1, dt = 40, 32, 0.1, 0.12, 0.6, 0.15, 0.01
    U1 = B1 * np.sqrt(G * h0)
    a1, a2 = fx * U1, fy * U1                # q1_x, q2_y: div q = a1 + a2
    al, be = 0.04, -0.03                     # H_x, H_y
    x = (np.arange(nx) + 0.5) * dx
    y = (np.arange(ny) + 0.5) * dy
    X, Y = np.meshgrid(x, y)
    H = 0.5 + al * X + be * Y
    h = np.full((ny, nx), h0)
    q1 = 0.1 + a1 * X
    q2 = -0.2 + a2 * Y
    w = np.zeros((ny + 1, nx + 1))
    c = O.cfg(nx, ny, dx=dx, dy=dy, B1=B1, breaking=True)
    r1, r2, rw = O.breaking_2d(c, H, h, q1, q2, w, dt)
    d = a1 + a2
    B = 1.0 - d / U1
    nu = B * h0 * abs(d) if (abs(d) >= U1 and B > 0) else 0.0
    du = d / h0
    ci = (slice(2, ny - 2), slice(2, nx - 2))
    assert np.allclose(r1[ci] - q1[ci], dt * 2 * nu * du * al, rtol=1e-10, atol=1e-15)
    assert np.allclose(r2[ci] - q2[ci], dt * 2 * nu * du * be, rtol=1e-10, atol=1e-15)
    ni = (slice(2, ny - 1), slice(2, nx - 1))
    assert np.allclose(rw[ni], dt * 2 * nu * du / h0, rtol=1e-10, atol=1e-15)
    assert (nu > 0) == (fx + fy <= -1.0)
