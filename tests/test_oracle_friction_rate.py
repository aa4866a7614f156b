"""Pins of the oracle's semi-implicit Manning friction and of the 2D Eq. (23) time step.

Friction (Sec. 2 source term -g n^2 |u| q / h^(4/3), taken semi-implicitly in each stage):
on a flat bottom with a uniform flow every flux difference vanishes, the pressure system's
right-hand side is zero and the flow only decays.  The continuous decay is the ODE
dq/dt = -k |q| q with k = g n^2 / h^(7/3) (h fixed), solved by
q(t) = q0 / (1 + k |q0| t).  The scheme must converge to it at first order in dt (each
stage is a backward-Euler-like update, and their average keeps the O(dt^2) local error).
A wrong depth exponent (h^(7/3) instead of h^(4/3)) or |q| in place of |u| changes k by a
factor of h and fails the convergence at h = 0.5 m.
"""
import numpy as np
import pytest

import oracle as O

G = 9.81


def uniform_2d(n, h0, u0, v0):
    h = np.full((n, n), h0)
    return h, h * u0, h * v0


def exact_speed(q0, k, t):
    return q0 / (1.0 + k * q0 * t)


@pytest.mark.parametrize("nonhydro", [True, False])
def test_manning_decay_converges_to_the_ode_at_first_order(nonhydro):
    n, h0, u0, v0, nm, T = 8, 0.5, 0.6, -0.3, 0.05, 4.0
    k = G * nm * nm / h0 ** (7.0 / 3.0)
    c = O.cfg(n, n, dx=0.5, bc=(O.OUTFLOW,) * 4, manning=nm, nonhydro=nonhydro)
    H = np.full((n, n), h0)
    z = np.zeros((n + 1, n + 1))
    errs = []
    for steps in (20, 40, 80, 160):
        h, a, b = uniform_2d(n, h0, u0, v0)
        ho, ao, bo, wo, po, t, s, it = O.run_2d(c, H, h, a, b, z, z, max_steps=steps,
                                                fixed_dt=T / steps)
        # uniform flow stays uniform: depth unchanged, direction unchanged
        assert np.abs(ho - h0).max() < 1e-13
        assert np.abs(ao * v0 - bo * u0).max() < 1e-13
        qmag = np.hypot(ao, bo)
        errs.append(np.abs(qmag - exact_speed(h0 * np.hypot(u0, v0), k, T)).max())
    ratios = [errs[i] / errs[i + 1] for i in range(len(errs) - 1)]
    assert all(1.8 < r < 2.2 for r in ratios), (errs, ratios)
    assert errs[-1] < 2e-3 * h0 * np.hypot(u0, v0)


def test_manning_decay_1d_converges_to_the_ode():
    n, h0, u0, nm, T = 16, 0.5, 0.8, 0.05, 3.0
    k = G * nm * nm / h0 ** (7.0 / 3.0)
    c = O.cfg(n, dx=0.5, bc=(O.OUTFLOW, O.OUTFLOW, 0, 0), manning=nm)
    H = np.full(n, h0)
    errs = []
    for steps in (30, 60, 120):
        h, q = np.full(n, h0), np.full(n, h0 * u0)
        ho, qo, wo, po, t, s = O.run_1d(c, H, h, q, np.zeros(n + 1), np.zeros(n + 1),
                                        max_steps=steps, fixed_dt=T / steps)
        errs.append(np.abs(qo - exact_speed(h0 * u0, k, T)).max())
    ratios = [errs[i] / errs[i + 1] for i in range(len(errs) - 1)]
    assert all(1.8 < r < 2.2 for r in ratios), (errs, ratios)


def test_manning_limit_without_friction_keeps_the_flow():
    n = 8
    c = O.cfg(n, n, dx=0.5, bc=(O.OUTFLOW,) * 4, manning=0.0)
    h, a, b = uniform_2d(n, 0.5, 0.6, -0.3)
    z = np.zeros((n + 1, n + 1))
    ho, ao, bo, *_ = O.run_2d(c, np.full((n, n), 0.5), h, a, b, z, z, max_steps=10,
                              fixed_dt=0.05)
    assert np.abs(ao - a).max() < 1e-14 and np.abs(bo - b).max() < 1e-14


# ------------------------------------------------------------------- Eq. (23), 2D rate


@pytest.mark.parametrize("u,v,dx,dy", [(0.7, -0.2, 0.1, 0.25), (-0.1, 0.9, 0.3, 0.05),
                                       (0.0, 0.0, 0.2, 0.1)])
def test_rate_2d_on_uniform_states(u, v, dx, dy):
    """On a uniform state of depth h the Eq. (23) step is CFL / ((|u| + c)/dx +
    (|v| + c)/dy), c = sqrt(g h), with u != v and dx != dy (a max(|u|, |v|) speed or a
    dropped y term fails)."""
    n, h0, cfl = 6, 0.4, 0.9
    c = O.cfg(n, n, dx=dx, dy=dy, cfl=cfl)
    h, a, b = uniform_2d(n, h0, u, v)
    cw = np.sqrt(G * h0)
    want = cfl / ((abs(u) + cw) / dx + (abs(v) + cw) / dy)
    got = O.cfl_dt_2d(c, np.full((n, n), h0), h, a, b)
    assert abs(got - want) <= 1e-14 * want


def test_rate_2d_takes_the_fastest_cell_and_scales_with_the_mesh():
    """The step is set by the cell with the largest rate (a single fast cell among slow
    ones), and scaling dx, dy by s scales it by s."""
    n, h0 = 10, 0.4
    h, a, b = uniform_2d(n, h0, 0.1, 0.05)
    h[3, 7], a[3, 7], b[3, 7] = 0.9, 0.9 * 1.3, 0.9 * -0.4
    H = np.full((n, n), h0)
    cw = np.sqrt(G * 0.9)
    for s in (1.0, 3.0):
        c = O.cfg(n, n, dx=0.1 * s, dy=0.2 * s, cfl=0.8)
        want = 0.8 / ((1.3 + cw) / (0.1 * s) + (0.4 + cw) / (0.2 * s))
        assert abs(O.cfl_dt_2d(c, H, h, a, b) - want) <= 1e-14 * want


def test_rate_2d_y_invariant_state_reduces_to_the_1d_rate():
    """With v = 0 and dy -> large, the 2D step tends to the 1D step of Eq. (23) (the
    y term only adds sqrt(g h) / dy)."""
    n = 12
    x = np.linspace(0, 1, n)
    h1 = 0.5 + 0.1 * np.sin(3 * x)
    q1 = 0.2 * np.cos(2 * x)
    c1 = O.cfg(n, dx=0.1, cfl=0.9)
    d1 = O.cfl_dt_1d(c1, np.full(n, 0.5), h1, q1)
    h = np.tile(h1, (4, 1))
    a = np.tile(q1, (4, 1))
    c2 = O.cfg(n, 4, dx=0.1, dy=1e9, cfl=0.9)
    d2 = O.cfl_dt_2d(c2, np.full((4, n), 0.5), h, a, np.zeros_like(a))
    assert abs(d2 - d1) <= 1e-9 * d1
