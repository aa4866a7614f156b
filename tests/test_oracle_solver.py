"""Pins of the oracle's non-hydrostatic pressure systems (CPU, no GPU).

Each check ties the oracle to something other than itself: the printed coefficients of
App. B Eq. (43) against the operator derived from Eqs. (24)-(28) (two independent
formulations), the closed form of App. B A.2, dense LU from numpy, the 1D system as the
y-invariant restriction of the 2D one, and the x/y symmetry of the 2D stencil.
"""
import numpy as np
import pytest

import oracle as O
from paper_1706_04551_b300 import inputs

RNG = np.random.default_rng(1234)


def _dense_tridiag(a, b, c, periodic):
    m = len(b)
    A = np.zeros((m, m))
    for k in range(m):
        A[k, k] += b[k]
        if periodic or k > 0:
            A[k, (k - 1) % m] += a[k]
        if periodic or k < m - 1:
            A[k, (k + 1) % m] += c[k]
    return A


def _state_1d(n, seed):
    rng = np.random.default_rng(seed)
    H = 1.0 + 0.3 * rng.random(n)
    h = H + 0.1 * rng.standard_normal(n)
    q = rng.standard_normal(n)
    w = rng.standard_normal(n + 1)
    return H, h, q, w


@pytest.mark.parametrize("bc", [O.WALL, O.OUTFLOW, O.PERIODIC])
def test_eq43_equals_operator_of_eqs_24_28(bc):
    """App. B Eq. (43) (as printed) equals, column by column, the map p -> B(dt T(p), dt p/h)
    built from the point values of Eqs. (25)-(27) and the correction of Eq. (28)."""
    n = 11
    c = O.cfg(n, dx=0.3, bc=(bc, bc, 0, 0))
    H, h, q, w = _state_1d(n, 7 + bc)
    dt = 0.05
    a, b, cc, _ = O.nh_matrix_1d(c, H, h, q, w, dt)
    A = _dense_tridiag(a, b, cc, bc == O.PERIODIC)
    m = len(b)
    G = np.zeros((m, m))
    for j in range(m):
        e = np.zeros(n + 1)
        e[j] = 1.0
        if bc == O.PERIODIC and j == 0:
            e[n] = 1.0
        G[:, j] = O.affine_apply_1d(c, H, h, e, dt)[:m]
    assert np.abs(A - G).max() <= 1e-13 * np.abs(A).max()


def test_appendix_A2_closed_form():
    """App. B A.2: h = delta, q = w = 0, H = alpha * i gives a = c = 4 (alpha^2 - delta^2),
    b = 8 (2 dx^2 + alpha^2 + delta^2), RHS = 0, and hence p = 0."""
    n, dx, alpha, delta = 16, 0.1, 0.03, 1e-5
    c = O.cfg(n, dx=dx, delta=delta)
    H = alpha * np.arange(n)
    h = np.full(n, delta)
    a, b, cc, r = O.nh_matrix_1d(c, H, h, np.zeros(n), np.zeros(n + 1), 0.01)
    inner = slice(2, n - 1)  # rows whose stencil stays off the mirrored boundary cells
    assert np.allclose(a[inner], 4 * (alpha - delta) * (alpha + delta), rtol=1e-12, atol=0)
    assert np.allclose(cc[inner], 4 * (alpha - delta) * (alpha + delta), rtol=1e-12, atol=0)
    assert np.allclose(b[inner], 8 * (2 * dx * dx + alpha ** 2 + delta ** 2), rtol=1e-12, atol=0)
    assert np.all(r == 0.0)
    # strictly diagonally dominant, as A.2 states
    assert np.all(np.abs(b) > np.abs(a) + np.abs(cc))
    p = O.nh_solve_1d(c, H, h, np.zeros(n), np.zeros(n + 1), 0.01)
    assert np.all(p == 0.0)


@pytest.mark.parametrize("bc", [O.WALL, O.OUTFLOW, O.PERIODIC])
def test_thomas_matches_dense_lu(bc):
    n = 23
    c = O.cfg(n, dx=0.2, bc=(bc, bc, 0, 0))
    H, h, q, w = _state_1d(n, 3 + bc)
    h = H + 0.02 * np.sin(np.arange(n))
    dt = 0.03
    a, b, cc, r = O.nh_matrix_1d(c, H, h, q, w, dt)
    A = _dense_tridiag(a, b, cc, bc == O.PERIODIC)
    x = np.linalg.solve(A, r)
    p = O.nh_solve_1d(c, H, h, q, w, dt)
    assert np.abs(p[: len(x)] - x).max() <= 1e-12 * np.abs(x).max()
    if bc == O.PERIODIC:
        assert p[n] == p[0]


def _dense_2d(c, H, h, dt):
    ny, nx = H.shape
    m = (nx + 1) * (ny + 1)
    M = np.zeros((m, m))
    for j in range(m):
        e = np.zeros(m)
        e[j] = 1.0
        M[:, j] = O.apply_M_2d(c, H, h, e.reshape(ny + 1, nx + 1), dt).ravel()
    return M


@pytest.mark.parametrize("bc", [O.WALL, O.OUTFLOW])
def test_2d_krylov_matches_dense_lu(bc):
    """The 2D pentadiagonal system (Sec. 5) solved by the oracle's BiCGStab equals dense LU."""
    nx, ny = 9, 7
    c = O.cfg(nx, ny, dx=0.1, dy=0.12, bc=(bc,) * 4, tol=1e-14)
    x = (np.arange(nx) + 0.5) * 0.1
    y = (np.arange(ny) + 0.5) * 0.12
    X, Y = np.meshgrid(x, y)
    H = 0.5 - 0.2 * np.exp(-((X - 0.4) ** 2 + (Y - 0.3) ** 2) / 0.05)
    h = H + 0.03 * np.cos(5 * X) * np.sin(4 * Y)
    q1 = 0.05 * np.sin(3 * X + Y)
    q2 = 0.04 * np.cos(2 * X - Y)
    w = 0.01 * RNG.standard_normal((ny + 1, nx + 1))
    dt = 0.01
    r = O.rhs_2d(c, H, h, q1, q2, w, dt)
    M = _dense_2d(c, H, h, dt)
    assert (np.abs(M) > 0).sum(1).max() == 5           # five-point stencil (Sec. 5)
    pd = np.linalg.solve(M, r.ravel())
    p, it, rs, st = O.solve_2d(c, H, h, r, dt)
    assert st == 0 and rs <= 1e-14
    assert np.abs(p.ravel() - pd).max() <= 1e-12 * np.abs(pd).max()


def test_2d_system_restricts_to_eq43():
    """On y-invariant data the 2D operator (App. A.2, Eqs. 36-41) applied to y-invariant p
    equals the 1D operator of Eq. (43), row by row; same for the right-hand sides."""
    n, ny = 13, 4
    c1 = O.cfg(n, dx=0.25)
    c2 = O.cfg(n, ny, dx=0.25)
    H, h, q, w = _state_1d(n, 11)
    h = H + 0.05 * np.cos(np.arange(n))
    dt = 0.02
    p = RNG.standard_normal(n + 1)
    a, b, cc, r1 = O.nh_matrix_1d(c1, H, h, q, w, dt)
    A = _dense_tridiag(a, b, cc, False)
    T = lambda v: np.tile(v, (ny, 1))
    out2 = O.apply_M_2d(c2, T(H), T(h), np.tile(p, (ny + 1, 1)), dt)
    for J in range(ny + 1):
        assert np.abs(out2[J] - A @ p).max() <= 1e-12 * np.abs(A @ p).max()
    r2 = O.rhs_2d(c2, T(H), T(h), T(q), np.zeros((ny, n)), np.tile(w, (ny + 1, 1)), dt)
    for J in range(ny + 1):
        assert np.abs(r2[J] - r1).max() <= 1e-12 * np.abs(r1).max()


def test_2d_system_transpose_symmetry():
    """Swapping the roles of x and y (transposed fields, q1 <-> q2) transposes the system."""
    nx, ny = 8, 6
    c = O.cfg(nx, ny, dx=0.1, dy=0.1)
    ct = O.cfg(ny, nx, dx=0.1, dy=0.1)
    H = 0.4 + 0.1 * RNG.random((ny, nx))
    h = H + 0.02 * RNG.standard_normal((ny, nx))
    q1, q2 = 0.1 * RNG.standard_normal((2, ny, nx))
    w = 0.01 * RNG.standard_normal((ny + 1, nx + 1))
    p = RNG.standard_normal((ny + 1, nx + 1))
    dt = 0.01
    Mp = O.apply_M_2d(c, H, h, p, dt)
    Mpt = O.apply_M_2d(ct, H.T.copy(), h.T.copy(), p.T.copy(), dt)
    assert np.abs(Mp.T - Mpt).max() <= 1e-12 * np.abs(Mp).max()
    r = O.rhs_2d(c, H, h, q1, q2, w, dt)
    rt = O.rhs_2d(ct, H.T.copy(), h.T.copy(), q2.T.copy(), q1.T.copy(), w.T.copy(), dt)
    assert np.abs(r.T - rt).max() <= 1e-12 * np.abs(r).max()


@pytest.mark.parametrize("which", ["shoals", "island"])
def test_2d_matrix_strictly_diagonally_dominant_on_workloads(which):
    """Sec. 5 reports that the matrices were strictly diagonally dominant in all its tests;
    check the same on the (coarsened) synthetic workloads."""
    if which == "shoals":
        wl = inputs.shoals_2d(n=24)
    else:
        wl = inputs.island_2d(n=48, L=19.2, center=(9.6, None), x0=3.0)
    c = O.cfg(wl.nx, wl.ny, dx=wl.dx, bc=wl.bc)
    dt = 0.5 * O.cfl_dt_2d(c, wl.H, wl.h, wl.q1, wl.q2)
    M = _dense_2d(c, wl.H, wl.h, dt)
    D = np.abs(np.diag(M))
    off = np.abs(M).sum(1) - D
    assert np.all(D > off)
