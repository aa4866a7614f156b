"""Pins of the FP64 oracle adjoint (oracle/adjoint.py): its forward is the C oracle's step,
its gradient equals central finite differences of the C oracle's forward, and its
Jacobian products satisfy the dot-product identity."""
import numpy as np
import pytest
import torch

import oracle as O
from oracle import adjoint as A
from paper_1706_04551_b300 import inputs


def small_case(nx=12, ny=10, seed=0):
    """All-wet smooth basin (depth 0.3 .. 0.8 m) with a moving smooth state."""
    rng = np.random.default_rng(seed)
    dx = 0.1
    y, x = np.mgrid[0:ny, 0:nx] / max(nx, ny)
    H = 0.55 + 0.25 * np.sin(3 * x + rng.uniform(0, 6)) * np.cos(2 * y + rng.uniform(0, 6))
    eta = 0.03 * np.cos(4 * x + rng.uniform(0, 6)) * np.sin(3 * y + 1.0)
    h = eta + H
    # generic (no velocity slope exactly zero: minmod is not differentiable at 0 / 0)
    q1 = 0.02 * h * np.sin(2 * x + 0.3) * np.cos(1.3 * y + 0.2)
    q2 = 0.02 * h * np.cos(3 * y + 0.7) * np.sin(1.7 * x + 0.4)
    return H, h, q1, q2, dx


def c_oracle_cfg(nx, ny, dx, bc=(0, 0, 0, 0)):
    return O.cfg(nx, ny, dx=dx, bc=bc, tol=1e-15, max_iter=20000)


@pytest.mark.parametrize("bc", [(0, 0, 0, 0), (1, 1, 0, 1)])
def test_forward_step_equals_c_oracle(bc):
    H, h, q1, q2, dx = small_case()
    ny, nx = H.shape
    rng = np.random.default_rng(3)
    w = 0.005 * rng.standard_normal((ny + 1, nx + 1))
    p0 = np.zeros((ny + 1, nx + 1))
    c = c_oracle_cfg(nx, ny, dx, bc)
    dt = 0.5 * O.cfl_dt_2d(c, H, h, q1, q2)
    ho, ao, bo, wo, po, _ = O.step_2d(c, H, h, q1, q2, w, p0, dt)
    ct = A.Cfg2(nx, ny, dx, dx, bc)
    T = lambda a: torch.as_tensor(a, dtype=torch.float64)
    hh, aa, bb, ww, pp = A.step(ct, T(H), T(h), T(q1), T(q2), T(w), dt)
    for got, ref in ((hh, ho), (aa, ao), (bb, bo), (ww, wo), (pp, po)):
        ref = np.asarray(ref)
        assert np.abs(got.numpy() - ref).max() <= 1e-11 * max(np.abs(ref).max(), 1e-30)


@pytest.mark.parametrize("dry_zero", [False, True])
def test_forward_wet_dry_equals_c_oracle(dry_zero):
    wl = inputs.island_2d(n=24, L=9.6, center=(4.8, None), x0=2.0)
    ny, nx = wl.H.shape
    h = np.maximum(wl.eta + wl.H, 0)
    c = O.cfg(nx, ny, dx=wl.dx, bc=wl.bc, tol=1e-15, max_iter=20000, dry_zero=dry_zero)
    dt = 0.5 * O.cfl_dt_2d(c, wl.H, h, wl.q1, wl.q2)
    z = np.zeros((ny + 1, nx + 1))
    ho, ao, bo, wo, po, _ = O.step_2d(c, wl.H, h, wl.q1, wl.q2, z, z, dt)
    ct = A.Cfg2(nx, ny, wl.dx, wl.dx, wl.bc, dry_zero=dry_zero)
    T = lambda a: torch.as_tensor(a, dtype=torch.float64)
    hh, aa, bb, ww, pp = A.step(ct, T(wl.H), T(h), T(wl.q1), T(wl.q2), T(z), dt)
    for got, ref in ((hh, ho), (aa, ao), (bb, bo), (pp, po)):
        assert np.abs(got.numpy() - ref).max() <= 1e-10 * max(np.abs(ref).max(), 1e-30)


def c_oracle_misfit(c, H, eta0, q1, q2, dt, nsteps, gauges, target):
    ny, nx = H.shape
    h, w, p = eta0 + H, np.zeros((ny + 1, nx + 1)), np.zeros((ny + 1, nx + 1))
    J = 0.0
    for n in range(nsteps):
        h, q1, q2, w, p, _ = O.step_2d(c, H, h, q1, q2, w, p, dt)
        eta = h - H
        J += sum((eta[i, j] - target[n][k]) ** 2 for k, (i, j) in enumerate(gauges))
    return J


def misfit_setup(nsteps=3):
    H, h, q1, q2, dx = small_case(seed=1)
    ny, nx = H.shape
    eta0 = h - H
    gauges = [(2, 3), (5, 8), (7, 1), (4, 6)]
    rng = np.random.default_rng(9)
    target = 0.01 * rng.standard_normal((nsteps, len(gauges)))
    c = c_oracle_cfg(nx, ny, dx)
    dt = O.cfl_dt_2d(c, H, h, q1, q2)
    return H, eta0, q1, q2, dx, gauges, target, c, dt


def test_gradient_equals_central_differences_of_the_c_oracle():
    nsteps = 3
    H, eta0, q1, q2, dx, gauges, target, c, dt = misfit_setup(nsteps)
    ny, nx = H.shape
    ct = A.Cfg2(nx, ny, dx, dx)
    J, gH, ge = A.gradient(ct, H, eta0, q1, q2, dt, nsteps, gauges, target)
    assert J == pytest.approx(c_oracle_misfit(c, H, eta0, q1, q2, dt, nsteps, gauges, target),
                              rel=1e-10)
    rng = np.random.default_rng(11)
    y, x = np.mgrid[0:ny, 0:nx] / max(nx, ny)
    for k in range(2):
        d = np.sin((k + 2) * x + rng.uniform(0, 6)) * np.cos((k + 1) * y + rng.uniform(0, 6))
        eps = 1e-5
        for which, g in (("H", gH), ("eta0", ge)):
            def Jat(s):
                if which == "H":
                    return c_oracle_misfit(c, H + s * d, eta0, q1, q2, dt, nsteps, gauges, target)
                return c_oracle_misfit(c, H, eta0 + s * d, q1, q2, dt, nsteps, gauges, target)
            fd = (Jat(eps) - Jat(-eps)) / (2 * eps)
            ad = float((g * d).sum())
            assert abs(ad - fd) <= 1e-6 * abs(fd) + 1e-14, (which, k, ad, fd)


def test_dot_product_identity_of_the_step_map():
    H, h, q1, q2, dx = small_case(seed=2)
    ny, nx = H.shape
    ct = A.Cfg2(nx, ny, dx, dx)
    c = c_oracle_cfg(nx, ny, dx)
    dt = O.cfl_dt_2d(c, H, h, q1, q2)
    rng = np.random.default_rng(5)
    T = lambda a: torch.as_tensor(a, dtype=torch.float64)
    w = T(0.003 * rng.standard_normal((ny + 1, nx + 1)))
    Ht = T(H)

    def F(hh, aa, bb, ww, HH):
        out = A.step(ct, HH, hh, aa, bb, ww, dt)
        return out[0], out[1], out[2], out[3]

    x0 = (T(h), T(q1), T(q2), w, Ht)
    v = tuple(T(rng.standard_normal(a.shape)) * 1e-3 for a in x0)
    lam = tuple(T(rng.standard_normal(a.shape)) for a in x0[:4])
    _, Jv = torch.func.jvp(F, x0, v)
    _, vjp = torch.func.vjp(F, *x0)
    JTl = vjp(lam)
    lhs = sum(float((a * b).sum()) for a, b in zip(Jv, lam))
    rhs = sum(float((a * b).sum()) for a, b in zip(v, JTl))
    assert abs(lhs - rhs) <= 1e-12 * max(abs(lhs), 1e-30)
