"""Hand-written GPU adjoint (nh_step_taped / nh_adjoint_step behind torch.autograd) against
the FP64 oracle adjoint (oracle/adjoint.py) and against central finite differences of the
GPU forward; checkpointed recomputation against a single segment."""
import numpy as np
import pytest
import torch

from oracle import adjoint as A
from paper_1706_04551_b300 import inputs, nh
from paper_1706_04551_b300.adjoint import gauge_series, misfit

pytestmark = pytest.mark.gpu


def rel(x, ref):
    x, ref = np.asarray(x, np.float64), np.asarray(ref, np.float64)
    s = np.abs(ref).max()
    return np.abs(x - ref).max() / (s if s > 0 else 1.0)


def small_case(nx=14, ny=11, seed=0):
    rng = np.random.default_rng(seed)
    dx = 0.1
    y, x = np.mgrid[0:ny, 0:nx] / max(nx, ny)
    H = 0.55 + 0.25 * np.sin(3 * x + rng.uniform(0, 6)) * np.cos(2 * y + rng.uniform(0, 6))
    eta = 0.03 * np.cos(4 * x + rng.uniform(0, 6)) * np.sin(3 * y + 1.0)
    h = eta + H
    q1 = 0.02 * h * np.sin(2 * x + 0.3) * np.cos(1.3 * y + 0.2)
    q2 = 0.02 * h * np.cos(3 * y + 0.7) * np.sin(1.7 * x + 0.4)
    return H, eta, q1, q2, dx


def gpu_grad(H, eta, q1, q2, dx, dt, nsteps, gauges, target, precision="fp64", checkpoint=2,
             bc=(0, 0, 0, 0), **kw):
    kw.setdefault("tol", 1e-13 if precision == "fp64" else 1e-5)
    T = lambda a: torch.tensor(a, dtype=torch.float64, requires_grad=True)
    Ht, et, at, bt = T(H), T(eta), T(q1), T(q2)
    s = gauge_series(Ht, et, at, bt, dx=dx, dt=dt, nsteps=nsteps, gauges=gauges,
                     precision=precision, checkpoint=checkpoint, bc=bc, **kw)
    J = misfit(s, torch.tensor(target, dtype=torch.float64))
    J.backward()
    return float(J), Ht.grad.numpy(), et.grad.numpy(), at.grad.numpy(), bt.grad.numpy()


def oracle_grad(H, eta, q1, q2, dx, dt, nsteps, gauges, target, bc=(0, 0, 0, 0), frozen=0):
    ny, nx = H.shape
    c = A.Cfg2(nx, ny, dx, dx, bc, frozen_limiter=bool(frozen))
    Tq = lambda a: torch.tensor(a, dtype=torch.float64, requires_grad=True)
    Ht, et, at, bt = Tq(H), Tq(eta), Tq(q1), Tq(q2)
    J = A.gauge_misfit(c, Ht, et, at, bt, dt, nsteps, gauges, torch.tensor(target))
    gH, ge, ga, gb = torch.autograd.grad(J, (Ht, et, at, bt))
    return float(J.detach()), gH.numpy(), ge.numpy(), ga.numpy(), gb.numpy()


def setup(bc=(0, 0, 0, 0), nsteps=4):
    H, eta, q1, q2, dx = small_case()
    gauges = [(2, 3), (5, 8), (7, 1), (4, 11), (9, 6)]
    rng = np.random.default_rng(9)
    target = 0.01 * rng.standard_normal((nsteps, len(gauges)))
    h = eta + H
    lam = np.max((np.abs(q1 / h) + np.sqrt(9.81 * h)) / dx + (np.abs(q2 / h) + np.sqrt(9.81 * h)) / dx)
    dt = 0.9 / lam
    return H, eta, q1, q2, dx, dt, nsteps, gauges, target


@pytest.mark.parametrize("bc,frozen", [((0, 0, 0, 0), 0), ((1, 1, 0, 1), 0), ((0, 0, 0, 0), 1)])
def test_fp64_adjoint_equals_oracle_adjoint(bc, frozen):
    H, eta, q1, q2, dx, dt, nsteps, gauges, target = setup(bc)
    Jg, gH, ge, ga, gb = gpu_grad(H, eta, q1, q2, dx, dt, nsteps, gauges, target, bc=bc,
                                  adjoint_frozen_limiter=frozen)
    Jo, oH, oe, oa, ob = oracle_grad(H, eta, q1, q2, dx, dt, nsteps, gauges, target, bc=bc,
                                     frozen=frozen)
    assert Jg == pytest.approx(Jo, rel=1e-10)
    assert rel(gH, oH) < 1e-8 and rel(ge, oe) < 1e-8
    assert rel(ga, oa) < 1e-8 and rel(gb, ob) < 1e-8


def test_fp32_adjoint_against_oracle_adjoint():
    H, eta, q1, q2, dx, dt, nsteps, gauges, target = setup()
    Jg, gH, ge, ga, gb = gpu_grad(H, eta, q1, q2, dx, dt, nsteps, gauges, target, "fp32")
    Jo, oH, oe, oa, ob = oracle_grad(H, eta, q1, q2, dx, dt, nsteps, gauges, target)
    assert rel(gH, oH) < 2e-3 and rel(ge, oe) < 2e-3


def test_checkpoint_segments_equal_single_segment():
    H, eta, q1, q2, dx, dt, nsteps, gauges, target = setup(nsteps=6)
    a = gpu_grad(H, eta, q1, q2, dx, dt, nsteps, gauges, target, checkpoint=6)
    b = gpu_grad(H, eta, q1, q2, dx, dt, nsteps, gauges, target, checkpoint=2)
    for x, y in zip(a[1:], b[1:]):
        assert rel(y, x) < 1e-11


def adjoint_workload(n, nsteps, sigma):
    wl = inputs.adjoint_2d(n=n, hump_sigma=sigma)
    gauges = [tuple(g) for g in wl.extra["gauges"]]
    h = wl.eta + wl.H
    dt = 0.9 / np.max(2 * np.sqrt(9.81 * h) / wl.dx)
    rng = np.random.default_rng(1)
    target = 0.002 * rng.standard_normal((nsteps, len(gauges)))
    return wl, gauges, dt, target


def J_fp64(wl, HH, ee, dt, nsteps, gauges, target):
    with torch.no_grad():
        s = gauge_series(torch.tensor(HH), torch.tensor(ee), dx=wl.dx, dt=dt, nsteps=nsteps,
                         gauges=gauges, precision="fp64", checkpoint=nsteps, tol=1e-13)
        return float(misfit(s, torch.tensor(target)))


@pytest.mark.parametrize("nsteps,bar", [(20, 1e-5), (40, 5e-5)])
def test_bathymetry_gradient_against_central_differences(nsteps, bar):
    """The adjoint workload's recipe at 96^2 (walls, Gaussian-sum depth 0.3 .. 0.8 m, hump,
    fixed dt), 16 gauges: <dJ/dH, d> of the exact FP64 adjoint against central differences
    of the GPU FP64 forward along two smooth directions.  The differences must take
    eps <= 1e-6: with larger eps the minmod branches switch inside +-eps and the
    differences scatter (measured at 10 steps: 1e-4 at eps 1e-4, 5e-5 at 1e-5, 6e-9 at
    1e-6).  At eps 1e-6 the adjoint meets 1e-5 over 20 steps (2e-9 and below); over 40
    steps the two directions agree to 1.5e-6 and 2.0e-5."""
    wl, gauges, dt, target = adjoint_workload(96, nsteps, 1.0)
    z = np.zeros_like(wl.H)
    J, gH, ge, _, _ = gpu_grad(wl.H, wl.eta, z, z, wl.dx, dt, nsteps, gauges, target,
                               checkpoint=10)
    y, x = np.mgrid[0:96, 0:96] / 96.0
    rng = np.random.default_rng(3)
    eps = 1e-6
    for k in range(2):
        d = np.sin((k + 2) * 3.1 * x + rng.uniform(0, 6)) * np.cos((k + 1) * 2.3 * y + rng.uniform(0, 6))
        fd = (J_fp64(wl, wl.H + eps * d, wl.eta, dt, nsteps, gauges, target) -
              J_fp64(wl, wl.H - eps * d, wl.eta, dt, nsteps, gauges, target)) / (2 * eps)
        assert abs(float((gH * d).sum()) - fd) <= bar * abs(fd), (k, float((gH * d).sum()), fd)


def test_exact_adjoint_grows_and_frozen_limiter_adjoint_stays_bounded():
    """The exact derivative with respect to eta0 grows by a grid-scale mode (the active
    minmod branches linearise to an unlimited, partly central reconstruction, which the
    Runge-Kutta stages do not damp); the frozen-limiter linearisation stays bounded."""
    nsteps = 60
    wl, gauges, dt, target = adjoint_workload(96, nsteps, 1.0)
    z = np.zeros_like(wl.H)
    out = {}
    for frozen in (0, 1):
        J, gH, ge, _, _ = gpu_grad(wl.H, wl.eta, z, z, wl.dx, dt, nsteps, gauges, target,
                                   checkpoint=20, adjoint_frozen_limiter=frozen)
        assert np.isfinite(gH).all() and np.isfinite(ge).all()
        out[frozen] = np.abs(ge).max()
    assert out[0] > 1e3 * out[1]


def test_adjoint_rejects_friction():
    H, eta, q1, q2, dx = small_case()
    sim = nh.Sim(H, dx, precision="fp64", manning_n=0.01)
    tape = torch.empty(sim.tape_bytes(), dtype=torch.uint8, device="cuda")
    sim.set_state(eta, q1, q2)
    sim.step_taped(tape, 1e-3)
    z = [torch.zeros(H.size, dtype=torch.float64, device="cuda") for _ in range(3)]
    wz = torch.zeros((H.shape[0] + 1) * (H.shape[1] + 1), dtype=torch.float64, device="cuda")
    with pytest.raises(nh.NHError):
        sim.adjoint_step(tape, 1e-3, z[0], z[1], z[2], wz, torch.zeros_like(z[0]))


def test_adjoint_rejects_the_literal_wet_dry_form():
    H, eta, q1, q2, dx = small_case()
    sim = nh.Sim(H, dx, precision="fp64", dry_zero=0)
    tape = torch.empty(sim.tape_bytes(), dtype=torch.uint8, device="cuda")
    sim.set_state(eta, q1, q2)
    with pytest.raises(nh.NHError) as ei:
        sim.step_taped(tape, 1e-3)
    assert ei.value.code == nh.EINVAL
    sim.close()


def test_adjoint_of_refined_fp64_steps_equals_plain():
    """Taped steps whose pressure solves are refined in FP32 (refine_fp32) give the
    gradient of the plain FP64 steps to the solver tolerance's order."""
    H, eta, q1, q2, dx, dt, nsteps, gauges, target = setup()
    a = gpu_grad(H, eta, q1, q2, dx, dt, nsteps, gauges, target)
    b = gpu_grad(H, eta, q1, q2, dx, dt, nsteps, gauges, target, refine_fp32=1)
    assert b[0] == pytest.approx(a[0], rel=1e-10)
    for x, y in zip(a[1:], b[1:]):
        assert rel(y, x) < 1e-8
