"""Energy-consistent w equation on the CUDA path (nh_params.w_equation = NH_W_TRANSPORT:
(hw)_t + div(hw u) = p, Sec. 2) against the FP64 oracle's `w_transport` form.

Bars: FP64 within 1e-10 relative L-infinity on h, the discharge, w and p (as the other
parity tests); FP32 within 1e-4 on eta and on w.  Plus the form's invariant at a size the
oracle does not reach: a uniform w stays uniform on any wet flow (hydrostatic mode).
"""
import numpy as np
import pytest

import oracle as O
from paper_1706_04551_b300 import inputs, nh
from test_gpu_parity import developed, island, make, rel, rel_q, shoals

pytestmark = pytest.mark.gpu


def _w0(wl, seed=9, amp=0.01):
    ny, nx = wl.H.shape
    y, x = np.mgrid[0:ny + 1, 0:nx + 1] / max(nx, ny)
    ph = np.random.default_rng(seed).uniform(0, 2 * np.pi, 2)
    return amp * np.sin(7 * x + ph[0]) * np.cos(4 * y + ph[1])


def _both(wl, steps, precision="fp64", seed=0, **kw):
    sim, c = make(wl, precision, w_equation=nh.W_TRANSPORT, **kw)
    c.w_transport = 1
    eta, q1, q2 = developed(wl, seed=seed)
    w0 = _w0(wl)
    dt = sim.dtype
    sim.set_state(eta.astype(dt), q1.astype(dt), q2.astype(dt), w=w0.astype(dt))
    for _ in range(steps):
        sim.step()
    g = sim.get_state()
    sim.close()
    h = np.maximum(eta + wl.H, 0)
    ro = O.run_2d(c, wl.H, h, q1, q2, w0, np.zeros_like(w0), max_steps=steps)
    return g, ro


@pytest.mark.parametrize("which,nonhydro", [("shoals", 1), ("island", 1), ("island", 0)])
def test_2d_fp64_matches_oracle(which, nonhydro):
    wl = shoals(64) if which == "shoals" else island(64)
    g, (h, q1, q2, w, p, t, s, it) = _both(wl, 12, nonhydrostatic=nonhydro)
    assert rel(g["eta"] + wl.H, h) < 1e-10
    assert rel_q(g["q1"], g["q2"], q1, q2) < 1e-10
    assert rel(g["w"], w) < 1e-10
    if nonhydro:
        assert rel(g["p"], p) < 1e-10
    assert abs(g["t"] - t) < 1e-12 * t


def test_the_two_w_equations_differ():
    """The option reaches the kernels: the same steps with h w_t = p end elsewhere."""
    wl = shoals(64)
    g, _ = _both(wl, 6)
    sim, _ = make(wl, "fp64")
    eta, q1, q2 = developed(wl)
    sim.set_state(eta, q1, q2, w=_w0(wl))
    for _ in range(6):
        sim.step()
    g0 = sim.get_state()
    sim.close()
    assert rel(g["w"], g0["w"]) > 1e-6


def test_2d_fp32_matches_oracle():
    wl = shoals(96)
    g, (h, q1, q2, w, p, t, s, it) = _both(wl, 10, "fp32")
    e_eta, e_w = rel(g["eta"], h - wl.H), rel(g["w"], w)
    print(f"fp32 eta {e_eta:.2e} w {e_w:.2e}")
    assert e_eta < 1e-4 and e_w < 1e-4


@pytest.mark.parametrize("bc", [(nh.WALL, nh.WALL), (nh.PERIODIC, nh.PERIODIC),
                                (nh.OUTFLOW, nh.OUTFLOW)])
def test_1d_channels_match_oracle_fp64(bc):
    wl = inputs.solitary_1d(n=300, L=60.0, x0=20.0)
    n = wl.nx
    rng = np.random.default_rng(4)
    w0 = 0.01 * rng.standard_normal(n + 1)
    if bc[0] == nh.PERIODIC:
        w0[n] = w0[0]
    sim = nh.Sim(wl.H, wl.dx, dim=1, bc=bc + (0, 0), precision="fp64", cfl=0.9,
                 w_equation=nh.W_TRANSPORT)
    sim.set_state(wl.eta[None, :], wl.q1[None, :], w=w0[None, :])
    steps = 40
    for _ in range(steps):
        sim.step()
    g = sim.get_state()
    sim.close()
    c = O.cfg(n, dx=wl.dx, cfl=0.9, bc=bc + (0, 0), w_transport=True)
    h, q, w, p, t, s = O.run_1d(c, wl.H, wl.h, wl.q1, w0, np.zeros(n + 1), max_steps=steps)
    assert rel(g["eta"][0] + wl.H, h) < 1e-10
    assert rel(g["q1"][0], q) < 1e-10
    assert rel(g["w"][0], w) < 1e-10 and rel(g["p"][0], p) < 1e-10


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("fp32", 1e-5)])
def test_uniform_w_stays_uniform_at_size(precision, tol):
    """2048^2 shoals basin, hydrostatic mode, outflow sides: w = 0.3 everywhere stays 0.3."""
    wl = inputs.shoals_2d(n=2048)
    wl.bc = (nh.OUTFLOW,) * 4
    sim, _ = make(wl, precision, w_equation=nh.W_TRANSPORT, nonhydrostatic=0)
    eta, q1, q2 = developed(wl, seed=2, amp=0.05)
    dt = sim.dtype
    sim.set_state(eta.astype(dt), q1.astype(dt), q2.astype(dt),
                  w=np.full((wl.ny + 1, wl.nx + 1), 0.3, dt))
    for _ in range(5):
        sim.step()
    g = sim.get_state()
    sim.close()
    assert np.max(np.abs(g["w"].astype(np.float64) - 0.3)) < tol * 0.3


def test_variant_is_rejected_where_it_is_not_built():
    wl = shoals(32)
    with pytest.raises(nh.NHError):
        nh.Batch([wl.H, wl.H], dx=wl.dx, precision="fp32", w_equation=nh.W_TRANSPORT)
    import torch
    sim, _ = make(wl, "fp64", w_equation=nh.W_TRANSPORT)
    tape = torch.empty(sim.tape_bytes(), dtype=torch.uint8, device="cuda")
    with pytest.raises(nh.NHError):
        sim.step_taped(tape)
    sim.close()
