"""Generating / absorbing relaxation zones (Sec. 4.4, nh_params.relax_width and
nh_set_relax_target) on the CUDA path against the FP64 oracle (`relax_2d`, `relax_1d`,
`run_*` with `cfg(relax=...)`), and the absorption of an outgoing wave at a size the
oracle's run takes minutes for.  Bars as the other parity tests: FP64 1e-10, FP32 1e-4."""
import numpy as np
import pytest

import oracle as O
from paper_1706_04551_b300 import nh
from test_gpu_parity import developed, island, make, rel, rel_q, shoals

pytestmark = pytest.mark.gpu
G = 9.81


def _cfg_relax(c, widths):
    for k in range(4):
        c.relax[k] = widths[k]
    return c


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_absorbing_zones_2d_match_oracle(precision):
    """Island basin (wet / dry, breaking, friction), absorbing zones of 3, 4, 2, 2 cells."""
    wl = island(64)
    widths = (1.0, 1.5, 0.5, 0.8)                 # dx = 0.4
    sim, c = make(wl, precision, relax_width=widths)
    _cfg_relax(c, widths)
    eta, q1, q2 = developed(wl, seed=5)
    dt = sim.dtype
    sim.set_state(eta.astype(dt), q1.astype(dt), q2.astype(dt))
    steps = 12
    for _ in range(steps):
        sim.step()
    g = sim.get_state()
    sim.close()
    zn = np.zeros((wl.ny + 1, wl.nx + 1))
    h, a, b, w, p, t, s, it = O.run_2d(c, wl.H, np.maximum(eta + wl.H, 0), q1, q2, zn, zn,
                                       max_steps=steps)
    if precision == "fp64":
        assert rel(g["eta"] + wl.H, h) < 1e-10
        assert rel_q(g["q1"], g["q2"], a, b) < 1e-10
        assert rel(g["w"], w) < 1e-10 and rel(g["p"], p) < 1e-10
        assert abs(g["t"] - t) < 1e-12 * t
    else:
        assert rel(g["eta"], h - wl.H) < 1e-4


def test_generating_target_2d_matches_oracle_fp64():
    """Walled shoals basin, zones on all four sides driven toward a smooth target set
    through nh_set_relax_target."""
    wl = shoals(64)
    widths = (0.5, 0.4, 0.3, 0.6)
    sim, c = make(wl, "fp64", relax_width=widths)
    _cfg_relax(c, widths)
    eta, q1, q2 = developed(wl, seed=6)
    ny, nx = wl.H.shape
    y, x = np.mgrid[0:ny, 0:nx] / nx
    yn, xn = np.mgrid[0:ny + 1, 0:nx + 1] / nx
    tg = (0.02 * np.sin(5 * x) * np.cos(3 * y), 0.01 * np.cos(4 * x), 0.01 * np.sin(2 * y),
          0.003 * np.sin(3 * xn + yn), 0.02 * np.cos(xn - 2 * yn))
    sim.set_state(eta, q1, q2)
    sim.set_relax_target(*tg)
    steps = 8
    for _ in range(steps):
        sim.step()
    g = sim.get_state()
    sim.close()
    h, a, b = np.maximum(eta + wl.H, 0), q1, q2
    w = np.zeros((ny + 1, nx + 1))
    p = np.zeros_like(w)
    for _ in range(steps):
        dt = O.cfl_dt_2d(c, wl.H, h, a, b)
        h, a, b, w, p, _ = O.step_2d(c, wl.H, h, a, b, w, p, dt)
        h, a, b, w, p = O.relax_2d(c, wl.H, h, a, b, w, p, *tg)
    assert rel(g["eta"] + wl.H, h) < 1e-10
    assert rel_q(g["q1"], g["q2"], a, b) < 1e-10
    assert rel(g["w"], w) < 1e-10 and rel(g["p"], p) < 1e-10


def _solitary_channel(n, Lc, A=0.1, h0=1.0, x0=40.0):
    dx = Lc / n
    x = (np.arange(n) + 0.5) * dx
    k = np.sqrt(3 * A / (4 * h0 ** 3))
    c0 = np.sqrt(G * (h0 + A))
    eta = A / np.cosh(k * (x - x0)) ** 2
    H = np.full(n, h0)
    q = (H + eta) * c0 * eta / (h0 + eta)
    return dx, H, eta, q, 6.0 / k, c0


def test_absorbing_zone_1d_matches_oracle_fp64():
    n, Lc = 600, 120.0
    dx, H, eta, q, lam, c0 = _solitary_channel(n, Lc)
    widths = (0.0, 1.5 * lam, 0.0, 0.0)
    sim = nh.Sim(H, dx, dim=1, bc=(0, 0, 0, 0), precision="fp64", cfl=0.9,
                 relax_width=widths)
    sim.set_state(eta[None, :], q[None, :])
    steps = 150
    for _ in range(steps):
        sim.step()
    g = sim.get_state()
    sim.close()
    c = O.cfg(n, dx=dx, cfl=0.9, relax=widths)
    h, qo, w, p, t, s = O.run_1d(c, H, H + eta, q, np.zeros(n + 1), np.zeros(n + 1),
                                 max_steps=steps)
    assert rel(g["eta"][0] + H, h) < 1e-10 and rel(g["q1"][0], qo) < 1e-10
    assert rel(g["w"][0], w) < 1e-10 and rel(g["p"][0], p) < 1e-10


def test_absorbing_zone_takes_the_wave_at_size_fp32():
    """512 channels of 2048 cells (1D rows): the wave leaves < 0.5 % of its energy in
    front of a walled end with a zone, > 80 % without one."""
    n, Lc = 2048, 240.0
    dx, H, eta, q, lam, c0 = _solitary_channel(n, Lc, x0=80.0)
    rows = 512
    out = {}
    for name, widths in (("wall", (0, 0, 0, 0)), ("zone", (0, 1.5 * lam, 0, 0))):
        sim = nh.Sim(np.tile(H, (rows, 1)), dx, dim=1, bc=(0, 0, 0, 0), precision="fp32",
                     cfl=0.9, relax_width=widths, tol=1e-6)
        sim.set_state(np.tile(eta, (rows, 1)).astype(np.float32),
                      np.tile(q, (rows, 1)).astype(np.float32))
        sim.run(t_end=(Lc - 80.0 + 30.0) / c0)
        g = sim.get_state()
        sim.close()
        e = g["eta"].astype(np.float64)
        qq = g["q1"].astype(np.float64)
        E = np.sum(0.5 * G * e ** 2 + 0.5 * qq ** 2 / (e + H), axis=1) * dx
        E0 = np.sum(0.5 * G * eta ** 2 + 0.5 * q ** 2 / (H + eta)) * dx
        out[name] = (E / E0).max()
    assert out["wall"] > 0.8 and out["zone"] < 0.005


def test_relaxation_is_rejected_where_it_is_not_built():
    wl = shoals(32)
    with pytest.raises(nh.NHError):
        nh.Batch([wl.H, wl.H], dx=wl.dx, precision="fp32", relax_width=(0.2, 0, 0, 0))
    import torch
    sim, _ = make(wl, "fp64", relax_width=(0.2, 0, 0, 0))
    tape = torch.empty(sim.tape_bytes(), dtype=torch.uint8, device="cuda")
    with pytest.raises(nh.NHError):
        sim.step_taped(tape)
    sim.close()
    sim, _ = make(wl, "fp64")
    with pytest.raises(nh.NHError):
        sim.set_relax_target(eta=np.zeros_like(wl.H))
    sim.close()
