"""Periodic 1D channels (Sec. 4.4: cyclic tridiagonal pressure system) on the CUDA path:
against the FP64 oracle, and the Table 1 convergence procedure of Sec. 7.1 run on the GPU
(orders against the printed ones, tests/golden/table1_convergence.json)."""
import json
import os

import numpy as np
import pytest

import oracle as O
from paper_1706_04551_b300 import nh

pytestmark = pytest.mark.gpu
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
L, A, G = 50.0, 0.1, 1.0   # Sec. 7.1: 50 m periodic channel, g = 1, H = 1, A = 0.1


def rel(x, ref):
    s = np.abs(ref).max()
    return np.abs(np.asarray(x, np.float64) - ref).max() / (s if s > 0 else 1.0)


def solitary(n):
    dx = L / n
    x = (np.arange(n) + 0.5) * dx
    k = np.sqrt(3 * A / 4)
    eta = A / np.cosh(k * (x - 25.0)) ** 2
    H = np.ones(n)
    q = (H + eta) * np.sqrt(G) * eta          # u of Eq. (33) with H = 1
    return dx, H, eta, q


def gpu_run(n, t_end, precision="fp64"):
    dx, H, eta, q = solitary(n)
    sim = nh.Sim(H, dx, dim=1, bc=(nh.PERIODIC, nh.PERIODIC, 0, 0), precision=precision,
                 g=G, cfl=0.4)
    dt = np.float64 if precision == "fp64" else np.float32
    sim.set_state(eta.astype(dt)[None, :], q.astype(dt)[None, :])
    steps = sim.run(t_end=t_end) if t_end > 0 else 0   # (t_end <= 0 is not "no steps")
    g = sim.get_state()
    sim.close()
    return g, steps, H


def test_periodic_channel_matches_oracle_fp64():
    n = 400
    g, steps, H = gpu_run(n, 3.0)
    dx, H, eta, q = solitary(n)
    c = O.cfg(n, dx=dx, g=G, cfl=0.4, bc=(O.PERIODIC, O.PERIODIC, 0, 0))
    h, qo, w, p, t, s = O.run_1d(c, H, H + eta, q, np.zeros(n + 1), np.zeros(n + 1), t_end=3.0)
    assert steps == s and abs(g["t"] - t) < 1e-12
    assert rel(g["eta"][0] + H, h) < 1e-10
    assert rel(g["q1"][0], qo) < 1e-10
    assert rel(g["p"][0], p) < 1e-10
    assert g["p"][0, n] == g["p"][0, 0] and g["w"][0, n] == g["w"][0, 0]


def test_periodic_channel_conserves_mass_fp32():
    g0, _, H = gpu_run(256, 0.0, "fp32")
    g, steps, H = gpu_run(256, 5.0, "fp32")
    m0 = float(np.sum(g0["eta"][0].astype(np.float64) + H))
    m = float(np.sum(g["eta"][0].astype(np.float64) + H))
    assert steps > 10 and abs(m - m0) <= 1e-6 * m0


def test_table1_orders_on_the_gpu_path():
    """Sec. 7.1 / Table 1 procedure on the CUDA path (FP64): L1 errors of h and q at t = 10 s
    against a 6400-cell run, orders between successive meshes within 0.2 of the printed."""
    ref = json.load(open(os.path.join(GOLDEN, "table1_convergence.json")))
    nref = 6400
    gr, _, _ = gpu_run(nref, 10.0)
    hr = gr["eta"][0] + 1.0
    qr = gr["q1"][0]
    errs = []
    for n in (100, 200, 400, 800):
        g, _, H = gpu_run(n, 10.0)
        f = nref // n
        errs.append((np.abs(g["eta"][0] + H - hr.reshape(n, f).mean(1)).sum() * L / n,
                     np.abs(g["q1"][0] - qr.reshape(n, f).mean(1)).sum() * L / n))
    for i in range(1, 4):
        oh = np.log2(errs[i - 1][0] / errs[i][0])
        oq = np.log2(errs[i - 1][1] / errs[i][1])
        assert abs(oh - ref["order_h"][i]) < 0.2, (i, oh)
        assert abs(oq - ref["order_q"][i]) < 0.2, (i, oq)
