"""nh_gauges: eta at chosen cells gathered on the device (the gauge time series of the
paper's experiments), equal to the same cells of the state nh_get_state returns."""
import ctypes as C

import numpy as np
import pytest
import torch

from paper_1706_04551_b300 import inputs, nh

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_gauges_equal_state_cells(precision):
    wl = inputs.island_2d(n=96, L=4.8, center=(3.0, None), x0=1.0)
    td = torch.float32 if precision == "fp32" else torch.float64
    sim = nh.Sim(wl.H, wl.dx, bc=wl.bc, precision=precision, manning_n=0.015, breaking=1)
    sim.set_state(wl.eta.astype(sim.dtype), wl.q1.astype(sim.dtype), wl.q2.astype(sim.dtype))
    rng = np.random.default_rng(0)
    cells = rng.integers(0, wl.nx * wl.ny, 37)
    idx = torch.tensor(cells, dtype=torch.int32, device="cuda")
    series = torch.empty((5, len(cells)), dtype=td, device="cuda")
    for k in range(5):
        sim.step()
        sim.gauges(idx, series[k])
        eta = sim.get_state()["eta"].reshape(-1)
        assert np.array_equal(series[k].cpu().numpy(), eta[cells])
    sim.close()


def test_gauges_reject_bad_arguments():
    wl = inputs.shoals_2d(n=16)
    sim = nh.Sim(wl.H, wl.dx)
    L = nh.load()
    assert L.nh_gauges(sim._h, None, 3, None) == nh.EINVAL
    assert L.nh_gauges(sim._h, None, -1, None) == nh.EINVAL
    assert L.nh_gauges(sim._h, None, 0, None) == nh.OK
    sim.close()
