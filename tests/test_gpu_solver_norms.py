"""Residual norms of the pressure solve stay meaningful at any wave amplitude.

The stopping test of the scheduled-relaxation Jacobi (Sec. 5: relative residual, or
criterion (32)) is scale-invariant, so a wave of amplitude 1e-22 m must take the same sweeps
as a larger one.  Squares of residuals that small lie below the FP32 range (1e-38): a norm
squared or summed in FP32 reads 0 there and stops the solve at its first pass, with p
still near its warm start.  The passes therefore square exactly rescaled residuals (by a
power of two set from ||D^-1 b||) and sum above the thread in FP64.

The oracle holds the state as h = H + eta, in which a wave below half an ulp of H (1e-17 m
here) does not exist, so these checks use what the mathematics fixes instead: with h = H
to the last bit the discrete step is linear in the amplitude, so p / A must not depend on A.
"""
import numpy as np
import pytest

from paper_1706_04551_b300 import inputs, nh

pytestmark = pytest.mark.gpu


def _p_per_amplitude(amp, precision, tol, dt, n=256):
    # dx = 0.1 m under 0.5 m of water: the solve takes tens of sweeps (many passes)
    wl = inputs.shoals_2d(n=n, L=25.6)
    pat = wl.eta / np.abs(wl.eta).max()
    eta = (amp * pat).astype(np.float64 if precision == "fp64" else np.float32)
    z = np.zeros_like(eta)
    sim = nh.Sim(wl.H, wl.dx, bc=wl.bc, precision=precision, tol=tol, solver=nh.CHEBYSHEV)
    sim.set_state(eta, z, z)
    sim.step(dt)
    st = sim.stats()
    p = sim.get_state()["p"].astype(np.float64) / amp
    sim.close()
    return p, st["last_iters"]


@pytest.mark.parametrize("precision,tiny,ref,tol,bar", [
    ("fp64", 1e-22, 1e-9, 1e-10, 1e-7),
    ("fp64", 1e-26, 1e-9, 1e-10, 1e-7),
    ("fp32", 1e-17, 1e-5, 1e-5, 2e-3),
])
def test_tiny_wave_pressure_scales_with_the_amplitude(precision, tiny, ref, tol, bar):
    """p / A at A = `tiny` equals p / A at a larger A to within the step's nonlinearity
    O(A / H) and the solver tolerance, after the same sweeps; a solve stopped by an
    underflowed norm would end after its first pass."""
    p_ref, it_ref = _p_per_amplitude(ref, precision, tol, 0.01)
    p_tiny, it_tiny = _p_per_amplitude(tiny, precision, tol, 0.01)
    err = np.abs(p_tiny - p_ref).max() / np.abs(p_ref).max()
    assert err < bar, (err, it_ref, it_tiny)
    assert min(it_tiny) >= 24 and min(it_ref) >= 24, (it_ref, it_tiny)
    assert max(abs(a - b) for a, b in zip(it_tiny, it_ref)) <= 8, (it_ref, it_tiny)


def test_sweeps_do_not_depend_on_the_wave_amplitude():
    """At 1e-22 and 1e-26 m the depth h = H + eta is the same FP64 number in both runs
    (eta is below half an ulp of H), so the systems differ only by the scale of the
    right-hand side and the relative stopping test takes the same sweeps."""
    a, it_a = _p_per_amplitude(1e-22, "fp64", 1e-12, 0.01)
    b, it_b = _p_per_amplitude(1e-26, "fp64", 1e-12, 0.01)
    assert it_a == it_b, (it_a, it_b)
    assert np.abs(a - b).max() <= 1e-9 * np.abs(a).max()
