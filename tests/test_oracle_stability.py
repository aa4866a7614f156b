"""How the discrete step treats small perturbations, at and below the paper's Courant number.

The paper runs its tests at CFL 0.9 (Eq. 23, in 2D the sum over both directions).  There the
MUSCL-minmod / SSP-RK2 step amplifies a perturbation of rounding size by orders of magnitude
within tens of steps, in the hydrostatic and the non-hydrostatic step alike, until the limiter
caps it (near 1e-3 of the wave amplitude); at CFL 0.7 and below it does not grow.  The
nonlinear scheme stays stable either way.  This fixes what any two implementations of the
step (or one run in FP32 and one in FP64) can agree to over long horizons at CFL 0.9, and why
an exact derivative of the step grows there.
"""
import numpy as np
import pytest

import oracle as O
from paper_1706_04551_b300 import inputs

pytestmark = pytest.mark.filterwarnings("ignore::DeprecationWarning")


def growth(cfl, nonhydro=True, steps=40, eps=1e-12):
    wl = inputs.shoals_2d(n=128, L=102.4)
    g = np.random.default_rng(1).standard_normal(wl.h.shape)
    c = O.cfg(wl.nx, wl.ny, dx=wl.dx, bc=wl.bc, tol=1e-13, cfl=cfl, nonhydro=nonhydro)
    z = np.zeros((wl.ny + 1, wl.nx + 1))
    a = O.run_2d(c, wl.H, wl.h, wl.q1, wl.q2, z, z, max_steps=steps)
    b = O.run_2d(c, wl.H, wl.h * (1 + eps * g), wl.q1, wl.q2, z, z, max_steps=steps)
    return np.abs(a[0] - b[0]).max() / (eps * np.abs(wl.h).max())


@pytest.mark.parametrize("nonhydro", [True, False])
def test_cfl09_amplifies_rounding_size_perturbations(nonhydro):
    assert growth(0.9, nonhydro) > 1e3


@pytest.mark.parametrize("cfl", [0.5, 0.7])
def test_below_cfl07_perturbations_do_not_grow(cfl):
    assert growth(cfl) < 10.0
