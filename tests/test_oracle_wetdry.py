"""Wet/dry fronts in the second step (Sec. 4.5) and the oracle's thread-count invariance.

Sec. 4.5 states that the non-hydrostatic step needs no special treatment at wet/dry fronts
and no truncation (``dry_zero=False``); ``dry_zero=True``, the default, sets q = 0 in dry
cells after each stage (App. B A.2 takes q = w = 0 where h vanishes).  These tests record
what the literal form does in dry cells: a small discharge, no worse conditioning under
perturbations of the wet depths -- but results that hang on depths of 1e-20 m and below,
which a state held as eta = h - H (as the FP32 form must hold it) cannot represent.
"""
import numpy as np
import pytest

import oracle as O
from paper_1706_04551_b300 import inputs

pytestmark = pytest.mark.filterwarnings("ignore::DeprecationWarning")

HDRY = 1e-5


def island64():
    return inputs.island_2d(n=64, L=25.6, center=(12.8, None), x0=4.0)


def run(wl, steps, dry_zero, h0=None):
    c = O.cfg(wl.nx, wl.ny, dx=wl.dx, bc=wl.bc, manning=0.015, breaking=True, tol=1e-13,
              dry_zero=dry_zero)
    zn = np.zeros((wl.ny + 1, wl.nx + 1))
    return O.run_2d(c, wl.H, wl.h if h0 is None else h0, wl.q1, wl.q2, zn, zn,
                    max_steps=steps)


def fully_dry_nodes(h):
    hp = np.pad(h, 1, mode="edge")
    return ((hp[:-1, :-1] <= HDRY) & (hp[1:, :-1] <= HDRY) & (hp[:-1, 1:] <= HDRY)
            & (hp[1:, 1:] <= HDRY))


def test_literal_second_step_leaves_dry_cells_a_small_discharge():
    """After the wave has run up the island (60 steps, t = 5.4 s), the literal form gives dry
    cells a discharge: the correction's p (2 eta - h)_x term does not vanish with h.  It
    stays below 1e-3 of the largest wet discharge (measured: 1.6e-5 m^2/s against 7.0e-2).
    With dry_zero the dry cells hold exactly none.  Fully dry nodes carry a pressure in both
    forms, since their rows couple to wet neighbours (measured: 2.7e-5 and 6.9e-6, against a
    largest |p| of 1.3e-2)."""
    wl = island64()
    out = {}
    for dz in (False, True):
        h, a, b, w, p, t, s, it = run(wl, 60, dz)
        dry = h <= HDRY
        q = np.hypot(a, b)
        nd = fully_dry_nodes(h)
        assert dry.sum() > 50 and nd.sum() > 30
        out[dz] = (q[dry].max(), q[~dry].max(), np.abs(p[nd]).max(), np.abs(p).max())
    qd, qw, pd, pm = out[False]
    assert 0.0 < qd < 1e-3 * qw
    assert 0.0 < pd < 1e-2 * pm
    qd, qw, pd, pm = out[True]
    assert qd == 0.0
    assert 0.0 < pd < 1e-2 * pm


@pytest.mark.parametrize("steps", [15, 40])
def test_both_forms_equally_sensitive_to_rounding(steps):
    """A one-ulp perturbation of the wet depths moves the literal form no more than the
    truncated one (measured equal to two digits at 15, 30 and 40 steps): the dry-cell
    discharges do not make the literal form worse conditioned."""
    wl = island64()
    rng = np.random.default_rng(0)
    hp = np.where(wl.h > 0, wl.h * (1 + 2.2e-16 * rng.choice([-1, 1], wl.h.shape)), 0.0)
    spread = {}
    for dz in (False, True):
        ref = run(wl, steps, dz)
        per = run(wl, steps, dz, h0=hp)
        spread[dz] = np.abs(per[0] - ref[0]).max() / np.abs(ref[0]).max()
    assert spread[True] > 0.0
    assert spread[False] <= 2.0 * spread[True], spread


def test_literal_form_depends_on_depths_below_1e20():
    """After 4 literal steps on an uneven ensemble domain with dry patches, the flux
    arithmetic has left depths down to ~1e-128 m in a few dry cells.  Setting just those
    depths (below 1e-20 m) to 0 -- what a state held as eta = h - H gives, since
    (h - H) + H rounds them away -- moves the next step's p by ~1e-5 and its discharges by
    ~1e-6 (measured 8.9e-6 and 2.8e-6): whether the depth clamp zeroes a dry cell's
    discharge turns on those depths.  With q = 0 in dry cells no such depths arise and the
    step is unchanged."""
    w = inputs.ensemble_member(1, sides=(40,))
    rel = lambda x, y: np.abs(x - y).max() / np.abs(y).max()
    out = {}
    for dz in (False, True):
        c = O.cfg(w.nx, w.ny, dx=w.dx, dy=w.dy, bc=w.bc, tol=1e-14, dry_zero=dz)
        zn = np.zeros((w.ny + 1, w.nx + 1))
        h, a, b, wv, p, t, s, it = O.run_2d(c, w.H, np.maximum(w.eta + w.H, 0), w.q1, w.q2,
                                            zn, zn, max_steps=4)
        tiny = (h > 0) & (h < 1e-20)
        dt = O.cfl_dt_2d(c, w.H, h, a, b)
        A = O.step_2d(c, w.H, h, a, b, wv, p, dt)
        B = O.step_2d(c, w.H, np.where(tiny, 0.0, h), a, b, wv, p, dt)
        out[dz] = (tiny.sum(), rel(B[4], A[4]), max(rel(B[1], A[1]), rel(B[2], A[2])))
    n, dp, dq = out[False]
    assert n > 0 and dp > 1e-7 and dq > 1e-8, out[False]
    n, dp, dq = out[True]
    assert n == 0 and dp == 0.0 and dq == 0.0, out[True]


def test_threads_do_not_change_results_bitwise():
    """The OpenMP loops write disjoint entries and every sum is serial: 1 and 4 threads give
    the same bits (full steps on the wet/dry island with breaking and friction)."""
    wl = inputs.island_2d(n=48, L=19.2, center=(9.6, None), x0=3.0)
    prev = O.set_threads(1)
    try:
        a = run(wl, 4, False)
        O.set_threads(4)
        b = run(wl, 4, False)
    finally:
        O.set_threads(prev)
    for x, y in zip(a[:5], b[:5]):
        assert np.array_equal(x, y)
    assert a[7] == b[7]
