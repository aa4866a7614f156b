"""Failure statuses of the C-ABI (Sec. 5's solve can stop without converging; the state can
turn non-finite; a bounded device-side wait can run out), each made on the host: a NaN in
the input, an iteration cap of one pass, and a wait on copies that were never issued (the
nh_debug_stall_copies hook).  Nothing here faults, traps or hangs the GPU: every wait in the
kernels is bounded, and the injected wait has no copy in flight.
"""
import numpy as np
import pytest

from paper_1706_04551_b300 import inputs, nh

pytestmark = pytest.mark.gpu


def shoals(n=128):
    return inputs.shoals_2d(n=n)


def sim(wl, precision, **kw):
    kw.setdefault("tol", 1e-12 if precision == "fp64" else 1e-5)
    return nh.Sim(wl.H, wl.dx, bc=wl.bc, precision=precision, **kw)


def state(wl, dtype):
    return (wl.eta.astype(dtype), wl.q1.astype(dtype), wl.q2.astype(dtype))


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("field", ["eta", "q1", "p"])
def test_nonfinite_input_is_rejected_and_a_clean_state_recovers(precision, field):
    wl = shoals(64)
    s = sim(wl, precision)
    e, a, b = state(wl, s.dtype)
    p = np.zeros(s.node_shape, s.dtype)
    bad = {"eta": e.copy(), "q1": a.copy(), "p": p.copy()}
    bad[field].flat[bad[field].size // 3] = np.nan
    with pytest.raises(nh.NHError) as ei:
        s.set_state(bad["eta"], bad["q1"], b, p=bad["p"])
    assert ei.value.code == nh.ENONFINITE
    s.set_state(e, a, b)
    s.step()
    st = s.stats()
    assert st["nonfinite"] == 0 and np.isfinite(s.get_state()["eta"]).all()
    s.close()


@pytest.mark.parametrize("solver", [nh.CHEBYSHEV, nh.BICGSTAB])
def test_iteration_cap_returns_enoconv_and_the_step_is_taken(solver):
    wl = shoals(64)
    s = sim(wl, "fp64", solver=solver, max_iter=1)
    s.set_state(*state(wl, s.dtype))
    with pytest.raises(nh.NHError) as ei:
        s.step()
    assert ei.value.code == nh.ENOCONV
    st = s.stats()
    assert st["steps"] == 1 and st["last_iters"][0] >= 1
    assert st["last_resid"][0] > 1e-12
    s.close()
    # the same state with the default cap converges
    s = sim(wl, "fp64", solver=solver)
    s.set_state(*state(wl, s.dtype))
    s.step()
    assert max(s.stats()["last_resid"]) <= 1e-12
    s.close()


@pytest.mark.parametrize("precision,form", [("fp32", 7), ("fp32", 5), ("fp64", 3), ("fp32", -1),
                                            ("fp64", -1)])
def test_bounded_wait_that_runs_out_returns_etimeout(precision, form):
    """Block 0 of a register-form pass (form -1: the cyclic form, the default) waits for a
    region whose copies were never issued:
    its wait runs out after wait_polls polls, the solve is abandoned with NH_ETIMEOUT, and a
    fresh handle on the same device then steps normally (the context is intact)."""
    wl = shoals(128)
    cyc = dict(cheb_cyclic=1) if form < 0 else {}
    s = sim(wl, precision, cheb_form=form, wait_polls=64, **cyc)
    s.set_state(*state(wl, s.dtype))
    s.debug_stall_copies(0)
    with pytest.raises(nh.NHError) as ei:
        s.step()
    assert ei.value.code == nh.ETIMEOUT, ei.value
    assert "ran out of polls" in str(ei.value)
    s.close()
    ok = sim(wl, precision, cheb_form=form, **cyc)
    ok.set_state(*state(wl, ok.dtype))
    for _ in range(2):
        ok.step()
    g = ok.get_state()
    assert np.isfinite(g["eta"]).all() and np.isfinite(g["p"]).all()
    assert ok.stats()["last_iters"][0] > 0
    ok.close()


def test_stall_hook_rejected_where_no_register_pass_runs():
    wl = shoals(64)
    s = sim(wl, "fp64", solver=nh.BICGSTAB)
    with pytest.raises(nh.NHError) as ei:
        s.debug_stall_copies(0)
    assert ei.value.code == nh.EINVAL
    s.close()
