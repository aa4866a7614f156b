"""FP64 CPU oracle for the non-hydrostatic shallow-water step (arXiv:1706.04551).

TEST INFRASTRUCTURE ONLY.  This package wraps ``nh_oracle.c`` (plain C, FP64) through
ctypes.  Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s cpu_baseline and
``--impl reference`` legs may import it; the CUDA library never does, and the two share
no code.  Each wrapper cites the section / equation of the paper its C function follows;
the C file lists the readings taken where the paper is silent or garbled.

Parity status: every function is pinned by ``tests/test_oracle_*.py``; the breaking terms
(Sec. 3, Eq. 12) by closed forms on linear fields and by invariants; Manning friction by the
decay of a uniform flow (first-order convergence to its ODE) and the Eq. (23) rate by closed
forms on uniform states (``tests/test_oracle_friction_rate.py``).  ``cfg(dry_zero=False)``
runs the wet/dry fronts as Sec. 4.5 states them (no truncation); ``dry_zero=True`` sets q = 0 in dry cells after
each stage, and is the default of ``cfg`` (``tests/test_oracle_wetdry.py`` records why).  The 2D loops run under OpenMP
(``set_threads``) with results bitwise independent of the thread count.  ``cfg(w_transport=True)`` selects the
energy-consistent w equation of Sec. 2 (pinned by donor-cell upwind on uniform flow and
by invariants); ``relax_1d`` / ``relax_2d`` and ``cfg(relax=...)`` the relaxation zones of
Sec. 4.4 (pinned by their end values, special distances and wave absorption / generation).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "nh_oracle.c")
_HDR = os.path.join(_HERE, "nh_oracle.h")
_LIB = os.path.join(_HERE, "liboracle.so")

WALL, OUTFLOW, PERIODIC = 0, 1, 2


class Cfg(C.Structure):
    """Mirror of ``or_cfg`` in nh_oracle.h."""

    _fields_ = [
        ("nx", C.c_int), ("ny", C.c_int),
        ("dx", C.c_double), ("dy", C.c_double),
        ("bc", C.c_int * 4),
        ("g", C.c_double), ("cfl", C.c_double),
        ("delta", C.c_double), ("hdry", C.c_double),
        ("manning", C.c_double), ("B1", C.c_double), ("B2", C.c_double),
        ("breaking", C.c_int), ("nonhydro", C.c_int),
        ("tol", C.c_double), ("max_iter", C.c_int),
        ("w_transport", C.c_int),
        ("relax", C.c_double * 4),
        ("dry_zero", C.c_int),
    ]


class Stats(C.Structure):
    _fields_ = [("iters", C.c_int * 2), ("resid", C.c_double * 2), ("clamped", C.c_int)]


def build(force: bool = False) -> str:
    """Compile nh_oracle.c into liboracle.so (gcc -O2 -fopenmp, FP64, no fast-math, no
    contraction).  OpenMP runs the 2D loops over disjoint entries in parallel; sums stay
    serial, so results do not depend on the thread count."""
    newest = max(os.path.getmtime(_SRC), os.path.getmtime(_HDR))
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < newest:
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call([
            "gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fno-fast-math",
            "-ffp-contract=off", "-fopenmp", "-o", tmp, _SRC, "-lm",
        ])
        os.replace(tmp, _LIB)
    return _LIB


_lib = None


def lib():
    global _lib
    if _lib is None:
        L = C.CDLL(build())
        dp = C.POINTER(C.c_double)
        cp = C.POINTER(Cfg)
        L.or_set_threads.restype = C.c_int
        L.or_set_threads.argtypes = [C.c_int]
        L.or1d_cfl_dt.restype = C.c_double
        L.or1d_cfl_dt.argtypes = [cp, dp, dp, dp]
        L.or1d_step.argtypes = [cp, dp, dp, dp, dp, dp, C.c_double, C.POINTER(Stats)]
        L.or1d_hyperbolic.argtypes = [cp, dp, dp, dp, C.c_double, dp, dp]
        L.or1d_nh_matrix.argtypes = [cp, dp, dp, dp, dp, C.c_double, dp, dp, dp, dp]
        L.or1d_affine_apply.argtypes = [cp, dp, dp, dp, C.c_double, dp]
        L.or1d_nh_solve.argtypes = [cp, dp, dp, dp, dp, C.c_double, dp]
        L.or1d_thomas.argtypes = [C.c_int, dp, dp, dp, dp, dp]
        L.or1d_run.restype = C.c_longlong
        L.or1d_run.argtypes = [cp, dp, dp, dp, dp, dp, C.c_double, C.c_longlong, C.c_double, dp]
        L.or2d_cfl_dt.restype = C.c_double
        L.or2d_cfl_dt.argtypes = [cp, dp, dp, dp, dp]
        L.or2d_step.argtypes = [cp, dp, dp, dp, dp, dp, dp, C.c_double, C.POINTER(Stats)]
        L.or2d_stage.argtypes = [cp, dp, dp, dp, dp, dp, dp, C.c_double, dp, dp, dp, dp,
                                 C.POINTER(C.c_int), dp]
        L.or2d_hyperbolic.argtypes = [cp, dp, dp, dp, dp, C.c_double, dp, dp, dp]
        L.or2d_rhs.argtypes = [cp, dp, dp, dp, dp, dp, C.c_double, dp]
        L.or2d_apply_M.argtypes = [cp, dp, dp, dp, C.c_double, dp]
        L.or2d_solve.argtypes = [cp, dp, dp, dp, C.c_double, dp, C.POINTER(C.c_int), dp]
        L.or1d_relax.argtypes = [cp, dp, dp, dp, dp, dp, dp, dp, dp, dp]
        L.or1d_breaking.argtypes = [cp, dp, dp, dp, dp, C.c_double]
        L.or2d_breaking.argtypes = [cp, dp, dp, dp, dp, dp, C.c_double]
        L.or2d_relax.argtypes = [cp, dp, dp, dp, dp, dp, dp, dp, dp, dp, dp, dp]
        L.or2d_run.restype = C.c_longlong
        L.or2d_run.argtypes = [cp, dp, dp, dp, dp, dp, dp, C.c_double, C.c_longlong,
                               C.c_double, dp, C.POINTER(C.c_longlong)]
        _lib = L
    return _lib


def _p(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def cfg(nx: int, ny: int = 1, dx: float = 1.0, dy: float | None = None, bc=(WALL,) * 4,
        g: float = 9.81, cfl: float = 0.9, delta: float = 1e-5, hdry: float | None = None,
        manning: float = 0.0, B1: float = 0.15, B2: float = 0.5, breaking: bool = False,
        nonhydro: bool = True, tol: float = 1e-13, max_iter: int = 4000,
        w_transport: bool = False, relax=(0.0, 0.0, 0.0, 0.0),
        dry_zero: bool = True) -> Cfg:
    c = Cfg()
    c.nx, c.ny = int(nx), int(ny)
    c.dx = float(dx)
    c.dy = float(dx if dy is None else dy)
    for k in range(4):
        c.bc[k] = int(bc[k])
    c.g, c.cfl, c.delta = float(g), float(cfl), float(delta)
    c.hdry = float(delta if hdry is None else hdry)
    c.manning, c.B1, c.B2 = float(manning), float(B1), float(B2)
    c.breaking, c.nonhydro = int(bool(breaking)), int(bool(nonhydro))
    c.tol, c.max_iter = float(tol), int(max_iter)
    c.w_transport = int(bool(w_transport))
    for k in range(4):
        c.relax[k] = float(relax[k])
    c.dry_zero = int(bool(dry_zero))
    return c


def set_threads(n: int) -> int:
    """Threads of the oracle's 2D loops (n <= 0: unchanged); returns the previous count.
    Results are the same, bit for bit, for every count."""
    return int(lib().or_set_threads(int(n)))


# ----------------------------------------------------------------------------- 1D (Sec. 4)

def cfl_dt_1d(c: Cfg, H, h, q) -> float:
    """Eq. (23)."""
    H, h, q = _f64(H), _f64(h), _f64(q)
    return lib().or1d_cfl_dt(C.byref(c), _p(H), _p(h), _p(q))


def step_1d(c: Cfg, H, h, q, w, p, dt: float):
    """One TVD-RK2 step of Sec. 4.3; returns new (h, q, w, p)."""
    H = _f64(H)
    h, q, w, p = (_f64(a).copy() for a in (h, q, w, p))
    st = Stats()
    lib().or1d_step(C.byref(c), _p(H), _p(h), _p(q), _p(w), _p(p), float(dt), C.byref(st))
    return h, q, w, p


def hyperbolic_1d(c: Cfg, H, h, q, dt: float):
    """Sec. 4.1 hyperbolic step (Eqs. 18-22) with friction and the depth clamp."""
    H, h, q = _f64(H), _f64(h), _f64(q)
    ho, qo = np.empty_like(h), np.empty_like(q)
    lib().or1d_hyperbolic(C.byref(c), _p(H), _p(h), _p(q), float(dt), _p(ho), _p(qo))
    return ho, qo


def nh_matrix_1d(c: Cfg, H, h, q, w, dt: float):
    """App. B, Eq. (43) coefficients (a, b, c) and -(8 dx^2/dt) B(q*, w*) (sign reading)."""
    H, h, q, w = _f64(H), _f64(h), _f64(q), _f64(w)
    n = c.nx if c.bc[0] == PERIODIC else c.nx + 1
    a, b, cc, r = (np.zeros(n) for _ in range(4))
    lib().or1d_nh_matrix(C.byref(c), _p(H), _p(h), _p(q), _p(w), float(dt), _p(a), _p(b),
                         _p(cc), _p(r))
    return a, b, cc, r


def affine_apply_1d(c: Cfg, H, h, p, dt: float):
    """Generic map p -> (8 dx^2/dt) B(dt T(p), dt p/h), Eqs. (24)-(28)."""
    H, h, p = _f64(H), _f64(h), _f64(p)
    out = np.zeros_like(p)
    lib().or1d_affine_apply(C.byref(c), _p(H), _p(h), _p(p), float(dt), _p(out))
    return out


def nh_solve_1d(c: Cfg, H, h, q, w, dt: float):
    """Eq. (43) assembled and solved by the Thomas algorithm (cyclic when periodic)."""
    H, h, q, w = _f64(H), _f64(h), _f64(q), _f64(w)
    p = np.zeros(c.nx + 1)
    lib().or1d_nh_solve(C.byref(c), _p(H), _p(h), _p(q), _p(w), float(dt), _p(p))
    return p


def thomas(a, b, cc, d):
    a, b, cc, d = _f64(a), _f64(b), _f64(cc), _f64(d)
    x = np.zeros_like(d)
    lib().or1d_thomas(len(d), _p(a), _p(b), _p(cc), _p(d), _p(x))
    return x


def run_1d(c: Cfg, H, h, q, w, p, t_end: float = 0.0, max_steps: int = 1 << 40,
           fixed_dt: float = 0.0):
    """Steps with dt = Eq. (23) (or fixed_dt) until t_end, the last step clamped to t_end."""
    H = _f64(H)
    h, q, w, p = (_f64(a).copy() for a in (h, q, w, p))
    t = C.c_double(0.0)
    s = lib().or1d_run(C.byref(c), _p(H), _p(h), _p(q), _p(w), _p(p), float(t_end),
                       int(max_steps), float(fixed_dt), C.byref(t))
    return h, q, w, p, t.value, s


# ----------------------------------------------------------------------------- 2D (Sec. 5)

def cfl_dt_2d(c: Cfg, H, h, q1, q2) -> float:
    H, h, q1, q2 = _f64(H), _f64(h), _f64(q1), _f64(q2)
    return lib().or2d_cfl_dt(C.byref(c), _p(H), _p(h), _p(q1), _p(q2))


def step_2d(c: Cfg, H, h, q1, q2, w, p, dt: float):
    """One TVD-RK2 step of App. A; returns (h, q1, q2, w, p, stats)."""
    H = _f64(H)
    h, q1, q2, w, p = (_f64(a).copy() for a in (h, q1, q2, w, p))
    st = Stats()
    lib().or2d_step(C.byref(c), _p(H), _p(h), _p(q1), _p(q2), _p(w), _p(p), float(dt),
                    C.byref(st))
    return h, q1, q2, w, p, st


def stage_2d(c: Cfg, H, h, q1, q2, w, p, dt: float):
    """First Runge-Kutta stage (hyperbolic, breaking, solve, correction) of App. A."""
    H, h, q1, q2, w = (_f64(a) for a in (H, h, q1, q2, w))
    p = _f64(p).copy()
    ho, ao, bo, wo = np.empty_like(h), np.empty_like(h), np.empty_like(h), np.empty_like(w)
    it = C.c_int(0)
    rs = C.c_double(0.0)
    lib().or2d_stage(C.byref(c), _p(H), _p(h), _p(q1), _p(q2), _p(w), _p(p), float(dt),
                     _p(ho), _p(ao), _p(bo), _p(wo), C.byref(it), C.byref(rs))
    return ho, ao, bo, wo, p, it.value, rs.value


def hyperbolic_2d(c: Cfg, H, h, q1, q2, dt: float):
    H, h, q1, q2 = (_f64(a) for a in (H, h, q1, q2))
    ho, ao, bo = np.empty_like(h), np.empty_like(h), np.empty_like(h)
    lib().or2d_hyperbolic(C.byref(c), _p(H), _p(h), _p(q1), _p(q2), float(dt), _p(ho),
                          _p(ao), _p(bo))
    return ho, ao, bo


def rhs_2d(c: Cfg, H, h, q1, q2, w, dt: float):
    H, h, q1, q2, w = (_f64(a) for a in (H, h, q1, q2, w))
    r = np.zeros((c.ny + 1, c.nx + 1))
    lib().or2d_rhs(C.byref(c), _p(H), _p(h), _p(q1), _p(q2), _p(w), float(dt), _p(r))
    return r


def apply_M_2d(c: Cfg, H, h, p, dt: float):
    H, h, p = _f64(H), _f64(h), _f64(p)
    out = np.zeros_like(p)
    lib().or2d_apply_M(C.byref(c), _p(H), _p(h), _p(p), float(dt), _p(out))
    return out


def solve_2d(c: Cfg, H, h, rhs, dt: float, p0=None):
    H, h, rhs = _f64(H), _f64(h), _f64(rhs)
    p = np.zeros_like(rhs) if p0 is None else _f64(p0).copy()
    it = C.c_int(0)
    rs = C.c_double(0.0)
    st = lib().or2d_solve(C.byref(c), _p(H), _p(h), _p(rhs), float(dt), _p(p), C.byref(it),
                          C.byref(rs))
    return p, it.value, rs.value, st


def run_2d(c: Cfg, H, h, q1, q2, w, p, t_end: float = 0.0, max_steps: int = 1 << 40,
           fixed_dt: float = 0.0):
    H = _f64(H)
    h, q1, q2, w, p = (_f64(a).copy() for a in (h, q1, q2, w, p))
    t = C.c_double(0.0)
    it = C.c_longlong(0)
    s = lib().or2d_run(C.byref(c), _p(H), _p(h), _p(q1), _p(q2), _p(w), _p(p), float(t_end),
                       int(max_steps), float(fixed_dt), C.byref(t), C.byref(it))
    return h, q1, q2, w, p, t.value, s, it.value


def _opt(a):
    return None if a is None else _p(a)


def relax_1d(c: Cfg, H, h, q, w, p, eta_t=None, q_t=None, w_t=None, p_t=None):
    """Sec. 4.4 relaxation zones (widths c.relax) toward the target; None = lake at rest."""
    H = _f64(H)
    h, q, w, p = (_f64(a).copy() for a in (h, q, w, p))
    tg = [None if a is None else _f64(a) for a in (eta_t, q_t, w_t, p_t)]
    lib().or1d_relax(C.byref(c), _p(H), _p(h), _p(q), _p(w), _p(p), *[_opt(a) for a in tg])
    return h, q, w, p


def relax_2d(c: Cfg, H, h, q1, q2, w, p, eta_t=None, q1_t=None, q2_t=None, w_t=None,
             p_t=None):
    """Sec. 4.4 relaxation zones on the four sides (m = m_x m_y) toward the target."""
    H = _f64(H)
    h, q1, q2, w, p = (_f64(a).copy() for a in (h, q1, q2, w, p))
    tg = [None if a is None else _f64(a) for a in (eta_t, q1_t, q2_t, w_t, p_t)]
    lib().or2d_relax(C.byref(c), _p(H), _p(h), _p(q1), _p(q2), _p(w), _p(p),
                     *[_opt(a) for a in tg])
    return h, q1, q2, w, p


def breaking_1d(c: Cfg, H, h, q, w, dt: float):
    """Sec. 3 / Eq. (12) breaking terms alone: returns (q, w) after them."""
    H, h = _f64(H), _f64(h)
    q, w = _f64(q).copy(), _f64(w).copy()
    lib().or1d_breaking(C.byref(c), _p(H), _p(h), _p(q), _p(w), float(dt))
    return q, w


def breaking_2d(c: Cfg, H, h, q1, q2, w, dt: float):
    """2D breaking terms (q_x -> div q, u_x -> div u): returns (q1, q2, w) after them."""
    H, h = _f64(H), _f64(h)
    q1, q2, w = _f64(q1).copy(), _f64(q2).copy(), _f64(w).copy()
    lib().or2d_breaking(C.byref(c), _p(H), _p(h), _p(q1), _p(q2), _p(w), float(dt))
    return q1, q2, w
