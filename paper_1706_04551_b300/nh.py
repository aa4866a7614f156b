"""Thin ctypes binding of libnh (C-ABI in include/nh.h): argument marshalling only.

Every step of the time integration runs in the CUDA kernels of ``libnh.so``; this module
only converts arguments.  ``load()`` raises if the library is missing, so no code path
falls back to anything else.  Arrays may be numpy (host) or torch CUDA tensors (device);
torch is used for device memory and streams only.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libnh.so")

OK, EINVAL, ENOMEM, ECUDA, ENOCONV, ENONFINITE, ETIMEOUT = 0, -1, -2, -3, -4, -5, -6
WALL, OUTFLOW, PERIODIC = 0, 1, 2
BICGSTAB, CHEBYSHEV = 0, 1
FP64, FP32 = 0, 1
HOST, DEVICE = 0, 1
W_YAMAZAKI, W_TRANSPORT = 0, 1   # w equation: h w_t = p, or (hw)_t + div(hw u) = p


class Grid(C.Structure):
    _fields_ = [("dim", C.c_int), ("nx", C.c_int), ("ny", C.c_int), ("dx", C.c_double),
                ("dy", C.c_double), ("bc", C.c_int * 4)]


class Params(C.Structure):
    _fields_ = [("g", C.c_double), ("cfl", C.c_double), ("delta", C.c_double),
                ("hdry", C.c_double), ("manning_n", C.c_double), ("B1", C.c_double),
                ("B2", C.c_double), ("breaking", C.c_int), ("nonhydrostatic", C.c_int),
                ("solver", C.c_int), ("tol", C.c_double), ("max_iter", C.c_int),
                ("precision", C.c_int), ("fixed_dt", C.c_double), ("eps_dp", C.c_double),
                ("adjoint_frozen_limiter", C.c_int), ("cheb_form", C.c_int),
                ("w_equation", C.c_int), ("relax_width", C.c_double * 4),
                ("dry_zero", C.c_int), ("wait_polls", C.c_int), ("capture", C.c_int),
                ("refine_fp32", C.c_int), ("fallback_block_nodes", C.c_int),
                ("cheb_cyclic", C.c_int)]


class StatsT(C.Structure):
    _fields_ = [("t", C.c_double), ("dt", C.c_double), ("dt_next", C.c_double),
                ("steps", C.c_longlong), ("solver_iters", C.c_longlong),
                ("last_iters", C.c_int * 2), ("last_resid", C.c_double * 2),
                ("mass", C.c_double), ("nonfinite", C.c_int), ("fallbacks", C.c_int),
                ("fallback_iters", C.c_longlong), ("cheb_form", C.c_int)]


class BatchTuning(C.Structure):
    _fields_ = [("hyp", C.c_int), ("assembly", C.c_int), ("cheb", C.c_int),
                ("persistent", C.c_int), ("graph", C.c_int), ("tuned", C.c_int),
                ("ms", C.c_double * 3)]


class NHError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"libnh error {code}: {msg}")
        self.code = code


_lib = None

EXPORTS = ("nh_default_params", "nh_create", "nh_set_state", "nh_get_state", "nh_step",
           "nh_run", "nh_stats", "nh_last_error", "nh_destroy", "nh_profile_enable",
           "nh_profile_read", "nh_tridiag_batched", "nh_debug_hyperbolic", "nh_debug_system",
           "nh_create_batch", "nh_batch_set_state", "nh_batch_get_state", "nh_batch_run",
           "nh_batch_stats", "nh_batch_get_tuning", "nh_batch_set_tuning",
           "nh_batch_candidate", "nh_batch_last_error", "nh_batch_destroy",
           "nh_batch_profile_enable", "nh_batch_profile_read", "nh_tape_bytes",
           "nh_step_taped", "nh_adjoint_step", "nh_cheb_forms", "nh_cheb_cyclic_forms",
           "nh_set_relax_target",
           "nh_debug_stall_copies", "nh_gauges")

BATCH_AUTOTUNE, BATCH_GRAPH = 1, 2

# kernel classes of nh_profile_t, in enum order
KERNELS = ("hyperbolic", "breaking", "assembly", "solve_init", "bicg_A", "bicg_B", "bicg_C",
           "cheb_pass", "tridiag", "correction", "adj_hyperbolic", "adj_assembly",
           "adj_correction", "w_transport", "relax", "bicg_block")


class ProfileT(C.Structure):
    _fields_ = [("launches", C.c_longlong * len(KERNELS)), ("ms", C.c_double * len(KERNELS))]


def load():
    """Load libnh.so (built in-tree by build.py / __graft_entry__.build()); raise if absent."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"libnh.so not found at {LIB_PATH}; run __graft_entry__.build()")
    L = C.CDLL(LIB_PATH)
    vp, H = C.c_void_p, C.c_void_p
    L.nh_default_params.argtypes = [C.POINTER(Params)]
    L.nh_create.argtypes = [C.POINTER(Grid), C.POINTER(C.c_double), C.POINTER(Params), vp,
                            C.POINTER(H)]
    L.nh_set_state.argtypes = [H, vp, vp, vp, vp, vp, C.c_double, C.c_int]
    L.nh_get_state.argtypes = [H, vp, vp, vp, vp, vp, C.POINTER(C.c_double), C.c_int]
    L.nh_step.argtypes = [H, C.c_double, C.POINTER(C.c_double)]
    L.nh_run.argtypes = [H, C.c_double, C.c_longlong, C.POINTER(C.c_longlong)]
    L.nh_stats.argtypes = [H, C.POINTER(StatsT)]
    L.nh_last_error.argtypes = [H]
    L.nh_last_error.restype = C.c_char_p
    L.nh_destroy.argtypes = [H]
    L.nh_destroy.restype = None
    L.nh_profile_enable.argtypes = [H, C.c_int]
    L.nh_profile_read.argtypes = [H, C.POINTER(ProfileT)]
    L.nh_tridiag_batched.argtypes = [C.c_int, C.c_int, C.c_int, vp, vp, vp, vp, vp, vp]
    L.nh_debug_hyperbolic.argtypes = [H, C.c_double, vp, vp, vp, C.c_int]
    L.nh_debug_system.argtypes = [H, C.c_double, vp, vp, vp, C.c_int]
    L.nh_debug_stall_copies.argtypes = [H, C.c_int]
    L.nh_gauges.argtypes = [H, vp, C.c_int, vp]
    L.nh_set_relax_target.argtypes = [H, vp, vp, vp, vp, vp, C.c_int]
    L.nh_create_batch.argtypes = [C.c_int, C.POINTER(Grid), C.POINTER(C.c_void_p),
                                  C.POINTER(Params), vp, C.c_int, C.POINTER(H)]
    L.nh_batch_set_state.argtypes = [H, C.c_int, vp, vp, vp, vp, vp, C.c_double, C.c_int]
    L.nh_batch_get_state.argtypes = [H, C.c_int, vp, vp, vp, vp, vp, C.POINTER(C.c_double),
                                     C.c_int]
    L.nh_batch_run.argtypes = [H, C.c_int]
    L.nh_batch_stats.argtypes = [H, C.c_int, C.POINTER(StatsT)]
    L.nh_batch_get_tuning.argtypes = [H, C.POINTER(BatchTuning)]
    L.nh_batch_set_tuning.argtypes = [H, C.POINTER(BatchTuning)]
    L.nh_batch_candidate.argtypes = [C.c_int, C.c_int, C.c_int, C.POINTER(C.c_int),
                                     C.POINTER(C.c_int), C.POINTER(C.c_int)]
    L.nh_batch_last_error.argtypes = [H]
    L.nh_batch_last_error.restype = C.c_char_p
    L.nh_batch_destroy.argtypes = [H]
    L.nh_batch_destroy.restype = None
    L.nh_tape_bytes.argtypes = [H]
    L.nh_tape_bytes.restype = C.c_size_t
    L.nh_step_taped.argtypes = [H, C.c_double, vp, C.POINTER(C.c_double)]
    L.nh_adjoint_step.argtypes = [H, C.c_double, vp, vp, vp, vp, vp, vp]
    L.nh_batch_profile_enable.argtypes = [H, C.c_int]
    L.nh_batch_profile_read.argtypes = [H, C.POINTER(ProfileT)]
    L.nh_cheb_forms.argtypes = [C.c_int]
    L.nh_cheb_cyclic_forms.argtypes = [C.c_int]
    _lib = L
    return L


def default_params() -> Params:
    p = Params()
    load().nh_default_params(C.byref(p))
    return p


def cheb_forms(precision: str = "fp32") -> int:
    """Number of kernel forms of the Chebyshev pass (values of the cheb_form parameter)."""
    n = load().nh_cheb_forms(FP32 if precision == "fp32" else FP64)
    if n < 0:
        raise ValueError(precision)
    return n


def cheb_cyclic_forms(precision: str = "fp32") -> int:
    """Number of kernel forms of the cyclic pass (reported as cheb_form = cheb_forms() + k)."""
    n = load().nh_cheb_cyclic_forms(FP32 if precision == "fp32" else FP64)
    if n < 0:
        raise ValueError(precision)
    return n


def tridiag_batched(a, b, c, d, x, stream=None):
    """Batched tridiagonal solve on torch CUDA tensors of shape [rows, n] (float32/64)."""
    import torch
    rows, n = d.shape
    prec = FP64 if d.dtype == torch.float64 else FP32
    for t in (a, b, c, d, x):
        assert t.is_cuda and t.is_contiguous() and t.dtype == d.dtype and t.shape == d.shape
    s = stream.cuda_stream if stream is not None else torch.cuda.current_stream().cuda_stream
    rc = load().nh_tridiag_batched(n, rows, prec, *[C.c_void_p(t.data_ptr()) for t in
                                                    (a, b, c, d, x)], C.c_void_p(s))
    if rc != OK:
        raise NHError(rc, "nh_tridiag_batched failed")


def _is_torch(a) -> bool:
    return type(a).__module__.startswith("torch")


class Sim:
    """One simulation handle (2D grid, or ny independent 1D channels when dim = 1)."""

    def __init__(self, H, dx, dy=None, dim=2, bc=(WALL,) * 4, precision="fp64", stream=None,
                 **params):
        L = load()
        H = np.ascontiguousarray(np.asarray(H, dtype=np.float64))
        if dim == 1 and H.ndim == 1:
            H = H[None, :]
        ny, nx = H.shape
        self.dim, self.nx, self.ny = dim, nx, ny
        self.dtype = np.float32 if precision == "fp32" else np.float64
        self.nnode = (nx + 1) * (ny + 1) if dim == 2 else (nx + 1) * ny
        g = Grid()
        g.dim, g.nx, g.ny, g.dx = dim, nx, ny, float(dx)
        g.dy = float(dx if dy is None else dy)
        for k in range(4):
            g.bc[k] = int(bc[k])
        p = default_params()
        p.precision = FP32 if precision == "fp32" else FP64
        for k, v in params.items():
            if not hasattr(p, k):
                raise TypeError(f"unknown parameter {k}")
            if isinstance(getattr(p, k), C.Array):   # e.g. relax_width = (w, e, s, n)
                v = type(getattr(p, k))(*v)
            setattr(p, k, v)
        self.params = p
        self._h = C.c_void_p()
        s = stream.cuda_stream if hasattr(stream, "cuda_stream") else (stream or 0)
        rc = L.nh_create(C.byref(g), H.ctypes.data_as(C.POINTER(C.c_double)), C.byref(p),
                         C.c_void_p(s), C.byref(self._h))
        if rc != OK:
            raise NHError(rc, "nh_create failed")
        self._keep = []

    # -------------------------------------------------------------- helpers
    def _check(self, rc):
        if rc != OK:
            raise NHError(rc, load().nh_last_error(self._h).decode())

    def _arr(self, a, n):
        """Pointer + where for a numpy host array or a torch CUDA tensor of n elements."""
        if a is None:
            return None, HOST
        if _is_torch(a):
            assert a.is_contiguous() and a.numel() == n
            assert a.element_size() == np.dtype(self.dtype).itemsize
            return C.c_void_p(a.data_ptr()), (DEVICE if a.is_cuda else HOST)
        a = np.ascontiguousarray(np.asarray(a, dtype=self.dtype)).reshape(-1)
        assert a.size == n, (a.size, n)
        self._keep.append(a)
        return C.c_void_p(a.ctypes.data), HOST

    @property
    def node_shape(self):
        return (self.ny + 1, self.nx + 1) if self.dim == 2 else (self.ny, self.nx + 1)

    # -------------------------------------------------------------- API
    def set_state(self, eta, q1, q2=None, w=None, p=None, t=0.0):
        nc = self.nx * self.ny
        args = [self._arr(eta, nc), self._arr(q1, nc), self._arr(q2, nc),
                self._arr(w, self.nnode), self._arr(p, self.nnode)]
        wheres = {wh for ptr, wh in args if ptr is not None}
        assert len(wheres) == 1, "mixing host and device arrays"
        self._check(load().nh_set_state(self._h, *[a[0] for a in args], float(t), wheres.pop()))
        self._keep.clear()

    def set_relax_target(self, eta=None, q1=None, q2=None, w=None, p=None):
        """nh_set_relax_target: target of the Sec. 4.4 relaxation zones (None: unchanged)."""
        nc = self.nx * self.ny
        args = [self._arr(eta, nc), self._arr(q1, nc), self._arr(q2, nc),
                self._arr(w, self.nnode), self._arr(p, self.nnode)]
        wheres = {wh for ptr, wh in args if ptr is not None}
        assert len(wheres) <= 1, "mixing host and device arrays"
        self._check(load().nh_set_relax_target(self._h, *[a[0] for a in args],
                                               wheres.pop() if wheres else HOST))
        self._keep.clear()

    def get_state(self):
        out = {k: np.empty((self.ny, self.nx), self.dtype) for k in ("eta", "q1", "q2")}
        out["w"] = np.empty(self.node_shape, self.dtype)
        out["p"] = np.empty(self.node_shape, self.dtype)
        t = C.c_double()
        self._check(load().nh_get_state(self._h, *[C.c_void_p(out[k].ctypes.data) for k in
                                                   ("eta", "q1", "q2", "w", "p")],
                                        C.byref(t), HOST))
        out["t"] = t.value
        return out

    def get_state_into(self, eta=None, q1=None, q2=None, w=None, p=None):
        """Copy the state into caller buffers (numpy host or torch CUDA tensors)."""
        nc = self.nx * self.ny
        args = [self._arr(eta, nc), self._arr(q1, nc), self._arr(q2, nc),
                self._arr(w, self.nnode), self._arr(p, self.nnode)]
        wheres = {wh for ptr, wh in args if ptr is not None}
        where = wheres.pop() if wheres else HOST
        self._check(load().nh_get_state(self._h, *[a[0] for a in args], None, where))
        self._keep.clear()

    def gauges(self, cells, out):
        """nh_gauges: eta at `cells` (torch CUDA int32 tensor of row-major cell indices)
        into `out` (torch CUDA tensor of the handle's precision), on the handle's stream."""
        assert cells.is_cuda and out.is_cuda and cells.dtype.itemsize == 4
        assert out.element_size() == np.dtype(self.dtype).itemsize
        assert cells.is_contiguous() and out.is_contiguous() and out.numel() >= cells.numel()
        self._check(load().nh_gauges(self._h, C.c_void_p(cells.data_ptr()), int(cells.numel()),
                                     C.c_void_p(out.data_ptr())))

    def step(self, dt=0.0):
        d = C.c_double()
        self._check(load().nh_step(self._h, float(dt), C.byref(d)))
        return d.value

    def run(self, t_end=0.0, max_steps=1 << 40):
        s = C.c_longlong()
        self._check(load().nh_run(self._h, float(t_end), int(max_steps), C.byref(s)))
        return s.value

    def stats(self):
        st = StatsT()
        self._check(load().nh_stats(self._h, C.byref(st)))
        return dict(t=st.t, dt=st.dt, dt_next=st.dt_next, steps=st.steps,
                    solver_iters=st.solver_iters, last_iters=tuple(st.last_iters),
                    last_resid=tuple(st.last_resid), mass=st.mass, nonfinite=st.nonfinite,
                    fallbacks=st.fallbacks, fallback_iters=st.fallback_iters,
                    cheb_form=st.cheb_form)

    def profile(self, on=True):
        """Record CUDA events around every kernel launch (resets the counters)."""
        self._check(load().nh_profile_enable(self._h, 1 if on else 0))

    def profile_read(self):
        pr = ProfileT()
        self._check(load().nh_profile_read(self._h, C.byref(pr)))
        return {k: (pr.launches[i], pr.ms[i]) for i, k in enumerate(KERNELS)}

    def debug_hyperbolic(self, dt):
        out = [np.empty((self.ny, self.nx), self.dtype) for _ in range(3)]
        self._check(load().nh_debug_hyperbolic(self._h, float(dt),
                                               *[C.c_void_p(o.ctypes.data) for o in out], HOST))
        return out

    def debug_stall_copies(self, block=0):
        """nh_debug_stall_copies: the next register-form pass lets `block` wait for copies
        it never issued (its wait runs out; the step returns ETIMEOUT)."""
        self._check(load().nh_debug_stall_copies(self._h, int(block)))

    def debug_system(self, dt, x):
        x = np.ascontiguousarray(np.asarray(x, dtype=self.dtype)).reshape(self.node_shape)
        rhs = np.empty(self.node_shape, self.dtype)
        mx = np.empty(self.node_shape, self.dtype)
        self._check(load().nh_debug_system(self._h, float(dt), C.c_void_p(x.ctypes.data),
                                           C.c_void_p(rhs.ctypes.data),
                                           C.c_void_p(mx.ctypes.data), HOST))
        return rhs, mx

    # -------------------------------------------------------------- adjoint
    def tape_bytes(self):
        return int(load().nh_tape_bytes(self._h))

    def step_taped(self, tape, dt=0.0):
        """nh_step_taped into a device buffer (torch tensor of >= tape_bytes bytes)."""
        d = C.c_double()
        self._check(load().nh_step_taped(self._h, float(dt), C.c_void_p(tape.data_ptr()),
                                         C.byref(d)))
        return d.value

    def adjoint_step(self, tape, dt, eta_bar, q1_bar, q2_bar, w_bar, H_bar):
        """nh_adjoint_step on torch CUDA tensors (in place; H_bar accumulates)."""
        for t in (eta_bar, q1_bar, q2_bar, w_bar, H_bar):
            assert t.is_cuda and t.is_contiguous()
            assert t.element_size() == np.dtype(self.dtype).itemsize
        self._check(load().nh_adjoint_step(self._h, float(dt), C.c_void_p(tape.data_ptr()),
                                           *[C.c_void_p(t.data_ptr()) for t in
                                             (eta_bar, q1_bar, q2_bar, w_bar, H_bar)]))

    def close(self):
        if self._h:
            load().nh_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def batch_candidates(precision="fp32"):
    """Kernel-shape candidates of the batched form: {kind: [(tile_x, tile_y, threads)]}."""
    L = load()
    prec = FP32 if precision == "fp32" else FP64
    out = {}
    for kind, name in enumerate(("hyp", "assembly", "cheb")):
        lst = []
        while True:
            tx, ty, th = C.c_int(), C.c_int(), C.c_int()
            if L.nh_batch_candidate(prec, kind, len(lst), C.byref(tx), C.byref(ty),
                                    C.byref(th)) != OK:
                break
            lst.append((tx.value, ty.value, th.value))
        out[name] = lst
    return out


class Batch:
    """An ensemble of independent 2D domains of uneven sizes advanced together
    (nh_create_batch).  Hs: list of [ny][nx] still-water depths; grids share dx unless
    `dxs` is given; bcs: one (w, e, s, n) tuple for all or one per domain."""

    def __init__(self, Hs, dx=0.1, dxs=None, bcs=(WALL,) * 4, precision="fp32", stream=None,
                 autotune=False, graph=False, **params):
        L = load()
        self.Hs = [np.ascontiguousarray(np.asarray(H, dtype=np.float64)) for H in Hs]
        n = len(self.Hs)
        self.n = n
        self.dtype = np.float32 if precision == "fp32" else np.float64
        grids = (Grid * n)()
        per_bc = len(bcs) == n and not isinstance(bcs[0], int)
        for d, H in enumerate(self.Hs):
            ny, nx = H.shape
            g = grids[d]
            g.dim, g.nx, g.ny = 2, nx, ny
            g.dx = g.dy = float(dx if dxs is None else dxs[d])
            bc = bcs[d] if per_bc else bcs
            for k in range(4):
                g.bc[k] = int(bc[k])
        self.shapes = [H.shape for H in self.Hs]
        p = default_params()
        p.precision = FP32 if precision == "fp32" else FP64
        for k, v in params.items():
            if not hasattr(p, k):
                raise TypeError(f"unknown parameter {k}")
            if isinstance(getattr(p, k), C.Array):   # e.g. relax_width = (w, e, s, n)
                v = type(getattr(p, k))(*v)
            setattr(p, k, v)
        self.params = p
        ptrs = (C.c_void_p * n)(*[H.ctypes.data for H in self.Hs])
        flags = (BATCH_AUTOTUNE if autotune else 0) | (BATCH_GRAPH if graph else 0)
        s = stream.cuda_stream if hasattr(stream, "cuda_stream") else (stream or 0)
        self._h = C.c_void_p()
        rc = L.nh_create_batch(n, grids, ptrs, C.byref(p), C.c_void_p(s), flags,
                               C.byref(self._h))
        if rc != OK:
            raise NHError(rc, "nh_create_batch failed")
        self._keep = []

    def _check(self, rc):
        if rc != OK:
            raise NHError(rc, load().nh_batch_last_error(self._h).decode())

    def _arr(self, a, n):
        if a is None:
            return None, HOST
        if _is_torch(a):
            assert a.is_contiguous() and a.numel() == n
            assert a.element_size() == np.dtype(self.dtype).itemsize
            return C.c_void_p(a.data_ptr()), (DEVICE if a.is_cuda else HOST)
        a = np.ascontiguousarray(np.asarray(a, dtype=self.dtype)).reshape(-1)
        assert a.size == n, (a.size, n)
        self._keep.append(a)
        return C.c_void_p(a.ctypes.data), HOST

    def set_state(self, d, eta, q1, q2=None, w=None, p=None, t=0.0):
        ny, nx = self.shapes[d]
        nc, nn = nx * ny, (nx + 1) * (ny + 1)
        args = [self._arr(eta, nc), self._arr(q1, nc), self._arr(q2, nc), self._arr(w, nn),
                self._arr(p, nn)]
        wheres = {wh for ptr, wh in args if ptr is not None}
        assert len(wheres) == 1, "mixing host and device arrays"
        self._check(load().nh_batch_set_state(self._h, d, *[a[0] for a in args], float(t),
                                              wheres.pop()))
        self._keep.clear()

    def get_state(self, d):
        ny, nx = self.shapes[d]
        out = {k: np.empty((ny, nx), self.dtype) for k in ("eta", "q1", "q2")}
        out["w"] = np.empty((ny + 1, nx + 1), self.dtype)
        out["p"] = np.empty((ny + 1, nx + 1), self.dtype)
        t = C.c_double()
        self._check(load().nh_batch_get_state(self._h, d, *[C.c_void_p(out[k].ctypes.data)
                                                            for k in ("eta", "q1", "q2", "w",
                                                                      "p")],
                                              C.byref(t), HOST))
        out["t"] = t.value
        return out

    def get_state_into(self, d, eta=None, q1=None, q2=None, w=None, p=None):
        ny, nx = self.shapes[d]
        nc, nn = nx * ny, (nx + 1) * (ny + 1)
        args = [self._arr(eta, nc), self._arr(q1, nc), self._arr(q2, nc), self._arr(w, nn),
                self._arr(p, nn)]
        wheres = {wh for ptr, wh in args if ptr is not None}
        where = wheres.pop() if wheres else HOST
        self._check(load().nh_batch_get_state(self._h, d, *[a[0] for a in args], None, where))
        self._keep.clear()

    def run(self, nsteps=1):
        self._check(load().nh_batch_run(self._h, int(nsteps)))

    def stats(self, d):
        st = StatsT()
        self._check(load().nh_batch_stats(self._h, d, C.byref(st)))
        return dict(t=st.t, dt=st.dt, dt_next=st.dt_next, steps=st.steps,
                    solver_iters=st.solver_iters, last_iters=tuple(st.last_iters),
                    last_resid=tuple(st.last_resid), mass=st.mass, nonfinite=st.nonfinite,
                    fallbacks=st.fallbacks, fallback_iters=st.fallback_iters,
                    cheb_form=st.cheb_form)

    def profile(self, on=True):
        """Record CUDA events around every kernel launch (steps then run eagerly)."""
        self._check(load().nh_batch_profile_enable(self._h, 1 if on else 0))

    def profile_read(self):
        pr = ProfileT()
        self._check(load().nh_batch_profile_read(self._h, C.byref(pr)))
        return {k: (pr.launches[i], pr.ms[i]) for i, k in enumerate(KERNELS)}

    def tuning(self):
        t = BatchTuning()
        self._check(load().nh_batch_get_tuning(self._h, C.byref(t)))
        return dict(hyp=t.hyp, assembly=t.assembly, cheb=t.cheb, persistent=t.persistent,
                    graph=t.graph, tuned=t.tuned, ms=tuple(t.ms))

    def set_tuning(self, hyp=0, assembly=0, cheb=0, persistent=0, graph=0):
        t = BatchTuning()
        t.hyp, t.assembly, t.cheb, t.persistent, t.graph = hyp, assembly, cheb, persistent, graph
        self._check(load().nh_batch_set_tuning(self._h, C.byref(t)))

    def close(self):
        if self._h:
            load().nh_batch_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
