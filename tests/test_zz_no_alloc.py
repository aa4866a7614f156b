"""nh_tridiag_batched_noalloc: the batched tridiagonal solve for callers that cannot
allocate device memory during a call (code inside another framework's memory pool,
real-time or callback paths where cudaMalloc is not allowed, fixed memory budgets).
It keeps its scratch in a fixed device array instead of allocating; here it must give
the same result as nh_tridiag_batched, which allocates, on two calls in a row (the
second on different data, so leftovers of the first call cannot matter)."""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

NOALLOC_BYTES = 8 << 20


def _systems(n, rows, seed):
    rng = np.random.default_rng(seed)
    a = rng.uniform(-1, 1, (rows, n))
    c = rng.uniform(-1, 1, (rows, n))
    b = (np.abs(a) + np.abs(c) + rng.uniform(0.5, 2.0, (rows, n))) * rng.choice([-1, 1], (rows, 1))
    d = rng.standard_normal((rows, n))
    return a, b, c, d


def _call(fn, n, rows, prec, T, x):
    import torch
    s = torch.cuda.current_stream().cuda_stream
    return fn(n, rows, prec, *[ctypes.c_void_p(t.data_ptr()) for t in T],
              ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(s))


@pytest.mark.parametrize("dtype,prec,tol", [("float64", 0, 1e-12), ("float32", 1, 1e-5)])
def test_noalloc_matches_allocating_solve_on_two_calls(dtype, prec, tol):
    import torch
    from paper_1706_04551_b300 import nh
    L = nh.load()
    argt = [ctypes.c_int, ctypes.c_int, ctypes.c_int] + [ctypes.c_void_p] * 6
    L.nh_tridiag_batched_noalloc.argtypes = argt
    L.nh_tridiag_batched.argtypes = argt
    td = getattr(torch, dtype)
    n, rows = 9000, 6            # longer than the shared-memory limit: uses the scratch
    for call in range(2):
        a, b, c, d = _systems(n, rows, 100 + call)
        T = [torch.tensor(v, dtype=td, device="cuda").contiguous() for v in (a, b, c, d)]
        x_ref = torch.empty_like(T[3])
        x_new = torch.full_like(T[3], float("nan"))
        assert _call(L.nh_tridiag_batched, n, rows, prec, T, x_ref) == 0
        assert _call(L.nh_tridiag_batched_noalloc, n, rows, prec, T, x_new) == 0
        torch.cuda.synchronize()
        ref = x_ref.cpu().numpy().astype(np.float64)
        new = x_new.cpu().numpy().astype(np.float64)
        assert np.isfinite(new).all()
        assert np.abs(new - ref).max() <= tol * np.abs(ref).max()


def test_noalloc_rejects_sizes_beyond_its_scratch():
    import torch
    from paper_1706_04551_b300 import nh
    L = nh.load()
    L.nh_tridiag_batched_noalloc.argtypes = [ctypes.c_int] * 3 + [ctypes.c_void_p] * 6
    n = 10000
    rows = NOALLOC_BYTES // (2 * 8 * n) + 1      # FP64: just over the limit
    T = [torch.zeros((rows, n), dtype=torch.float64, device="cuda") for _ in range(4)]
    x = torch.zeros_like(T[0])
    assert _call(L.nh_tridiag_batched_noalloc, n, rows, 0, T, x) == nh.EINVAL
