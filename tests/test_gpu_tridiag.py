"""Batched tridiagonal solve (App. B Eqs. 42-43 systems) through the C-ABI, against
scipy's banded LU on random diagonally dominant systems."""
import numpy as np
import pytest
from scipy.linalg import solve_banded

pytestmark = pytest.mark.gpu


def systems(n, rows, seed):
    rng = np.random.default_rng(seed)
    a = rng.uniform(-1, 1, (rows, n))
    c = rng.uniform(-1, 1, (rows, n))
    b = np.abs(a) + np.abs(c) + rng.uniform(0.5, 2.0, (rows, n))
    b *= rng.choice([-1, 1], (rows, 1))
    d = rng.standard_normal((rows, n))
    return a, b, c, d


def reference(a, b, c, d):
    rows, n = d.shape
    x = np.empty_like(d)
    for r in range(rows):
        ab = np.zeros((3, n))
        ab[0, 1:] = c[r, :-1]
        ab[1] = b[r]
        ab[2, :-1] = a[r, 1:]
        x[r] = solve_banded((1, 1), ab, d[r])
    return x


@pytest.mark.parametrize("n,rows", [(1001, 3), (37, 5), (6000, 4)])
@pytest.mark.parametrize("dtype", ["float64", "float32"])
def test_tridiag_batched_matches_banded_lu(n, rows, dtype):
    import torch
    from paper_1706_04551_b300 import nh
    a, b, c, d = systems(n, rows, n + rows)
    ref = reference(a, b, c, d)
    td = getattr(torch, dtype)
    T = [torch.tensor(v, dtype=td, device="cuda").contiguous() for v in (a, b, c, d)]
    x = torch.empty_like(T[3])
    nh.tridiag_batched(*T, x)
    torch.cuda.synchronize()
    err = np.abs(x.cpu().numpy().astype(np.float64) - ref).max() / np.abs(ref).max()
    assert err < (1e-12 if dtype == "float64" else 1e-5), err
