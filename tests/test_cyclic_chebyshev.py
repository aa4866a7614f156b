"""The cyclic form of the Chebyshev-scheduled Jacobi solve, on the CPU (numpy, no GPU).

Sec. 5 solves the pressure system by Jacobi with scheduled relaxation; the passes use
Chebyshev weights for the interval [1 - g, 1 + g] of D^-1 M (g the largest Gershgorin
radius), x_{k+1} = x_k + c1_k (x_k - x_{k-1}) + c2_k r_k with r_k = D^-1 (b - M x_k).  The
five-point rows (mirror images at walls included) couple each node only with nodes of the
other colour (I + J) mod 2, and the interval is centred at 1, so c1 = c2 - 1 and one colour
at the odd steps and the other at the even steps form a closed recurrence (Golub and
Varga's cyclic Chebyshev method).  These tests check that reading of the method on small
mirrored systems: the in-place colour steps x <- x + c2 r reproduce the full iteration's
values, and the residual the cyclic pass measures is that of a well-defined vector.
"""
import numpy as np


def mirrored_rows(ny, nx, seed):
    """Random non-symmetric, diagonally dominant five-point rows on (ny x nx) nodes with the
    wall mirror of the pass (a neighbour outside the grid is the node's mirror image)."""
    rng = np.random.default_rng(seed)
    n = ny * nx
    M = np.zeros((n, n))
    for j in range(ny):
        for i in range(nx):
            r = j * nx + i
            M[r, r] += 4.0 + rng.random()
            for dj, di in ((0, -1), (0, 1), (-1, 0), (1, 0)):
                jj, ii = j + dj, i + di
                ii = -ii if ii < 0 else (2 * (nx - 1) - ii if ii >= nx else ii)
                jj = -jj if jj < 0 else (2 * (ny - 1) - jj if jj >= ny else jj)
                M[r, jj * nx + ii] -= 0.95 * rng.random()
    colour = (np.add.outer(np.arange(ny), np.arange(nx)) & 1).ravel()
    return M, colour


def weights(g, n):
    """The pass control's Chebyshev weights for [1 - g, 1 + g]: c1_0 = 0, c2_0 = 1, then
    rho_{k+1} = 1 / (2 / g - rho_k), c1 = rho_{k+1} rho_k, c2 = 2 rho_{k+1} / g."""
    c1, c2, rp = [0.0], [1.0], g
    for _ in range(1, n):
        rn = 1.0 / (2.0 / g - rp)
        c1.append(rn * rp)
        c2.append(2.0 * rn / g)
        rp = rn
    return np.array(c1), np.array(c2)


def setup(seed, ny=11, nx=14):
    M, colour = mirrored_rows(ny, nx, seed)
    D = np.diag(M)
    g = np.abs(np.eye(len(D)) - M / D[:, None]).sum(1).max()
    assert g < 1.0
    rng = np.random.default_rng(seed + 100)
    return M, D, colour, g, rng.standard_normal(len(D)), rng.standard_normal(len(D))


def test_rows_couple_the_two_colours_only():
    for seed in range(3):
        M, _, colour, *_ = setup(seed)
        off = M - np.diag(np.diag(M))
        same = colour[:, None] == colour[None, :]
        assert not off[same].any() and off[~same].any()


def test_weights_centred_at_one():
    """c1 = c2 - 1 for every step: the x_k term of the three-term step cancels."""
    for g in (0.3, 0.9, 0.983):
        c1, c2 = weights(g, 60)
        assert np.abs(c1 - (c2 - 1.0)).max() < 1e-15
        assert (c2 >= 1.0).all() and (c2 < 2.0).all()


def test_colour_steps_reproduce_the_full_iteration():
    """Step s updates colour s mod 2 in place; afterwards that colour holds x_s of the full
    Chebyshev-Jacobi iteration and the other colour x_{s-1} (from the same x_0)."""
    for seed in range(3):
        M, D, colour, g, b, x0 = setup(seed)
        c1, c2 = weights(g, 48)
        full = [x0.copy()]
        xp, x = x0.copy(), x0.copy()
        for k in range(48):
            xn = x + c1[k] * (x - xp) + c2[k] * (b - M @ x) / D
            xp, x = x, xn
            full.append(x)
        y = x0.copy()
        for k in range(48):
            u = (k + 1) & 1
            y = np.where(colour == u, y + c2[k] * (b - M @ y) / D, y)
            s = 1.0 + np.abs(full[k + 1]).max()
            assert np.abs(y - np.where(colour == u, full[k + 1], full[k])).max() < 1e-12 * s
        # and the cyclic iterate converges with the full one
        r_full = np.linalg.norm((b - M @ full[-1]) / D)
        r_cyc = np.linalg.norm((b - M @ y) / D)
        assert r_cyc < 1e-3 * np.linalg.norm(b / D) and r_cyc < 10 * r_full


def test_measured_residual_is_that_of_a_mixed_iterate():
    """Within a pass of K steps (K even, starting with colour 1), the colour-1 nodes of step
    K - 1 contribute (1 - c2) r and the colour-0 nodes of step K contribute r: together the
    scaled residual D^-1 (b - M z) of z = (colour 0 at step K - 2, colour 1 at step K - 1)."""
    K = 8
    for seed in range(3):
        M, D, colour, g, b, x0 = setup(seed)
        c1, c2 = weights(g, 3 * K)
        y = x0.copy()
        for k in range(3 * K):
            u = (k + 1) & 1
            r = (b - M @ y) / D
            if k % K == K - 2:   # step K - 1 of the pass: colour 1
                z = y.copy()
                meas = np.where(colour == 1, (1.0 - c2[k]) * r, 0.0)
            if k % K == K - 1:   # step K: colour 0; z's colour 1 is the step-(K-1) value
                meas = meas + np.where(colour == 0, r, 0.0)
            y = np.where(colour == u, y + c2[k] * r, y)
            if k % K == K - 2:
                z = np.where(colour == 1, y, z)   # colour 1 at step K - 1, colour 0 at K - 2
            if k % K == K - 1:
                want = (b - M @ z) / D
                assert np.abs(meas - want).max() < 1e-12 * (1.0 + np.abs(want).max())
