"""Seeded synthetic workloads shaped like the paper's tests (Sec. 7).

This module only draws inputs: still-water depth H (positive below the datum), initial
free surface eta0 and discharges.  It holds none of the scheme's arithmetic and is the
one piece shared by the CUDA path's callers and the oracle's callers.  All arrays are
float64, row-major [ny][nx] with x fastest; cell (i, j) is centred at ((i+1/2) dx,
(j+1/2) dy).

Workloads (names used by tests and bench.py):
  solitary_1d      -- flat channel, solitary wave of Eq. (33) (Sec. 7.1 setup, walls).
  shoals_2d        -- all-wet basin over Gaussian shoals with a Gaussian hump.
  island_2d        -- conical island with a dry top and an incoming solitary wave
                      (geometry of Sec. 7.6; wet/dry, breaking and friction on).
  ensemble_member  -- one domain of an uneven ensemble (Gaussian-sum bathymetry with
                      dry patches, random humps).
  adjoint_2d       -- all-wet Gaussian-sum basin, initial hump, target-run bathymetry and
                      gauge positions for a gauge-misfit gradient.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

G = 9.81


@dataclass
class Workload:
    name: str
    nx: int
    ny: int
    dx: float
    dy: float
    H: np.ndarray            # still-water depth, [ny][nx] (1D: [nx])
    eta: np.ndarray          # initial free surface (dry cells: eta = -H)
    q1: np.ndarray
    q2: np.ndarray
    bc: tuple = (0, 0, 0, 0)  # west, east, south, north: 0 wall, 1 outflow
    params: dict = field(default_factory=dict)
    extra: dict = field(default_factory=dict)

    @property
    def h(self) -> np.ndarray:
        return np.maximum(self.eta + self.H, 0.0)


def _sech2(z):
    return 1.0 / np.cosh(np.clip(z, -350.0, 350.0)) ** 2


def solitary_1d(n: int = 1000, L: float = 200.0, h0: float = 1.0, A: float = 0.2,
                x0: float = 50.0, g: float = G) -> Workload:
    """Flat channel with walls and the solitary wave of Eq. (33):
    eta = A sech^2(k (x - x0)), k = sqrt(3A / (4 h0^3)), u = c eta / (h0 + eta),
    c = sqrt(g (h0 + A))."""
    dx = L / n
    x = (np.arange(n) + 0.5) * dx
    k = np.sqrt(3.0 * A / (4.0 * h0 ** 3))
    c = np.sqrt(g * (h0 + A))
    eta = A * _sech2(k * (x - x0))
    H = np.full(n, h0)
    h = H + eta
    q = h * c * eta / (h0 + eta)
    return Workload("solitary_1d", n, 1, dx, dx, H, eta, q, np.zeros(n),
                    params=dict(g=g, cfl=0.9, t_end=20.0))


def shoals_2d(n: int = 1024, L: float = 102.4, seed: int = 2, depth: float = 0.5,
              nshoal: int = 8, hump: float = 0.05, hump_sigma: float = 3.0,
              min_depth: float = 0.1) -> Workload:
    """All-wet basin with walls: H = depth - sum of nshoal Gaussian shoals (height
    U[0.1, 0.3] m, sigma U[2, 6] m, centres uniform over [0.1 L, 0.9 L]^2), redrawn with
    seed + 1, seed + 2, ... until min H >= min_depth.  Initial Gaussian hump of amplitude
    `hump` and sigma `hump_sigma` at the basin centre, at rest."""
    dx = L / n
    x = (np.arange(n) + 0.5) * dx
    X, Y = np.meshgrid(x, x)
    s = seed
    for _ in range(10000):
        rng = np.random.default_rng(s)
        amp = rng.uniform(0.1, 0.3, nshoal)
        sig = rng.uniform(2.0, 6.0, nshoal)
        cen = rng.uniform(0.1 * L, 0.9 * L, (nshoal, 2))
        H = np.full((n, n), depth)
        for a, sg, (cx, cy) in zip(amp, sig, cen):
            H -= a * np.exp(-((X - cx) ** 2 + (Y - cy) ** 2) / (2.0 * sg * sg))
        if H.min() >= min_depth:
            break
        s += 1
    else:
        raise ValueError("shoals_2d: no draw with min depth >= %g for L = %g" % (min_depth, L))
    eta = hump * np.exp(-((X - L / 2) ** 2 + (Y - L / 2) ** 2) / (2.0 * hump_sigma ** 2))
    z = np.zeros((n, n))
    return Workload("shoals_2d", n, n, dx, dx, H, eta, z, z.copy(),
                    params=dict(g=G, cfl=0.9), extra=dict(seed_used=s))


def island_2d(n: int = 4096, L: float = 204.8, depth: float = 0.32,
              center=(25.0, None), A: float = 0.064, x0: float = 5.0,
              base_radius: float = 3.6, crest: float = 0.625, slope: float = 0.25) -> Workload:
    """Conical island (Sec. 7.6 geometry: slope 1:4, 0.625 m high, base radius 3.6 m) in
    a basin of still depth 0.32 m with outflow boundaries; the bed is
    z_b = min(crest, slope (base_radius - r)) inside the base, H = depth - z_b, dry where
    H <= 0.  A solitary wave of Eq. (33) with amplitude A has its crest at x = x0 and
    travels in +x over the flat part."""
    dx = L / n
    x = (np.arange(n) + 0.5) * dx
    X, Y = np.meshgrid(x, x)
    cx = center[0]
    cy = L / 2 if center[1] is None else center[1]
    r = np.sqrt((X - cx) ** 2 + (Y - cy) ** 2)
    zb = np.where(r < base_radius, np.minimum(crest, slope * (base_radius - r)), 0.0)
    H = depth - zb
    k = np.sqrt(3.0 * A / (4.0 * depth ** 3))
    c = np.sqrt(G * (depth + A))
    eta_w = A * _sech2(k * (X - x0))
    flat = zb == 0.0
    wet = H > 0.0
    eta = np.where(flat, eta_w, np.where(wet, 0.0, -H))
    h = np.maximum(eta + H, 0.0)
    q1 = np.where(flat, h * c * eta_w / (depth + eta_w), 0.0)
    z = np.zeros((n, n))
    return Workload("island_2d", n, n, dx, dx, H, eta, q1, z, bc=(1, 1, 1, 1),
                    params=dict(g=G, cfl=0.9, manning=0.015, breaking=True,
                                B1=0.15, B2=0.5))


ENSEMBLE_SIDES = (128, 256, 512, 1024)


def ensemble_member(i: int, dx: float = 0.1, base_seed: int = 4000,
                    sides=ENSEMBLE_SIDES) -> Workload:
    """Domain i of the uneven ensemble (seed base_seed + i): side drawn uniformly from
    `sides`, walls, H = d0 - sum of m Gaussian bumps (d0 ~ U[0.2, 1.0], m ~ U{3..8},
    heights U[0.05, 1.0], sigma U[0.02, 0.08] L), dry where H <= 0; 1 to 3 Gaussian humps
    of amplitude U[0.01, 0.1] m and sigma U[0.02, 0.05] L on the wet cells."""
    rng = np.random.default_rng(base_seed + i)
    n = int(rng.choice(np.asarray(sides)))
    L = n * dx
    x = (np.arange(n) + 0.5) * dx
    X, Y = np.meshgrid(x, x)
    d0 = rng.uniform(0.2, 1.0)
    m = int(rng.integers(3, 9))
    H = np.full((n, n), d0)
    for _ in range(m):
        a = rng.uniform(0.05, 1.0)
        sg = rng.uniform(0.02, 0.08) * L
        cx, cy = rng.uniform(0.0, L, 2)
        H -= a * np.exp(-((X - cx) ** 2 + (Y - cy) ** 2) / (2.0 * sg * sg))
    wet = H > 0.0
    eta = np.zeros((n, n))
    for _ in range(int(rng.integers(1, 4))):
        a = rng.uniform(0.01, 0.1)
        sg = rng.uniform(0.02, 0.05) * L
        cx, cy = rng.uniform(0.2 * L, 0.8 * L, 2)
        eta += a * np.exp(-((X - cx) ** 2 + (Y - cy) ** 2) / (2.0 * sg * sg))
    eta = np.where(wet, eta, -H)
    z = np.zeros((n, n))
    return Workload(f"ensemble_member_{i}", n, n, dx, dx, H, eta, z, z.copy(),
                    params=dict(g=G, cfl=0.9))


def adjoint_2d(n: int = 512, dx: float = 0.1, seed: int = 5, target_seed: int = 6,
               ngauges: int = 16, hump: float = 0.05, hump_sigma: float = 3.0) -> Workload:
    """All-wet basin (walls): a Gaussian-sum field mapped affinely into [0.3, 0.8] m
    (seed), an initial hump at a seeded location, a target bathymetry H plus a seeded
    0.02-m Gaussian (target_seed), and ngauges seeded cell indices (row, column)."""
    L = n * dx
    x = (np.arange(n) + 0.5) * dx
    X, Y = np.meshgrid(x, x)
    rng = np.random.default_rng(seed)
    F = np.zeros((n, n))
    for _ in range(8):
        a = rng.uniform(-1.0, 1.0)
        sg = rng.uniform(0.05, 0.2) * L
        cx, cy = rng.uniform(0.0, L, 2)
        F += a * np.exp(-((X - cx) ** 2 + (Y - cy) ** 2) / (2.0 * sg * sg))
    F = (F - F.min()) / max(F.max() - F.min(), 1e-30)
    H = 0.3 + 0.5 * F
    hx, hy = rng.uniform(0.3 * L, 0.7 * L, 2)
    eta = hump * np.exp(-((X - hx) ** 2 + (Y - hy) ** 2) / (2.0 * hump_sigma ** 2))
    trng = np.random.default_rng(target_seed)
    tx, ty = trng.uniform(0.2 * L, 0.8 * L, 2)
    tsg = trng.uniform(0.05, 0.1) * L
    H_target = H + 0.02 * np.exp(-((X - tx) ** 2 + (Y - ty) ** 2) / (2.0 * tsg * tsg))
    grng = np.random.default_rng(seed + 1000)
    gauges = np.stack([grng.integers(2, n - 2, ngauges), grng.integers(2, n - 2, ngauges)], 1)
    z = np.zeros((n, n))
    return Workload("adjoint_2d", n, n, dx, dx, H, eta, z, z.copy(),
                    params=dict(g=G, cfl=0.9),
                    extra=dict(H_target=H_target, gauges=gauges))


def dambreak_2d(n: int = 1000, L: float = 10.0) -> Workload:
    """Circular dam-break of Sec. 7.7: [-L/2, L/2]^2, H = 1 - 0.25 exp(-x^2 - y^2), h0 = H
    for r <= 0.5 and H + 0.25 outside (eta0 = 0 inside, 0.25 outside), q = 0, open
    (outflow) boundaries; the paper runs t in [0, 1] at CFL 0.9 on n^2 meshes, n from 250
    to 1500."""
    dx = L / n
    x = (np.arange(n) + 0.5) * dx - L / 2
    X, Y = np.meshgrid(x, x)
    H = 1.0 - 0.25 * np.exp(-X * X - Y * Y)
    eta = np.where(np.sqrt(X * X + Y * Y) <= 0.5, 0.0, 0.25)
    z = np.zeros((n, n))
    return Workload("dambreak_2d", n, n, dx, dx, H, eta, z, z.copy(), bc=(1, 1, 1, 1),
                    params=dict(g=G, cfl=0.9, t_end=1.0))
