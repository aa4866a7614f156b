"""FP64 oracle of the adjoint (reverse-mode derivative) of the 2D step.

TEST INFRASTRUCTURE ONLY (same rule as the rest of ``oracle/``): imported by ``tests/`` and
``bench.py``'s baseline legs, never by the CUDA library, and sharing no code with it.

The paper has no adjoint; what is differentiated is the discrete step of App. A as the C
oracle computes it (``nh_oracle.c``: Eq. (30) hyperbolic update with MUSCL-minmod and the
PVM-HLL fluctuations of Eqs. (18)-(19), the pressure system of Eqs. (36)-(41) and the
correction, inside the Shu-Osher TVD-RK2 of Sec. 4.3 / 6).  This module restates that step
with plain PyTorch CPU operations in FP64, in the same order, so that torch.autograd (a
library primitive) gives the exact derivative of the discrete map:

  * ghost cells (walls: mirror with the normal discharge odd; outflow: copy) as padding;
  * the pressure system is built as a dense matrix from the linear map
    p -> B(q* + dt T(p), w* + dt p / h) (the same affine-map construction as the C
    oracle) and solved by a direct dense solve, so the derivative of the solve is the
    transposed solve M^T lambda = p_bar (plus the dependence of M on eta* and H);
  * friction and the breaking terms are not restated (the adjoint workload has neither);
    the emerging-bottom and dry-cell rules are kept, so the forward agrees with the C
    oracle on wet/dry states too.

Pins (``tests/test_oracle_adjoint.py``): the forward equals the C oracle's step; the
gradient of a gauge misfit equals central finite differences of the C oracle's forward;
the Jacobian-vector and vector-Jacobian products satisfy the dot-product identity.

Variables follow the C oracle: h (depth), q1, q2 at cells [ny][nx]; w, p at nodes
[ny+1][nx+1]; H still-water depth; eta = h - H.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import torch

WALL, OUTFLOW = 0, 1
SQRT2 = math.sqrt(2.0)


@dataclass
class Cfg2:
    nx: int
    ny: int
    dx: float
    dy: float
    bc: tuple = (WALL, WALL, WALL, WALL)
    g: float = 9.81
    delta: float = 1e-5
    hdry: float = 1e-5
    frozen_limiter: bool = False   # derivative with the limiter ratio held fixed (see slope())
    dry_zero: bool = True          # q = 0 in dry cells after each stage (as the C oracle's cfg)


def desing(h, q, delta):
    """Sec. 4.5: u = sqrt(2) h q / sqrt(h^4 + max(h^4, delta^4))."""
    h4 = h * h * h * h
    d4 = delta ** 4
    return SQRT2 * h * q / torch.sqrt(h4 + torch.clamp(h4, min=d4))


def minmod(a, b):
    """MUSCL limiter of Sec. 4.1 (zero when the signs differ)."""
    pos = (a > 0) & (b > 0)
    neg = (a < 0) & (b < 0)
    lo = torch.where(a < b, a, b)
    hi = torch.where(a > b, a, b)
    return torch.where(pos, lo, torch.where(neg, hi, torch.zeros_like(a)))


def slope(c: Cfg2, cm, c0, cp):
    """MUSCL slope minmod(c0 - cm, cp - c0).  Exact derivative by default; with
    c.frozen_limiter the derivative is that of phi * (cp - cm) / 2 with the ratio
    phi = slope / ((cp - cm) / 2) held at its value (0 where the centred difference is 0),
    a linearisation without the unlimited one-sided branches."""
    s = minmod(c0 - cm, cp - c0)
    if not c.frozen_limiter:
        return s
    cc = 0.5 * (cp - cm)
    nz = (cc != 0) & (s != 0)
    phi = torch.where(nz, s / torch.where(nz, cc, torch.ones_like(cc)), torch.zeros_like(s))
    return s.detach() + phi.detach() * (cc - cc.detach())


def pad_cells(c: Cfg2, v, px, py):
    """Two ghost layers: columns first (interior rows), then rows over every column."""
    w, e, s, n = c.bc
    if w == WALL:
        left = torch.stack([px * v[:, 1], px * v[:, 0]], 1)
    else:
        left = torch.stack([v[:, 0], v[:, 0]], 1)
    if e == WALL:
        right = torch.stack([px * v[:, -1], px * v[:, -2]], 1)
    else:
        right = torch.stack([v[:, -1], v[:, -1]], 1)
    v = torch.cat([left, v, right], 1)
    if s == WALL:
        bot = torch.stack([py * v[1], py * v[0]], 0)
    else:
        bot = torch.stack([v[0], v[0]], 0)
    if n == WALL:
        top = torch.stack([py * v[-1], py * v[-2]], 0)
    else:
        top = torch.stack([v[-1], v[-1]], 0)
    return torch.cat([bot, v, top], 0)


def pad_nodes(p):
    """Ghost nodes: the outside neighbour of a boundary node mirrors the inside one."""
    p = torch.cat([p[:, 1:2], p, p[:, -2:-1]], 1)
    return torch.cat([p[1:2], p, p[-2:-1]], 0)


def pvm(c: Cfg2, hL, eL, unL, utL, hR, eR, unR, utR):
    """Eqs. (18)-(19) in the face-normal frame (h, normal, tangential components)."""
    g = c.g
    qnL, qnR = hL * unL, hR * unR
    qtL, qtR = hL * utL, hR * utR
    hbar = 0.5 * (hL + hR)
    sL, sR = torch.sqrt(hL), torch.sqrt(hR)
    ss = sL + sR
    ubar = torch.where(ss > 0, (unL * sL + unR * sR) / torch.where(ss > 0, ss, torch.ones_like(ss)),
                       torch.zeros_like(ss))
    cbar = torch.sqrt(g * hbar)
    a_l, b_l = ubar - cbar, unL - torch.sqrt(g * hL)
    SL = torch.where(a_l < b_l, a_l, b_l)
    a_r, b_r = ubar + cbar, unR + torch.sqrt(g * hR)
    SR = torch.where(a_r > b_r, a_r, b_r)
    deta = eR - eL
    zero = torch.zeros_like(deta)
    deta = torch.where((hR <= c.hdry) & ((eR - hR) >= eL), zero, deta)
    deta = torch.where((hL <= c.hdry) & ((eL - hL) >= eR), zero, deta)
    span = SR - SL
    ok = span > 0
    sp = torch.where(ok, span, torch.ones_like(span))
    a0 = (SR * torch.abs(SL) - SL * torch.abs(SR)) / sp
    a1 = (torch.abs(SR) - torch.abs(SL)) / sp
    R = [qnR - qnL, qnR * unR - qnL * unL + g * hbar * deta, qnR * utR - qnL * utL]
    V = [deta, qnR - qnL, qtR - qtL]
    Dm = [torch.where(ok, 0.5 * ((1.0 - a1) * R[k] - a0 * V[k]), zero) for k in range(3)]
    Dp = [torch.where(ok, 0.5 * ((1.0 + a1) * R[k] + a0 * V[k]), zero) for k in range(3)]
    return Dm, Dp


def hyperbolic(c: Cfg2, H, h, q1, q2, dt):
    """Eq. (30) with the depth clamp (no friction): returns h, q1, q2 after dt."""
    nx, ny, g = c.nx, c.ny, c.g
    he, He = pad_cells(c, h, 1.0, 1.0), pad_cells(c, H, 1.0, 1.0)
    ae, be = pad_cells(c, q1, -1.0, 1.0), pad_cells(c, q2, 1.0, -1.0)
    ee = he - He
    ue, ve = desing(he, ae, c.delta), desing(he, be, c.delta)
    fld = [he, ee, ue, ve]
    # x reconstruction: interior rows, cells -1 .. nx (extended columns 1 .. nx+2)
    rows = slice(2, ny + 2)
    dry = (he[rows, 0:nx + 2] <= c.hdry) | (he[rows, 1:nx + 3] <= c.hdry) | \
          (he[rows, 2:nx + 4] <= c.hdry)
    xE, xW = [], []
    for f, v in enumerate(fld):
        c0, cm, cp = v[rows, 1:nx + 3], v[rows, 0:nx + 2], v[rows, 2:nx + 4]
        s = slope(c, cm, c0, cp)
        if f == 1:
            s = torch.where(dry, torch.zeros_like(s), s)
        xE.append(c0 + 0.5 * s)
        xW.append(c0 - 0.5 * s)
    # y reconstruction: interior columns, cells -1 .. ny (extended rows 1 .. ny+2)
    cols = slice(2, nx + 2)
    dry = (he[0:ny + 2, cols] <= c.hdry) | (he[1:ny + 3, cols] <= c.hdry) | \
          (he[2:ny + 4, cols] <= c.hdry)
    yN, yS = [], []
    for f, v in enumerate(fld):
        c0, cm, cp = v[1:ny + 3, cols], v[0:ny + 2, cols], v[2:ny + 4, cols]
        s = slope(c, cm, c0, cp)
        if f == 1:
            s = torch.where(dry, torch.zeros_like(s), s)
        yN.append(c0 + 0.5 * s)
        yS.append(c0 - 0.5 * s)
    # x faces I = 0 .. nx between cells I-1 (index I) and I (index I+1): normal u, tangential v
    DmX, DpX = pvm(c, xE[0][:, 0:nx + 1], xE[1][:, 0:nx + 1], xE[2][:, 0:nx + 1], xE[3][:, 0:nx + 1],
                   xW[0][:, 1:nx + 2], xW[1][:, 1:nx + 2], xW[2][:, 1:nx + 2], xW[3][:, 1:nx + 2])
    # y faces J = 0 .. ny: normal v, tangential u
    DmY, DpY = pvm(c, yN[0][0:ny + 1], yN[1][0:ny + 1], yN[3][0:ny + 1], yN[2][0:ny + 1],
                   yS[0][1:ny + 2], yS[1][1:ny + 2], yS[3][1:ny + 2], yS[2][1:ny + 2])
    hc = he[2:ny + 2, 2:nx + 2]
    # cell values of the reconstructions (interior cells at index 1 .. n)
    hEx, hWx, uEx, uWx = xE[0][:, 1:nx + 1], xW[0][:, 1:nx + 1], xE[2][:, 1:nx + 1], xW[2][:, 1:nx + 1]
    vEx, vWx = xE[3][:, 1:nx + 1], xW[3][:, 1:nx + 1]
    eEx, eWx = xE[1][:, 1:nx + 1], xW[1][:, 1:nx + 1]
    hNy, hSy, uNy, uSy = yN[0][1:ny + 1], yS[0][1:ny + 1], yN[2][1:ny + 1], yS[2][1:ny + 1]
    vNy, vSy = yN[3][1:ny + 1], yS[3][1:ny + 1]
    eNy, eSy = yN[1][1:ny + 1], yS[1][1:ny + 1]
    Ix0 = hEx * uEx - hWx * uWx
    Ix1 = hEx * uEx * uEx - hWx * uWx * uWx + g * hc * (eEx - eWx)
    Ix2 = hEx * uEx * vEx - hWx * uWx * vWx
    Iy0 = hNy * vNy - hSy * vSy
    Iy1 = hNy * uNy * vNy - hSy * uSy * vSy
    Iy2 = hNy * vNy * vNy - hSy * vSy * vSy + g * hc * (eNy - eSy)
    mx = [d[:, 1:nx + 1] for d in DmX]   # east face D^-
    px = [d[:, 0:nx] for d in DpX]       # west face D^+
    my = [d[1:ny + 1] for d in DmY]      # north face D^-
    py = [d[0:ny] for d in DpY]          # south face D^+
    rx, ry = dt / c.dx, dt / c.dy
    hn = hc - rx * (mx[0] + px[0] + Ix0) - ry * (my[0] + py[0] + Iy0)
    an = q1 - rx * (mx[1] + px[1] + Ix1) - ry * (my[2] + py[2] + Iy1)
    bn = q2 - rx * (mx[2] + px[2] + Ix2) - ry * (my[1] + py[1] + Iy2)
    neg = hn < 0
    z = torch.zeros_like(hn)
    return torch.where(neg, z, hn), torch.where(neg, z, an), torch.where(neg, z, bn)


def nh_fields(c: Cfg2, H, h):
    """Extended h, s = 2 eta - h and the centred X = dx (2 eta - h)_x, Y (App. A.2) for
    cells -1 .. nx, -1 .. ny (arrays [ny+2][nx+2])."""
    he, He = pad_cells(c, h, 1.0, 1.0), pad_cells(c, H, 1.0, 1.0)
    s = 2.0 * (he - He) - he
    X = 0.5 * (s[1:-1, 2:] - s[1:-1, :-2])
    Y = 0.5 * (s[2:, 1:-1] - s[:-2, 1:-1])
    return he[1:-1, 1:-1], s[1:-1, 1:-1], X, Y


def half_T(c: Cfg2, hx, X, Y, pe, dt):
    """dt T^Hor_N, T^Hor_S, T^Ver_E, T^Ver_W (App. A.2) of cells -1 .. nx, -1 .. ny from the
    extended node pressure pe (nodes -1 .. nx+1); leading batch dimensions allowed."""
    dx, dy = c.dx, c.dy
    pSW, pSE = pe[..., 0:-1, 0:-1], pe[..., 0:-1, 1:]
    pNW, pNE = pe[..., 1:, 0:-1], pe[..., 1:, 1:]
    TN = dt * (-0.5 * hx * (pNE - pNW) / dx - 0.5 * 0.5 * (pNE + pNW) * X / dx)
    TS = dt * (-0.5 * hx * (pSE - pSW) / dx - 0.5 * 0.5 * (pSE + pSW) * X / dx)
    TE = dt * (-0.5 * hx * (pNE - pSE) / dy - 0.5 * 0.5 * (pNE + pSE) * Y / dy)
    TW = dt * (-0.5 * hx * (pNW - pSW) / dy - 0.5 * 0.5 * (pNW + pSW) * Y / dy)
    return TN, TS, TE, TW


def B_nodes(c: Cfg2, hx, s, Q1, Q2, T, twohw):
    """Eqs. (37)-(41) at every node from extended cell arrays (cells -1 .. n); T = None or
    the four dt half-corrections; twohw the 2 h w term."""
    dx, dy = c.dx, c.dy
    a = (slice(None), slice(0, -1), slice(0, -1))
    b = (slice(None), slice(0, -1), slice(1, None))
    d = (slice(None), slice(1, None), slice(0, -1))
    e = (slice(None), slice(1, None), slice(1, None))

    def at(v, k):
        return v[(Ellipsis,) + k[1:]]

    q1E = 0.5 * (at(Q1, e) + at(Q1, b))
    q1W = 0.5 * (at(Q1, d) + at(Q1, a))
    q2N = 0.5 * (at(Q2, e) + at(Q2, d))
    q2S = 0.5 * (at(Q2, b) + at(Q2, a))
    if T is not None:
        TN, TS, TE, TW = T
        q1E = q1E + 0.5 * (at(TS, e) + at(TN, b))
        q1W = q1W + 0.5 * (at(TS, d) + at(TN, a))
        q2N = q2N + 0.5 * (at(TW, e) + at(TE, d))
        q2S = q2S + 0.5 * (at(TW, b) + at(TE, a))
    sE, sW = 0.5 * (at(s, e) + at(s, b)), 0.5 * (at(s, d) + at(s, a))
    sN, sS = 0.5 * (at(s, e) + at(s, d)), 0.5 * (at(s, b) + at(s, a))
    hcn = 0.25 * (at(hx, a) + at(hx, b) + at(hx, d) + at(hx, e))
    divQ = (q1E - q1W) / dx + (q2N - q2S) / dy
    Qx, Qy = 0.5 * (q1E + q1W), 0.5 * (q2N + q2S)
    gx, gy = (sE - sW) / dx, (sN - sS) / dy
    return hcn * divQ - (Qx * gx + Qy * gy) + twohw


def node_depth(hx):
    return 0.25 * (hx[:-1, :-1] + hx[:-1, 1:] + hx[1:, :-1] + hx[1:, 1:])


def nh_matrix(c: Cfg2, hx, s, X, Y, dt):
    """Dense matrix of p -> (8 dx dy / dt) [B(dt T(p), dt p / h) - B(0, 0)] (Sec. 5), from
    the linear map applied to every unit vector."""
    nn = (c.nx + 1) * (c.ny + 1)
    eye = torch.eye(nn, dtype=hx.dtype).reshape(nn, c.ny + 1, c.nx + 1)
    pe = torch.cat([eye[:, :, 1:2], eye, eye[:, :, -2:-1]], 2)
    pe = torch.cat([pe[:, 1:2], pe, pe[:, -2:-1]], 1)
    T = half_T(c, hx, X, Y, pe, dt)
    zero = torch.zeros_like(hx)
    cols = B_nodes(c, hx, s, zero, zero, T, 2.0 * dt * eye)
    return (8.0 * c.dx * c.dy / dt) * cols.reshape(nn, nn).T


def stage(c: Cfg2, H, hb, q1b, q2b, wb, h, q1, q2, w, a, bw, dt):
    """Shu-Osher stage of App. A: U* = a U_base + b (U + dt L(U)), w* = a w_base + b w,
    p from the dense solve, correction with de = b dt (Eq. 36, w += de p / h_c)."""
    ho, ao, bo = hyperbolic(c, H, h, q1, q2, dt)
    ho, ao, bo = a * hb + bw * ho, a * q1b + bw * ao, a * q2b + bw * bo
    wo = a * wb + bw * w
    de = bw * dt
    hx, s, X, Y = nh_fields(c, H, ho)
    Q1, Q2 = pad_cells(c, ao, -1.0, 1.0)[1:-1, 1:-1], pad_cells(c, bo, 1.0, -1.0)[1:-1, 1:-1]
    hcn = node_depth(hx)
    rhs = -(8.0 * c.dx * c.dy / de) * B_nodes(c, hx, s, Q1, Q2, None, 2.0 * hcn * wo)
    M = nh_matrix(c, hx, s, X, Y, de)
    p = torch.linalg.solve(M, rhs.reshape(-1)).reshape(c.ny + 1, c.nx + 1)
    TN, TS, TE, TW = half_T(c, hx, X, Y, pad_nodes(p), de)
    ao = ao + 0.5 * (TN + TS)[1:-1, 1:-1]
    bo = bo + 0.5 * (TE + TW)[1:-1, 1:-1]
    wo = wo + de * p * desing(hcn, torch.ones_like(hcn), c.delta)
    if not c.dry_zero:   # Sec. 4.5 as stated: no truncation at wet/dry fronts
        return ho, ao, bo, wo, p
    wet = ho > c.hdry
    z = torch.zeros_like(ao)
    return ho, torch.where(wet, ao, z), torch.where(wet, bo, z), wo, p


def step(c: Cfg2, H, h, q1, q2, w, dt):
    """TVD-RK2: U1 = P(U^n + dt L(U^n)); U^{n+1} = P_{dt/2}((U^n + U1 + dt L(U1)) / 2)."""
    h1, a1, b1, w1, _ = stage(c, H, h, q1, q2, w, h, q1, q2, w, 0.0, 1.0, dt)
    return stage(c, H, h, q1, q2, w, h1, a1, b1, w1, 0.5, 0.5, dt)


def gauge_misfit(c: Cfg2, H, eta0, q1, q2, dt, nsteps, gauges, target):
    """J = sum over steps n = 1..N and gauges g of (eta_g^n - target[n-1, g])^2, from
    eta0 (h = eta0 + H), at rest in w; gauges: (row, column) pairs."""
    h = eta0 + H
    w = torch.zeros((c.ny + 1, c.nx + 1), dtype=H.dtype)
    gi = torch.as_tensor([gg[0] for gg in gauges])
    gj = torch.as_tensor([gg[1] for gg in gauges])
    J = torch.zeros((), dtype=H.dtype)
    for n in range(nsteps):
        h, q1, q2, w, _ = step(c, H, h, q1, q2, w, dt)
        eta = h - H
        J = J + ((eta[gi, gj] - target[n]) ** 2).sum()
    return J


def gradient(c: Cfg2, H, eta0, q1, q2, dt, nsteps, gauges, target):
    """(J, dJ/dH, dJ/deta0) by reverse-mode differentiation of the restated step."""
    H = torch.as_tensor(H, dtype=torch.float64).clone().requires_grad_(True)
    e0 = torch.as_tensor(eta0, dtype=torch.float64).clone().requires_grad_(True)
    q1 = torch.as_tensor(q1, dtype=torch.float64)
    q2 = torch.as_tensor(q2, dtype=torch.float64)
    tg = torch.as_tensor(target, dtype=torch.float64)
    J = gauge_misfit(c, H, e0, q1, q2, dt, nsteps, gauges, tg)
    gH, ge = torch.autograd.grad(J, (H, e0))
    return float(J.detach()), gH.numpy(), ge.numpy()
