// nh_adjoint.cu -- hand-written reverse-mode (adjoint) kernels of the 2D step.
//
// The paper has no adjoint; these kernels differentiate the discrete step that
// nh_kernels.cu computes (Eq. 30 hyperbolic update with MUSCL-minmod and the PVM-HLL
// fluctuations of Eqs. 18-19, the pressure system of Eqs. 36-41 with its solve, and the
// correction), one Runge-Kutta stage at a time in reverse order.  With U* the state after
// the hyperbolic step and the combination, p = M(eta*, H)^-1 b(eta*, H, q*, w*), and the
// corrected state U = (eta*, q* + de T(p), w* + de p / h_c):
//
//   p_bar   = (dU/dp)^T U_bar                              (k_adj_pbar, gather form)
//   lambda  = M^-T p_bar                                   (transposed solve)
//   theta_bar += lambda^T d(b - M p)/d theta + (dU/d theta)^T U_bar
//             for theta = eta*, H, q*, w*                  (k_adj_node, k_adj_cell_corr)
//   U_in_bar += b (U*_bar + (d L / d U)^T U*_bar dt)       (k_adj_face, k_adj_cell_hyp)
//
// The node and face adjoints scatter into cell accumulators with atomics; their order of
// summation is not fixed, so FP32 results vary in the last bits from run to run.
// Differentiability: minmod, min / max and |.| are differentiated along the branch the
// forward takes; friction, breaking and depth clamps are not part of the adjoint (the
// entry point rejects friction and breaking; dry cells follow the forward's branches).
#include "nh_device.cuh"

#include <cuda_runtime.h>

namespace nh {
namespace {

using namespace dev;

// d/dh of desing(h, 1) = sqrt(2) h / sqrt(h^4 + max(h^4, d4)).
template <typename T>
__device__ __forceinline__ T desing1_dh(T h, T d4)
{
    const T h2 = h * h, h4 = h2 * h2;
    const bool big = h4 > d4;
    const T D = sqrt(h4 + (big ? h4 : d4));
    const T c = big ? T(4) : T(2);
    return T(1.4142135623730951) / D - T(1.4142135623730951) * h * (c * h2 * h) / (D * D * D);
}

// d/dq of desing(h, q) (it is linear in q).
template <typename T>
__device__ __forceinline__ T desing_dq(T h, T d4)
{
    const T h2 = h * h, h4 = h2 * h2;
    return T(1.4142135623730951) * h / sqrt(h4 + tmax(h4, d4));
}

// minmod branch: 1 returns a, 2 returns b, 0 returns zero (as the forward minmod).
template <typename T>
__device__ __forceinline__ int mm_branch(T a, T b)
{
    if (a > T(0) && b > T(0)) return a < b ? 1 : 2;
    if (a < T(0) && b < T(0)) return a > b ? 1 : 2;
    return 0;
}

template <typename T>
__device__ __forceinline__ void aadd(T* p, T v)
{
    if (v != T(0)) atomicAdd(p, v);
}

// Cell (i, j) under the boundary mapping: linear index and the signs of q1, q2.
struct MapC {
    int k;
    signed char sx, sy;
};
template <typename T>
__device__ __forceinline__ MapC mapc(const Prm<T>& P, int i, int j)
{
    bool rx, ry;
    const int ii = map_cell(i, P.nx, P.bcw, P.bce, rx);
    const int jj = map_cell(j, P.ny, P.bcs, P.bcn, ry);
    MapC m;
    m.k = jj * P.nx + ii;
    m.sx = rx ? -1 : 1;
    m.sy = ry ? -1 : 1;
    return m;
}

// ---------------------------------------------------------------- correction: p_bar

// p_bar at node (I, J): de desing(h_c, 1) w_bar (the w correction) plus the gather of the
// four cells' T-derivatives with their q_bar (Eq. 36).
template <typename T>
__global__ void __launch_bounds__(kThreads)
k_adj_pbar(Prm<T> P, const T* __restrict__ eta, const T* __restrict__ H,
           const T* __restrict__ a1o, const T* __restrict__ a2o, const T* __restrict__ wo,
           T de, T* __restrict__ pbar)
{
    const T d2 = P.delta * P.delta, d4 = d2 * d2;
    const int nxn = P.nx + 1;
    GRID_STRIDE(idx, (long long)(P.nx + 1) * (P.ny + 1))
    {
        const int I = (int)(idx % nxn), J = (int)(idx / nxn);
        T hs = T(0);
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const MapC m = mapc(P, I - 1 + (k & 1), J - 1 + (k >> 1));
            hs += tmax(eta[m.k] + H[m.k], T(0));
        }
        const T hc = T(0.25) * hs;
        T acc = wo[idx] * de * desing(hc, T(1), d4);
        // cells having this node as a corner: (I-1,J-1) NE, (I,J-1) NW, (I-1,J) SE, (I,J) SW
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int i = I - 1 + (k & 1), j = J - 1 + (k >> 1);
            if (i < 0 || j < 0 || i >= P.nx || j >= P.ny) continue;
            const int c = j * P.nx + i;
            const T h = tmax(eta[c] + H[c], T(0));
            if (!(h > P.hdry)) continue;   // dry: q = 0, no dependence on p
            const MapC mw = mapc(P, i - 1, j), me = mapc(P, i + 1, j);
            const MapC ms = mapc(P, i, j - 1), mn = mapc(P, i, j + 1);
            const T X = T(0.5) * ((eta[me.k] - H[me.k]) - (eta[mw.k] - H[mw.k]));
            const T Y = T(0.5) * ((eta[mn.k] - H[mn.k]) - (eta[ms.k] - H[ms.k]));
            const T g1 = T(0.5) * de * a1o[c], g2 = T(0.5) * de * a2o[c];   // TN_bar = TS_bar, TE_bar = TW_bar
            const bool east = (k & 1) == 0;    // node is on the east side of cell c
            const bool north = (k >> 1) == 0;  // node is on the north side of cell c
            // x part (TN if north, TS if south): d/dp_east = (-h/2 - X/4)/dx, west (h/2 - X/4)/dx
            acc += g1 * (east ? (-T(0.5) * h - T(0.25) * X) : (T(0.5) * h - T(0.25) * X)) / P.dx;
            // y part (TE if east, TW if west): d/dp_north = (-h/2 - Y/4)/dy, south (h/2 - Y/4)/dy
            acc += g2 * (north ? (-T(0.5) * h - T(0.25) * Y) : (T(0.5) * h - T(0.25) * Y)) / P.dy;
        }
        pbar[idx] = acc;
    }
}

// ---------------------------------------------------------------- transposed rows

// Rows of M^T in the five-point form (the boundary fold of M moves to the neighbour of the
// boundary node), with the reductions of the assembly: ||b||^2, ||D^-1 b||^2 and the
// Gershgorin radius of the rows of D^-1 M.  D^-1 M^T = (M D^-1)^T is similar to D^-1 M, so
// the interval that holds the spectrum of the forward iteration holds that of the
// transposed one, although the rows of D^-1 M^T need not be diagonally dominant.  The last
// block prepares the solve (asm_finish).
template <typename T>
__global__ void __launch_bounds__(kThreads)
k_transpose(Rows<T> R, const T* __restrict__ b, T* __restrict__ tW, T* __restrict__ tE,
            T* __restrict__ tS, T* __restrict__ tN, double* partials, SolveCtl* ctl,
            double tol2, int max_iter, int kpass)
{
    const int nx = R.nx, ny = R.ny, nxn = nx + 1;
    double acc[3] = {0.0, 0.0, 0.0};
    GRID_STRIDE(idx, (long long)(nx + 1) * (ny + 1))
    {
        const int I = (int)(idx % nxn), J = (int)(idx / nxn);
        // entry (k, m) of M^T = entry (m, k) of M: the coefficient of node k in row m
        auto fold_x = [&](int Im) {   // coefficient of (I, J) in row (Im, J) along x
            const size_t m = (size_t)J * nxn + Im;
            T v = T(0);
            if (map_node(Im - 1, nx) == I) v += R.cW[m];
            if (map_node(Im + 1, nx) == I) v += R.cE[m];
            return v;
        };
        auto fold_y = [&](int Jm) {
            const size_t m = (size_t)Jm * nxn + I;
            T v = T(0);
            if (map_node(Jm - 1, ny) == J) v += R.cS[m];
            if (map_node(Jm + 1, ny) == J) v += R.cN[m];
            return v;
        };
        // west neighbour column of row k in M^T = coefficient of k in row (I-1); at I = 0 the
        // only x neighbour is I+1 (east), so west stays 0 there; symmetric at I = nx.
        const T w = I > 0 ? fold_x(I - 1) : T(0);
        const T e = I < nx ? fold_x(I + 1) : T(0);
        const T s = J > 0 ? fold_y(J - 1) : T(0);
        const T n = J < ny ? fold_y(J + 1) : T(0);
        tW[idx] = w; tE[idx] = e; tS[idx] = s; tN[idx] = n;
        const T dC = R.cC[idx];
        const T id = T(1) / fabs(dC);
        const T bv = b[idx];
        acc[0] += (double)bv * (double)bv;
        acc[1] += (double)(bv * id) * (double)(bv * id);
        acc[2] = fmax(acc[2], (double)((fabs(R.cW[idx]) + fabs(R.cE[idx]) + fabs(R.cS[idx]) +
                                        fabs(R.cN[idx])) * id));
    }
    if (grid_reduce<3, 4u>(acc, partials, &ctl->counter) && threadIdx.x == 0)
        asm_finish(ctl, acc, tol2, max_iter, kpass, 1);
}

// ---------------------------------------------------------------- assembly / solve adjoint

struct AdjNodeArgs {
    double scale;   // 8 dx dy / de
    double de;
    double a, b;    // Shu-Osher weights of the stage (w* = a w_base + b w_in)
    int assign_in;  // 1: w_in_bar = b w*_bar; 0: w_in_bar += b w*_bar
};

// lambda^T d(b - M p)/d theta at node (I, J) for theta = h, s = eta - H, X, Y of the four
// cells around it, their q*, and w*; plus the h_c dependence of the w correction.
// Cell terms go to the accumulators Hh (depth), Sb (s), A1, A2 (q*) with atomics.
template <typename T>
__global__ void __launch_bounds__(kThreads)
k_adj_node(Prm<T> P, const T* __restrict__ eta, const T* __restrict__ H,
           const T* __restrict__ q1, const T* __restrict__ q2, const T* __restrict__ ws,
           const T* __restrict__ p, const T* __restrict__ lam, const T* __restrict__ wo,
           AdjNodeArgs G, T* __restrict__ Hh, T* __restrict__ Sb, T* __restrict__ A1,
           T* __restrict__ A2, T* __restrict__ w_in_bar, T* __restrict__ w_base_bar)
{
    const T d2 = P.delta * P.delta, d4 = d2 * d2;
    const int nx = P.nx, ny = P.ny, nxn = nx + 1;
    const T inv2dx = T(1) / (T(2) * P.dx), inv2dy = T(1) / (T(2) * P.dy);
    const T rxl = P.dy / P.dx, ryl = P.dx / P.dy;
    const T scale = (T)G.scale, de = (T)G.de;
    GRID_STRIDE(idx, (long long)(nx + 1) * (ny + 1))
    {
        const int I = (int)(idx % nxn), J = (int)(idx / nxn);
        // cells a (I-1,J-1), b (I,J-1), d (I-1,J), e (I,J)
        const int ci[4] = {I - 1, I, I - 1, I}, cj[4] = {J - 1, J - 1, J, J};
        MapC m[4];
        T hh[4], ss[4], X[4], Y[4], Q1[4], Q2[4];
        bool wet[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            m[k] = mapc(P, ci[k], cj[k]);
            const T e = eta[m[k].k], Hm = H[m[k].k];
            wet[k] = e + Hm > T(0);
            hh[k] = tmax(e + Hm, T(0));
            ss[k] = e - Hm;
            const MapC mw = mapc(P, ci[k] - 1, cj[k]), me = mapc(P, ci[k] + 1, cj[k]);
            const MapC ms = mapc(P, ci[k], cj[k] - 1), mn = mapc(P, ci[k], cj[k] + 1);
            X[k] = T(0.5) * ((eta[me.k] - H[me.k]) - (eta[mw.k] - H[mw.k]));
            Y[k] = T(0.5) * ((eta[mn.k] - H[mn.k]) - (eta[ms.k] - H[ms.k]));
            Q1[k] = m[k].sx < 0 ? -q1[m[k].k] : q1[m[k].k];
            Q2[k] = m[k].sy < 0 ? -q2[m[k].k] : q2[m[k].k];
        }
        const T ha = hh[0], hb = hh[1], hd = hh[2], he = hh[3];
        const T hc = T(0.25) * (ha + hb + hd + he);
        const T Xi = T(0.5) * (ss[3] + ss[1]) - T(0.5) * (ss[2] + ss[0]);
        const T Yi = T(0.5) * (ss[2] + ss[3]) - T(0.5) * (ss[0] + ss[1]);
        const T q1E = T(0.5) * (Q1[3] + Q1[1]), q1W = T(0.5) * (Q1[2] + Q1[0]);
        const T q2N = T(0.5) * (Q2[3] + Q2[2]), q2S = T(0.5) * (Q2[1] + Q2[0]);
        const T wv = ws[idx];
        const T apE = (hb + he) + T(0.5) * (X[1] + X[3]), amE = T(0.5) * (X[1] + X[3]) - (hb + he);
        const T apW = (ha + hd) + T(0.5) * (X[0] + X[2]), amW = T(0.5) * (X[0] + X[2]) - (ha + hd);
        const T apN = (hd + he) + T(0.5) * (Y[2] + Y[3]), amN = T(0.5) * (Y[2] + Y[3]) - (hd + he);
        const T apS = (ha + hb) + T(0.5) * (Y[0] + Y[1]), amS = T(0.5) * (Y[0] + Y[1]) - (ha + hb);
        const T bmx = Xi - T(2) * hc, bpx = Xi + T(2) * hc;
        const T bmy = Yi - T(2) * hc, bpy = Yi + T(2) * hc;
        const int Iw = map_node(I - 1, nx), Ie = map_node(I + 1, nx);
        const int Js = map_node(J - 1, ny), Jn = map_node(J + 1, ny);
        const T l = lam[idx];
        const T pC = p[idx], pW = p[(size_t)J * nxn + Iw], pE = p[(size_t)J * nxn + Ie];
        const T pS = p[(size_t)Js * nxn + I], pN = p[(size_t)Jn * nxn + I];
        // G = l (b - M p): partials of the row quantities
        const T gB = -scale * l;   // d G / d Bs (b = -scale Bs)
        const T gvE = -l * pE, gvW = -l * pW, gvN = -l * pN, gvS = -l * pS, gdC = -l * pC;
        T g_bmx = rxl * (apE * gvE + amE * gdC), g_bpx = rxl * (amW * gvW + apW * gdC);
        T g_bmy = ryl * (apN * gvN + amN * gdC), g_bpy = ryl * (amS * gvS + apS * gdC);
        const T g_apE = rxl * bmx * gvE, g_amW = rxl * bpx * gvW;
        const T g_apN = ryl * bmy * gvN, g_amS = ryl * bpy * gvS;
        const T g_amE = rxl * bmx * gdC, g_apW = rxl * bpx * gdC;
        const T g_amN = ryl * bmy * gdC, g_apS = ryl * bpy * gdC;
        // Bs = ((2hc - Xi) q1E - (2hc + Xi) q1W) i2x + ((2hc - Yi) q2N - (2hc + Yi) q2S) i2y + 2 hc w
        T g_hc = gB * (T(2) * (q1E - q1W) * inv2dx + T(2) * (q2N - q2S) * inv2dy + T(2) * wv);
        T g_Xi = gB * (-(q1E + q1W) * inv2dx);
        T g_Yi = gB * (-(q2N + q2S) * inv2dy);
        const T g_q1E = gB * (T(2) * hc - Xi) * inv2dx, g_q1W = -gB * (T(2) * hc + Xi) * inv2dx;
        const T g_q2N = gB * (T(2) * hc - Yi) * inv2dy, g_q2S = -gB * (T(2) * hc + Yi) * inv2dy;
        const T g_w = gB * T(2) * hc;
        // w correction: w = w* + de p desing(hc, 1)
        const T wob = wo[idx];
        g_hc += wob * de * pC * desing1_dh(hc, d4);
        // bmx = Xi - 2hc, bpx = Xi + 2hc, ...
        g_Xi += g_bmx + g_bpx;
        g_Yi += g_bmy + g_bpy;
        g_hc += T(2) * (g_bpx - g_bmx) + T(2) * (g_bpy - g_bmy);
        // per-cell partials: h, X, Y (a, b, d, e = 0, 1, 2, 3)
        T gh[4], gX[4], gY[4], gs[4], gq1[4], gq2[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) { gh[k] = T(0.25) * g_hc; gX[k] = T(0); gY[k] = T(0); }
        // apE = (hb + he) + (Xb + Xe)/2, amE = (Xb + Xe)/2 - (hb + he)
        gh[1] += g_apE - g_amE; gh[3] += g_apE - g_amE;
        gX[1] += T(0.5) * (g_apE + g_amE); gX[3] += T(0.5) * (g_apE + g_amE);
        gh[0] += g_apW - g_amW; gh[2] += g_apW - g_amW;
        gX[0] += T(0.5) * (g_apW + g_amW); gX[2] += T(0.5) * (g_apW + g_amW);
        gh[2] += g_apN - g_amN; gh[3] += g_apN - g_amN;
        gY[2] += T(0.5) * (g_apN + g_amN); gY[3] += T(0.5) * (g_apN + g_amN);
        gh[0] += g_apS - g_amS; gh[1] += g_apS - g_amS;
        gY[0] += T(0.5) * (g_apS + g_amS); gY[1] += T(0.5) * (g_apS + g_amS);
        // Xi = (s_e + s_b)/2 - (s_d + s_a)/2, Yi = (s_d + s_e)/2 - (s_a + s_b)/2
        gs[0] = T(0.5) * (-g_Xi - g_Yi);
        gs[1] = T(0.5) * (g_Xi - g_Yi);
        gs[2] = T(0.5) * (-g_Xi + g_Yi);
        gs[3] = T(0.5) * (g_Xi + g_Yi);
        gq1[0] = T(0.5) * g_q1W; gq1[1] = T(0.5) * g_q1E; gq1[2] = T(0.5) * g_q1W; gq1[3] = T(0.5) * g_q1E;
        gq2[0] = T(0.5) * g_q2S; gq2[1] = T(0.5) * g_q2S; gq2[2] = T(0.5) * g_q2N; gq2[3] = T(0.5) * g_q2N;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            if (wet[k]) aadd(&Hh[m[k].k], gh[k]);
            aadd(&Sb[m[k].k], gs[k]);
            aadd(&A1[m[k].k], m[k].sx < 0 ? -gq1[k] : gq1[k]);
            aadd(&A2[m[k].k], m[k].sy < 0 ? -gq2[k] : gq2[k]);
            if (gX[k] != T(0)) {
                const MapC mw = mapc(P, ci[k] - 1, cj[k]), me = mapc(P, ci[k] + 1, cj[k]);
                aadd(&Sb[me.k], T(0.5) * gX[k]);
                aadd(&Sb[mw.k], -T(0.5) * gX[k]);
            }
            if (gY[k] != T(0)) {
                const MapC ms = mapc(P, ci[k], cj[k] - 1), mn = mapc(P, ci[k], cj[k] + 1);
                aadd(&Sb[mn.k], T(0.5) * gY[k]);
                aadd(&Sb[ms.k], -T(0.5) * gY[k]);
            }
        }
        // w* = a w_base + b w_in; w = w* + ... so w*_bar = w_bar + g_w
        const T wsb = wob + g_w;
        const T bw = (T)G.b, aw = (T)G.a;
        if (G.assign_in) w_in_bar[idx] = bw * wsb;
        else w_in_bar[idx] += bw * wsb;
        if (aw != T(0)) w_base_bar[idx] += aw * wsb;
    }
}

// Correction terms of the cells (Eq. 36): the T-derivatives with respect to h, X, Y of the
// cell with its q_bar, and the identity parts eta = eta*, q = q* + ...
template <typename T>
__global__ void __launch_bounds__(kThreads)
k_adj_cell_corr(Prm<T> P, const T* __restrict__ eta, const T* __restrict__ H,
                const T* __restrict__ p, const T* __restrict__ eo_bar,
                const T* __restrict__ a1o, const T* __restrict__ a2o, T de,
                T* __restrict__ Es, T* __restrict__ Hh, T* __restrict__ Sb, T* __restrict__ A1,
                T* __restrict__ A2)
{
    const int nxn = P.nx + 1;
    GRID_STRIDE(idx, (long long)P.nx * P.ny)
    {
        const int i = (int)(idx % P.nx), j = (int)(idx / P.nx);
        Es[idx] += eo_bar[idx];
        const T e = eta[idx], Hc = H[idx];
        const T h = tmax(e + Hc, T(0));
        if (!(h > P.hdry)) continue;   // dry: q = 0 whatever q*, p
        const T ab = a1o[idx], bb = a2o[idx];
        A1[idx] += ab;
        A2[idx] += bb;
        const T pSW = p[(size_t)j * nxn + i], pSE = p[(size_t)j * nxn + i + 1];
        const T pNW = p[(size_t)(j + 1) * nxn + i], pNE = p[(size_t)(j + 1) * nxn + i + 1];
        const T g1 = T(0.5) * de * ab, g2 = T(0.5) * de * bb;
        const T gh = g1 * (-T(0.5) * (pNE - pNW) - T(0.5) * (pSE - pSW)) / P.dx +
                     g2 * (-T(0.5) * (pNE - pSE) - T(0.5) * (pNW - pSW)) / P.dy;
        const T gX = g1 * (-T(0.25) * (pNE + pNW) - T(0.25) * (pSE + pSW)) / P.dx;
        const T gY = g2 * (-T(0.25) * (pNE + pSE) - T(0.25) * (pNW + pSW)) / P.dy;
        if (e + Hc > T(0)) Hh[idx] += gh;
        const MapC mw = mapc(P, i - 1, j), me = mapc(P, i + 1, j);
        const MapC ms = mapc(P, i, j - 1), mn = mapc(P, i, j + 1);
        aadd(&Sb[me.k], T(0.5) * gX);
        aadd(&Sb[mw.k], -T(0.5) * gX);
        aadd(&Sb[mn.k], T(0.5) * gY);
        aadd(&Sb[ms.k], -T(0.5) * gY);
    }
}

// eta*_bar = eta_bar + h_bar + s_bar; H_bar += h_bar - s_bar (h = eta + H, s = eta - H).
template <typename T>
__global__ void __launch_bounds__(kThreads)
k_adj_combine(long long n, T* __restrict__ Es, const T* __restrict__ Hh,
              const T* __restrict__ Sb, T* __restrict__ Hbar)
{
    GRID_STRIDE(idx, n)
    {
        const T h = Hh[idx], s = Sb[idx];
        Es[idx] += h + s;
        Hbar[idx] += h - s;
    }
}

// ---------------------------------------------------------------- hyperbolic adjoint

template <typename T>
struct FaceIn {
    T h[4], e[4], un[4], ut[4];   // cells m, l, r, p along the normal
};

// Reverse of one face: from the adjoints oLb, oRb of the two per-face outputs (normal
// frame) to the adjoints of (h, e, u_n, u_t) of the four cells.  Recomputes the forward.
// frozen != 0: the reconstruction's derivative is that of phi (x_p - x_m)/2 with the
// limiter ratio phi = slope / ((x_p - x_m)/2) held at its value (a linearisation that
// keeps the limiter's damping of grid-scale perturbations); 0: the exact derivative of
// the branch minmod takes.
template <typename T>
__device__ __forceinline__ void face_adjoint(const FaceIn<T>& c, T g, T hdry, const T oLb[3],
                                             const T oRb[3], int frozen, FaceIn<T>& gb)
{
#pragma unroll
    for (int k = 0; k < 4; ++k) { gb.h[k] = T(0); gb.e[k] = T(0); gb.un[k] = T(0); gb.ut[k] = T(0); }
    // ---- forward: reconstruction
    const int bLh = mm_branch(c.h[1] - c.h[0], c.h[2] - c.h[1]);
    const int bLu = mm_branch(c.un[1] - c.un[0], c.un[2] - c.un[1]);
    const int bLt = mm_branch(c.ut[1] - c.ut[0], c.ut[2] - c.ut[1]);
    const bool dL = c.h[0] <= hdry || c.h[1] <= hdry || c.h[2] <= hdry;
    const int bLe = dL ? 0 : mm_branch(c.e[1] - c.e[0], c.e[2] - c.e[1]);
    const int bRh = mm_branch(c.h[2] - c.h[1], c.h[3] - c.h[2]);
    const int bRu = mm_branch(c.un[2] - c.un[1], c.un[3] - c.un[2]);
    const int bRt = mm_branch(c.ut[2] - c.ut[1], c.ut[3] - c.ut[2]);
    const bool dR = c.h[1] <= hdry || c.h[2] <= hdry || c.h[3] <= hdry;
    const int bRe = dR ? 0 : mm_branch(c.e[2] - c.e[1], c.e[3] - c.e[2]);
    auto slope = [](int br, T a, T b) { return br == 1 ? a : (br == 2 ? b : T(0)); };
    const T hL = c.h[1] + T(0.5) * slope(bLh, c.h[1] - c.h[0], c.h[2] - c.h[1]);
    const T eL = c.e[1] + T(0.5) * slope(bLe, c.e[1] - c.e[0], c.e[2] - c.e[1]);
    const T nL = c.un[1] + T(0.5) * slope(bLu, c.un[1] - c.un[0], c.un[2] - c.un[1]);
    const T tL = c.ut[1] + T(0.5) * slope(bLt, c.ut[1] - c.ut[0], c.ut[2] - c.ut[1]);
    const T hR = c.h[2] - T(0.5) * slope(bRh, c.h[2] - c.h[1], c.h[3] - c.h[2]);
    const T eR = c.e[2] - T(0.5) * slope(bRe, c.e[2] - c.e[1], c.e[3] - c.e[2]);
    const T nR = c.un[2] - T(0.5) * slope(bRu, c.un[2] - c.un[1], c.un[3] - c.un[2]);
    const T tR = c.ut[2] - T(0.5) * slope(bRt, c.ut[2] - c.ut[1], c.ut[3] - c.ut[2]);
    // ---- forward: PVM (as pvm())
    const T qnL = hL * nL, qnR = hR * nR, qtL = hL * tL, qtR = hR * tR;
    const T hb = T(0.5) * (hL + hR);
    const T sL = qsqrt(hL), sR = qsqrt(hR), ss = sL + sR;
    const bool ssp = ss > T(0);
    const T ub = ssp ? qdiv(nL * sL + nR * sR, ss) : T(0);
    const T sg = qsqrt(g);
    const T cb = qsqrt(g * hb), cL = sg * sL, cR = sg * sR;
    const T sl1 = ub - cb, sl2 = nL - cL;
    const bool slb = sl1 < sl2;
    const T SL = slb ? sl1 : sl2;
    const T sr1 = ub + cb, sr2 = nR + cR;
    const bool srb = sr1 > sr2;
    const T SR = srb ? sr1 : sr2;
    T de = eR - eL;
    bool dz = false;
    if (hR <= hdry && (eR - hR) >= eL) dz = true;
    if (hL <= hdry && (eL - hL) >= eR) dz = true;
    if (dz) de = T(0);
    const T span = SR - SL;
    // adjoints of the reconstructed states
    T hLb = T(0), eLb = T(0), nLb = T(0), tLb = T(0), hRb = T(0), eRb = T(0), nRb = T(0), tRb = T(0);
    if (span > T(0)) {
        const T aSL = fabs(SL), aSR = fabs(SR);
        const T sgL = SL > T(0) ? T(1) : (SL < T(0) ? T(-1) : T(0));
        const T sgR = SR > T(0) ? T(1) : (SR < T(0) ? T(-1) : T(0));
        const T isp = qdiv(T(1), span);
        const T a0 = (SR * aSL - SL * aSR) * isp;
        const T a1 = (aSR - aSL) * isp;
        const T R0 = qnR - qnL;
        const T R1 = qnR * nR - qnL * nL + g * hb * de;
        const T R2 = qnR * tR - qnL * tL;
        const T V2 = qtR - qtL;
        const T dm0 = oLb[0], dm1 = oLb[1], dm2 = oLb[2];
        const T dp0 = oRb[0], dp1 = oRb[1], dp2 = oRb[2];
        T R0b = T(0.5) * (T(1) - a1) * dm0 + T(0.5) * (T(1) + a1) * dp0 - T(0.5) * a0 * dm1 + T(0.5) * a0 * dp1;
        const T R1b = T(0.5) * (T(1) - a1) * dm1 + T(0.5) * (T(1) + a1) * dp1;
        const T R2b = T(0.5) * (T(1) - a1) * dm2 + T(0.5) * (T(1) + a1) * dp2;
        const T V2b = T(0.5) * a0 * (dp2 - dm2);
        T deb = T(0.5) * a0 * (dp0 - dm0);
        const T a1b = T(0.5) * (R0 * (dp0 - dm0) + R1 * (dp1 - dm1) + R2 * (dp2 - dm2));
        const T a0b = T(0.5) * (de * (dp0 - dm0) + R0 * (dp1 - dm1) + V2 * (dp2 - dm2));
        // R1 = qnR nR - qnL nL + g hb de
        T qnRb = nR * R1b + R0b + tR * R2b, qnLb = -nL * R1b - R0b - tL * R2b;
        nRb += qnR * R1b; nLb -= qnL * R1b;
        T hbb = g * de * R1b;
        deb += g * hb * R1b;
        tRb += qnR * R2b; tLb -= qnL * R2b;
        const T qtRb = V2b, qtLb = -V2b;
        if (!dz) { eRb += deb; eLb -= deb; }
        // a0, a1 as functions of SL, SR
        const T SRb = a1b * (sgR - a1) / span + a0b * (aSL - SL * sgR - a0) / span;
        const T SLb = a1b * (a1 - sgL) / span + a0b * (SR * sgL - aSR + a0) / span;
        T ubb = T(0), cbb = T(0), cLb = T(0), cRb = T(0);
        if (slb) { ubb += SLb; cbb -= SLb; } else { nLb += SLb; cLb -= SLb; }
        if (srb) { ubb += SRb; cbb += SRb; } else { nRb += SRb; cRb += SRb; }
        if (sL > T(0)) hLb += cLb * sg / (T(2) * sL);
        if (sR > T(0)) hRb += cRb * sg / (T(2) * sR);
        if (cb > T(0)) hbb += cbb * g / (T(2) * cb);
        if (ssp) {
            nLb += ubb * sL / ss;
            nRb += ubb * sR / ss;
            const T sLb = ubb * (nL - ub) / ss, sRb = ubb * (nR - ub) / ss;
            if (sL > T(0)) hLb += sLb / (T(2) * sL);
            if (sR > T(0)) hRb += sRb / (T(2) * sR);
        }
        hLb += T(0.5) * hbb; hRb += T(0.5) * hbb;
        hLb += nL * qnLb + tL * qtLb; nLb += hL * qnLb; tLb += hL * qtLb;
        hRb += nR * qnRb + tR * qtRb; nRb += hR * qnRb; tRb += hR * qtRb;
    }
    // direct terms: oL = Dm + (qL, qL nL + g h_l eL, qL tL), oR = Dp - (qR, qR nR + g h_r eR, qR tR)
    {
        const T qL = hL * nL, qR = hR * nR;
        const T qLb = oLb[0] + nL * oLb[1] + tL * oLb[2];
        nLb += qL * oLb[1];
        tLb += qL * oLb[2];
        gb.h[1] += g * eL * oLb[1];
        eLb += g * c.h[1] * oLb[1];
        hLb += nL * qLb; nLb += hL * qLb;
        const T qRb = -oRb[0] - nR * oRb[1] - tR * oRb[2];
        nRb -= qR * oRb[1];
        tRb -= qR * oRb[2];
        gb.h[2] -= g * eR * oRb[1];
        eRb -= g * c.h[2] * oRb[1];
        hRb += nR * qRb; nRb += hR * qRb;
    }
    // ---- reconstruction reverse
    // slope = minmod(x0 - xm, xp - x0) of the values vm, v0, vp; sb its adjoint
    auto back = [&](int br, T vm, T v0, T vp, T sb, T& xm, T& x0, T& xp) {
        if (frozen) {
            const T s = slope(br, v0 - vm, vp - v0), cc = T(0.5) * (vp - vm);
            if (s != T(0) && cc != T(0)) {
                const T ph = s / cc;
                xp += T(0.5) * ph * sb;
                xm -= T(0.5) * ph * sb;
            }
        } else if (br == 1) { x0 += sb; xm -= sb; }
        else if (br == 2) { xp += sb; x0 -= sb; }
    };
    gb.h[1] += hLb; back(bLh, c.h[0], c.h[1], c.h[2], T(0.5) * hLb, gb.h[0], gb.h[1], gb.h[2]);
    gb.e[1] += eLb; back(bLe, c.e[0], c.e[1], c.e[2], T(0.5) * eLb, gb.e[0], gb.e[1], gb.e[2]);
    gb.un[1] += nLb; back(bLu, c.un[0], c.un[1], c.un[2], T(0.5) * nLb, gb.un[0], gb.un[1], gb.un[2]);
    gb.ut[1] += tLb; back(bLt, c.ut[0], c.ut[1], c.ut[2], T(0.5) * tLb, gb.ut[0], gb.ut[1], gb.ut[2]);
    gb.h[2] += hRb; back(bRh, c.h[1], c.h[2], c.h[3], -T(0.5) * hRb, gb.h[1], gb.h[2], gb.h[3]);
    gb.e[2] += eRb; back(bRe, c.e[1], c.e[2], c.e[3], -T(0.5) * eRb, gb.e[1], gb.e[2], gb.e[3]);
    gb.un[2] += nRb; back(bRu, c.un[1], c.un[2], c.un[3], -T(0.5) * nRb, gb.un[1], gb.un[2], gb.un[3]);
    gb.ut[2] += tRb; back(bRt, c.ut[1], c.ut[2], c.ut[3], -T(0.5) * tRb, gb.ut[1], gb.ut[2], gb.ut[3]);
}

// All faces (x faces first, then y faces): face reverse with the outputs' adjoints
// -dt/dx b U*_bar of the two cells it updates; scatter to the four cells' (h, e, u, v).
template <typename T>
__global__ void __launch_bounds__(kThreads)
k_adj_face(Prm<T> P, const T* __restrict__ eta, const T* __restrict__ q1,
           const T* __restrict__ q2, const T* __restrict__ H, const T* __restrict__ Es,
           const T* __restrict__ A1, const T* __restrict__ A2, T bfac, T dt, int frozen,
           T* __restrict__ Gh, T* __restrict__ Ge, T* __restrict__ Gu, T* __restrict__ Gv)
{
    const T d2 = P.delta * P.delta, d4 = d2 * d2;
    const int nx = P.nx, ny = P.ny;
    const long long nfx = (long long)(nx + 1) * ny, nfy = (long long)nx * (ny + 1);
    GRID_STRIDE(f, nfx + nfy)
    {
        const bool xf = f < nfx;
        int i, j;   // x face: between cells (i-1, j), (i, j); y face: (i, j-1), (i, j)
        if (xf) { i = (int)(f % (nx + 1)); j = (int)(f / (nx + 1)); }
        else { const long long g2 = f - nfx; i = (int)(g2 % nx); j = (int)(g2 / nx); }
        FaceIn<T> c;
        MapC m[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int ci = xf ? i - 2 + k : i, cj = xf ? j : j - 2 + k;
            m[k] = mapc(P, ci, cj);
            const T e = eta[m[k].k];
            const T h = tmax(e + H[m[k].k], T(0));
            const T a = m[k].sx < 0 ? -q1[m[k].k] : q1[m[k].k];
            const T b = m[k].sy < 0 ? -q2[m[k].k] : q2[m[k].k];
            c.h[k] = h; c.e[k] = e;
            c.un[k] = desing(h, xf ? a : b, d4);
            c.ut[k] = desing(h, xf ? b : a, d4);
        }
        // outputs: left cell (index 1) uses this face as its east / north face, right cell
        // (index 2) as its west / south face; ghost cells have no update
        const T r = -(xf ? dt / P.dx : dt / P.dy) * bfac;
        T oL[3] = {T(0), T(0), T(0)}, oR[3] = {T(0), T(0), T(0)};
        const bool lreal = xf ? i - 1 >= 0 : j - 1 >= 0;
        const bool rreal = xf ? i < nx : j < ny;
        if (lreal) {
            const int k = m[1].k;
            oL[0] = r * Es[k];
            oL[1] = r * (xf ? A1[k] : A2[k]);
            oL[2] = r * (xf ? A2[k] : A1[k]);
        }
        if (rreal) {
            const int k = m[2].k;
            oR[0] = r * Es[k];
            oR[1] = r * (xf ? A1[k] : A2[k]);
            oR[2] = r * (xf ? A2[k] : A1[k]);
        }
        if (!lreal && !rreal) continue;
        FaceIn<T> gb;
        face_adjoint(c, P.g, P.hdry, oL, oR, frozen, gb);
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int ck = m[k].k;
            aadd(&Gh[ck], gb.h[k]);
            aadd(&Ge[ck], gb.e[k]);
            const T ub = xf ? gb.un[k] : gb.ut[k], vb = xf ? gb.ut[k] : gb.un[k];
            aadd(&Gu[ck], m[k].sx < 0 ? -ub : ub);
            aadd(&Gv[ck], m[k].sy < 0 ? -vb : vb);
        }
    }
}

// Cells: U_in_bar (=, or +=) b U*_bar + face terms through h = eta + H, u = desing(h, q1),
// v = desing(h, q2); U_base_bar += a U*_bar; H_bar += the depth terms.
template <typename T>
__global__ void __launch_bounds__(kThreads)
k_adj_cell_hyp(Prm<T> P, const T* __restrict__ eta, const T* __restrict__ q1,
               const T* __restrict__ q2, const T* __restrict__ H, const T* __restrict__ Es,
               const T* __restrict__ A1, const T* __restrict__ A2, const T* __restrict__ Gh,
               const T* __restrict__ Ge, const T* __restrict__ Gu, const T* __restrict__ Gv,
               T a, T b, int assign_in, T* __restrict__ ein_b, T* __restrict__ a1in_b,
               T* __restrict__ a2in_b, T* __restrict__ eb_b, T* __restrict__ a1b_b,
               T* __restrict__ a2b_b, T* __restrict__ Hbar)
{
    const T d2 = P.delta * P.delta, d4 = d2 * d2;
    GRID_STRIDE(idx, (long long)P.nx * P.ny)
    {
        const T e = eta[idx], Hc = H[idx];
        const T h = tmax(e + Hc, T(0));
        const T dq = desing_dq(h, d4), dh = desing1_dh(h, d4);
        const T gu = Gu[idx], gv = Gv[idx];
        T hb = Gh[idx] + gu * q1[idx] * dh + gv * q2[idx] * dh;
        if (!(e + Hc > T(0))) hb = T(0);
        const T eb = b * Es[idx] + Ge[idx] + hb;
        const T ab = b * A1[idx] + gu * dq;
        const T bb = b * A2[idx] + gv * dq;
        if (assign_in) { ein_b[idx] = eb; a1in_b[idx] = ab; a2in_b[idx] = bb; }
        else { ein_b[idx] += eb; a1in_b[idx] += ab; a2in_b[idx] += bb; }
        if (a != T(0)) {
            eb_b[idx] += a * Es[idx];
            a1b_b[idx] += a * A1[idx];
            a2b_b[idx] += a * A2[idx];
        }
        Hbar[idx] += hb;
    }
}

}  // namespace

// ---------------------------------------------------------------- launchers

template <typename T>
void launch_adj_pbar(const Prm<T>& P, const Launch& L, const T* eta, const T* H, const T* a1o,
                     const T* a2o, const T* wo, T de, T* pbar)
{
    k_adj_pbar<T><<<L.nblk, kThreads, 0, L.s>>>(P, eta, H, a1o, a2o, wo, de, pbar);
}

template <typename T>
void launch_transpose(const Prm<T>& P, const Launch& L, const Bufs<T>& B, const T* b, T* tW,
                      T* tE, T* tS, T* tN, double tol2, int max_iter, int kpass)
{
    Rows<T> R;
    R.cC = B.cC; R.cW = B.cW; R.cE = B.cE; R.cS = B.cS; R.cN = B.cN;
    R.nx = P.nx; R.ny = P.ny;
    k_transpose<T><<<L.nblk, kThreads, 0, L.s>>>(R, b, tW, tE, tS, tN, B.partials, B.sctl,
                                                 tol2, max_iter, kpass);
}

template <typename T>
void launch_adj_node(const Prm<T>& P, const Launch& L, const T* eta, const T* H, const T* q1,
                     const T* q2, const T* ws, const T* p, const T* lam, const T* wo,
                     double scale, double de, double a, double b, int assign_in, T* Hh, T* Sb,
                     T* A1, T* A2, T* w_in_bar, T* w_base_bar)
{
    AdjNodeArgs G;
    G.scale = scale; G.de = de; G.a = a; G.b = b; G.assign_in = assign_in;
    k_adj_node<T><<<L.nblk, kThreads, 0, L.s>>>(P, eta, H, q1, q2, ws, p, lam, wo, G, Hh, Sb,
                                                A1, A2, w_in_bar, w_base_bar);
}

template <typename T>
void launch_adj_cell_corr(const Prm<T>& P, const Launch& L, const T* eta, const T* H,
                          const T* p, const T* eo_bar, const T* a1o, const T* a2o, T de, T* Es,
                          T* Hh, T* Sb, T* A1, T* A2)
{
    k_adj_cell_corr<T><<<L.nblk, kThreads, 0, L.s>>>(P, eta, H, p, eo_bar, a1o, a2o, de, Es, Hh,
                                                     Sb, A1, A2);
}

template <typename T>
void launch_adj_combine(const Launch& L, long long n, T* Es, const T* Hh, const T* Sb, T* Hbar)
{
    k_adj_combine<T><<<L.nblk, kThreads, 0, L.s>>>(n, Es, Hh, Sb, Hbar);
}

template <typename T>
void launch_adj_face(const Prm<T>& P, const Launch& L, const T* eta, const T* q1, const T* q2,
                     const T* H, const T* Es, const T* A1, const T* A2, T bfac, T dt,
                     int frozen, T* Gh, T* Ge, T* Gu, T* Gv)
{
    k_adj_face<T><<<L.nblk, kThreads, 0, L.s>>>(P, eta, q1, q2, H, Es, A1, A2, bfac, dt, frozen,
                                                Gh, Ge, Gu, Gv);
}

template <typename T>
void launch_adj_cell_hyp(const Prm<T>& P, const Launch& L, const T* eta, const T* q1,
                         const T* q2, const T* H, const T* Es, const T* A1, const T* A2,
                         const T* Gh, const T* Ge, const T* Gu, const T* Gv, T a, T b,
                         int assign_in, T* ein_b, T* a1in_b, T* a2in_b, T* eb_b, T* a1b_b,
                         T* a2b_b, T* Hbar)
{
    k_adj_cell_hyp<T><<<L.nblk, kThreads, 0, L.s>>>(P, eta, q1, q2, H, Es, A1, A2, Gh, Ge, Gu, Gv,
                                                    a, b, assign_in, ein_b, a1in_b, a2in_b, eb_b,
                                                    a1b_b, a2b_b, Hbar);
}

#define NH_ADJ_INSTANTIATE(T)                                                                    \
    template void launch_adj_pbar<T>(const Prm<T>&, const Launch&, const T*, const T*, const T*, \
                                     const T*, const T*, T, T*);                                 \
    template void launch_transpose<T>(const Prm<T>&, const Launch&, const Bufs<T>&, const T*,    \
                                      T*, T*, T*, T*, double, int, int);                         \
    template void launch_adj_node<T>(const Prm<T>&, const Launch&, const T*, const T*, const T*, \
                                     const T*, const T*, const T*, const T*, const T*, double,   \
                                     double, double, double, int, T*, T*, T*, T*, T*, T*);        \
    template void launch_adj_cell_corr<T>(const Prm<T>&, const Launch&, const T*, const T*,      \
                                          const T*, const T*, const T*, const T*, T, T*, T*, T*, \
                                          T*, T*);                                               \
    template void launch_adj_combine<T>(const Launch&, long long, T*, const T*, const T*, T*);   \
    template void launch_adj_face<T>(const Prm<T>&, const Launch&, const T*, const T*, const T*, \
                                     const T*, const T*, const T*, const T*, T, T, int, T*, T*,  \
                                     T*, T*);                                                    \
    template void launch_adj_cell_hyp<T>(const Prm<T>&, const Launch&, const T*, const T*,       \
                                         const T*, const T*, const T*, const T*, const T*,       \
                                         const T*, const T*, const T*, const T*, T, T, int, T*,  \
                                         T*, T*, T*, T*, T*, T*);

NH_ADJ_INSTANTIATE(float)
NH_ADJ_INSTANTIATE(double)

}  // namespace nh
