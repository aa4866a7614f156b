// nh_kernels.cu -- sm_103a kernels of one non-hydrostatic shallow-water time step
// (Escalante, Morales de Luna & Castro, arXiv:1706.04551).
//
// Every kernel is a grid-stride loop over cells or nodes on a grid sized to a multiple of
// the SM count.  Boundary conditions are applied by index mapping at load time (walls:
// mirror, normal discharge odd; outflow: copy), so no ghost arrays exist.  Global sums
// (FP64) use per-block partials and a last-block-done finish, which is deterministic for a
// given grid size.  State precision T is float or double.
#include "nh_internal.h"

#include <cuda_runtime.h>
#include <stdint.h>

namespace nh {
namespace {

constexpr int kThreads = 256;

template <typename T> __device__ __forceinline__ T tmin(T a, T b) { return a < b ? a : b; }
template <typename T> __device__ __forceinline__ T tmax(T a, T b) { return a > b ? a : b; }

// minmod slope limiter of the MUSCL reconstruction (Sec. 4.1).
template <typename T>
__device__ __forceinline__ T minmod(T a, T b)
{
    if (a > T(0) && b > T(0)) return tmin(a, b);
    if (a < T(0) && b < T(0)) return tmax(a, b);
    return T(0);
}

// Desingularised q / h (Sec. 4.5): sqrt(2) h q / sqrt(h^4 + max(h^4, delta^4)); d4 = delta^4.
template <typename T>
__device__ __forceinline__ T desing(T h, T q, T d4)
{
    T h2 = h * h;
    T h4 = h2 * h2;
    return T(1.4142135623730951) * h * q / sqrt(h4 + tmax(h4, d4));
}

// Cell index under the boundary condition of each side: wall = mirror (refl = true),
// outflow = copy of the first interior cell.  Valid for up to n cells outside.
__device__ __forceinline__ int map_cell(int i, int n, int bclo, int bchi, bool& refl)
{
    refl = false;
    if (i < 0) {
        if (bclo == 0) { refl = true; return -1 - i; }
        return 0;
    }
    if (i >= n) {
        if (bchi == 0) { refl = true; return 2 * n - 1 - i; }
        return n - 1;
    }
    return i;
}

// Pressure node index: the outside neighbour of a boundary node mirrors the inside one.
__device__ __forceinline__ int map_node(int I, int n)
{
    return I < 0 ? -I : (I > n ? 2 * n - I : I);
}

template <typename T>
struct St { T h, e, u, v; };

// Cell (i, j) with boundary mapping: depth, free surface and desingularised velocities.
template <typename T>
__device__ __forceinline__ St<T> load_st(const Prm<T>& P, const T* __restrict__ eta,
                                         const T* __restrict__ q1, const T* __restrict__ q2,
                                         const T* __restrict__ H, int i, int j, T d4)
{
    bool rx, ry;
    int ii = map_cell(i, P.nx, P.bcw, P.bce, rx);
    int jj = map_cell(j, P.ny, P.bcs, P.bcn, ry);
    size_t k = (size_t)jj * P.nx + ii;
    T e = eta[k];
    T h = tmax(e + H[k], T(0));
    T a = q1[k], b = q2[k];
    if (rx) a = -a;
    if (ry) b = -b;
    St<T> s;
    s.h = h; s.e = e; s.u = desing(h, a, d4); s.v = desing(h, b, d4);
    return s;
}

// MUSCL-minmod values at the low (W / S) and high (E / N) edges of cell k of a 3-cell
// window c[k-1..k+1]; the free-surface slope is 0 next to dry cells (Sec. 4.1).
template <typename T>
__device__ __forceinline__ void recon(const St<T>* c, int k, T hdry, St<T>& lo, St<T>& hi)
{
    T sh = minmod(c[k].h - c[k - 1].h, c[k + 1].h - c[k].h);
    T su = minmod(c[k].u - c[k - 1].u, c[k + 1].u - c[k].u);
    T sv = minmod(c[k].v - c[k - 1].v, c[k + 1].v - c[k].v);
    bool dry = c[k - 1].h <= hdry || c[k].h <= hdry || c[k + 1].h <= hdry;
    T se = dry ? T(0) : minmod(c[k].e - c[k - 1].e, c[k + 1].e - c[k].e);
    lo.h = c[k].h - T(0.5) * sh; hi.h = c[k].h + T(0.5) * sh;
    lo.e = c[k].e - T(0.5) * se; hi.e = c[k].e + T(0.5) * se;
    lo.u = c[k].u - T(0.5) * su; hi.u = c[k].u + T(0.5) * su;
    lo.v = c[k].v - T(0.5) * sv; hi.v = c[k].v + T(0.5) * sv;
}

// PVM-HLL fluctuations (Eqs. 18-19) at a face in its normal frame from the left state
// (hL, eL, unL, utL) and the right one.  Components: h, normal, tangential discharge.
template <typename T>
__device__ __forceinline__ void pvm(T g, T hdry, T hL, T eL, T unL, T utL, T hR, T eR,
                                    T unR, T utR, T Dm[3], T Dp[3])
{
    T qnL = hL * unL, qnR = hR * unR, qtL = hL * utL, qtR = hR * utR;
    T hb = T(0.5) * (hL + hR);
    T sL = sqrt(hL), sR = sqrt(hR), ss = sL + sR;
    T ub = ss > T(0) ? (unL * sL + unR * sR) / ss : T(0);   // Roe velocity
    T cb = sqrt(g * hb);
    T SL = tmin(ub - cb, unL - sqrt(g * hL));
    T SR = tmax(ub + cb, unR + sqrt(g * hR));
    // emerging bottom (Sec. 4.5): dry side's bed at or above the wet free surface
    T de = eR - eL;
    if (hR <= hdry && (eR - hR) >= eL) de = T(0);
    if (hL <= hdry && (eL - hL) >= eR) de = T(0);
    T span = SR - SL;
    if (!(span > T(0))) {
        Dm[0] = Dm[1] = Dm[2] = Dp[0] = Dp[1] = Dp[2] = T(0);
        return;
    }
    T a0 = (SR * fabs(SL) - SL * fabs(SR)) / span;
    T a1 = (fabs(SR) - fabs(SL)) / span;
    T R0 = qnR - qnL;
    T R1 = qnR * unR - qnL * unL + g * hb * de;
    T R2 = qnR * utR - qnL * utL;
    T V2 = qtR - qtL;
    Dm[0] = T(0.5) * ((T(1) - a1) * R0 - a0 * de);
    Dp[0] = T(0.5) * ((T(1) + a1) * R0 + a0 * de);
    Dm[1] = T(0.5) * ((T(1) - a1) * R1 - a0 * R0);
    Dp[1] = T(0.5) * ((T(1) + a1) * R1 + a0 * R0);
    Dm[2] = T(0.5) * ((T(1) - a1) * R2 - a0 * V2);
    Dp[2] = T(0.5) * ((T(1) + a1) * R2 + a0 * V2);
}

// Breaking eddy viscosity of Eq. (9), stateless switch (active where |d| >= U1, B > 0).
template <typename T>
__device__ __forceinline__ T nu_break(T h, T d, T g, T B1, T hdry)
{
    if (!(h > hdry)) return T(0);
    T U1 = B1 * sqrt(g * h);
    if (!(fabs(d) >= U1) || !(U1 > T(0))) return T(0);
    T B = T(1) - d / U1;
    return B > T(0) ? B * h * fabs(d) : T(0);
}

// ---------------------------------------------------------------- block reductions

__device__ __forceinline__ double warp_sum(double v)
{
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ double warp_max(double v)
{
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// Reduce NV values over the block; value k is a max when bit k of MAXMASK is set, else a
// sum.  Thread 0 gets the result.
template <int NV, unsigned MAXMASK>
__device__ __forceinline__ void block_reduce(double (&v)[NV])
{
    __shared__ double sm[NV][32];
    const int tid = threadIdx.x + blockDim.x * threadIdx.y;
    const int lane = tid & 31, wid = tid >> 5, nw = (blockDim.x * blockDim.y + 31) >> 5;
#pragma unroll
    for (int k = 0; k < NV; ++k) v[k] = ((MAXMASK >> k) & 1u) ? warp_max(v[k]) : warp_sum(v[k]);
    if (lane == 0)
#pragma unroll
        for (int k = 0; k < NV; ++k) sm[k][wid] = v[k];
    __syncthreads();
    if (wid == 0) {
#pragma unroll
        for (int k = 0; k < NV; ++k) {
            const bool mx = (MAXMASK >> k) & 1u;
            double x = lane < nw ? sm[k][lane] : (mx ? -1.0e300 : 0.0);
            v[k] = mx ? warp_max(x) : warp_sum(x);
        }
    }
    __syncthreads();
}

// Write this block's partials, then return true in the last block to finish; that block
// receives the grid totals (fixed summation order) in v.  Blocks are numbered linearly
// over a 1D or 2D grid.
template <int NV, unsigned MAXMASK>
__device__ __forceinline__ bool grid_reduce(double (&v)[NV], double* partials,
                                            unsigned* counter)
{
    block_reduce<NV, MAXMASK>(v);
    const unsigned nblocks = gridDim.x * gridDim.y;
    const unsigned bid = blockIdx.y * gridDim.x + blockIdx.x;
    const unsigned tid = threadIdx.x + blockDim.x * threadIdx.y;
    const unsigned nthr = blockDim.x * blockDim.y;
    __shared__ bool last;
    if (tid == 0) {
#pragma unroll
        for (int k = 0; k < NV; ++k) partials[(size_t)bid * NV + k] = v[k];
        __threadfence();
        last = atomicAdd(counter, 1u) == nblocks - 1;
    }
    __syncthreads();
    if (!last) return false;
    __threadfence();
    double acc[NV];
#pragma unroll
    for (int k = 0; k < NV; ++k) acc[k] = ((MAXMASK >> k) & 1u) ? -1.0e300 : 0.0;
    for (unsigned bb = tid; bb < nblocks; bb += nthr)
#pragma unroll
        for (int k = 0; k < NV; ++k) {
            double x = __ldcg(partials + (size_t)bb * NV + k);
            acc[k] = ((MAXMASK >> k) & 1u) ? fmax(acc[k], x) : acc[k] + x;
        }
    block_reduce<NV, MAXMASK>(acc);
#pragma unroll
    for (int k = 0; k < NV; ++k) v[k] = acc[k];
    if (tid == 0) *counter = 0u;
    return true;
}

// Block partial of (sum, max) in FP32 (a few thousand terms per block), written as FP64
// partials; the last block finishes in FP64 like grid_reduce.
__device__ __forceinline__ bool grid_reduce_sum_max_f(float s, float m, double* partials,
                                                      unsigned* counter, double out[2])
{
    __shared__ float fs[32], fm[32];
    const int tid = threadIdx.x + blockDim.x * threadIdx.y;
    const int lane = tid & 31, wid = tid >> 5, nw = (blockDim.x * blockDim.y + 31) >> 5;
    for (int o = 16; o > 0; o >>= 1) {
        s += __shfl_xor_sync(0xffffffffu, s, o);
        m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    }
    if (lane == 0) { fs[wid] = s; fm[wid] = m; }
    __syncthreads();
    double v[2] = {0.0, 0.0};
    if (wid == 0) {
        float a = lane < nw ? fs[lane] : 0.f, b = lane < nw ? fm[lane] : 0.f;
        for (int o = 16; o > 0; o >>= 1) {
            a += __shfl_xor_sync(0xffffffffu, a, o);
            b = fmaxf(b, __shfl_xor_sync(0xffffffffu, b, o));
        }
        v[0] = a; v[1] = b;
    }
    const unsigned nblocks = gridDim.x * gridDim.y;
    const unsigned bid = blockIdx.y * gridDim.x + blockIdx.x;
    const unsigned nthr = blockDim.x * blockDim.y;
    __shared__ bool last;
    if (tid == 0) {
        partials[(size_t)bid * 2] = v[0];
        partials[(size_t)bid * 2 + 1] = v[1];
        __threadfence();
        last = atomicAdd(counter, 1u) == nblocks - 1;
    }
    __syncthreads();
    if (!last) return false;
    __threadfence();
    double acc[2] = {0.0, 0.0};
    for (unsigned bb = tid; bb < nblocks; bb += nthr) {
        acc[0] += __ldcg(partials + (size_t)bb * 2);
        acc[1] = fmax(acc[1], __ldcg(partials + (size_t)bb * 2 + 1));
    }
    block_reduce<2, 2u>(acc);
    out[0] = acc[0];
    out[1] = acc[1];
    if (tid == 0) *counter = 0u;
    return true;
}

#define GRID_STRIDE(idx, n) \
    for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < (long long)(n); \
         idx += (long long)gridDim.x * blockDim.x)

// ================================================================ 2D kernels

// Hyperbolic update of one cell (Eq. 30; reconstruction Sec. 4.1; Eqs. 18-19 per face in
// its normal frame), semi-implicit Manning friction, depth clamp, then the Shu-Osher
// combination U* = a U_base + b U**.
template <typename T>
__global__ void __launch_bounds__(kThreads)
k_hyp2d(Prm<T> P, const T* __restrict__ eta, const T* __restrict__ q1,
        const T* __restrict__ q2, const T* __restrict__ etab, const T* __restrict__ q1b,
        const T* __restrict__ q2b, const T* __restrict__ H, T a, T b, T dt,
        T* __restrict__ eo, T* __restrict__ q1o, T* __restrict__ q2o, StepCtl* st)
{
    const T d2 = P.delta * P.delta, d4 = d2 * d2;
    const T g = P.g, hdry = P.hdry;
    int nclamp = 0;
    GRID_STRIDE(idx, (long long)P.nx * P.ny)
    {
        const int i = (int)(idx % P.nx), j = (int)(idx / P.nx);
        St<T> cx[5], cy[5];
#pragma unroll
        for (int k = 0; k < 5; ++k) {
            cx[k] = load_st(P, eta, q1, q2, H, i - 2 + k, j, d4);
            cy[k] = load_st(P, eta, q1, q2, H, i, j - 2 + k, d4);
        }
        St<T> xlo[3], xhi[3], ylo[3], yhi[3];
#pragma unroll
        for (int k = 1; k <= 3; ++k) {
            recon(cx, k, hdry, xlo[k - 1], xhi[k - 1]);
            recon(cy, k, hdry, ylo[k - 1], yhi[k - 1]);
        }
        T DpW[3], DmW[3], DmE[3], DpE[3], DpS[3], DmS[3], DmN[3], DpN[3];
        // x faces: normal u, tangential v
        pvm(g, hdry, xhi[0].h, xhi[0].e, xhi[0].u, xhi[0].v, xlo[1].h, xlo[1].e, xlo[1].u,
            xlo[1].v, DmW, DpW);
        pvm(g, hdry, xhi[1].h, xhi[1].e, xhi[1].u, xhi[1].v, xlo[2].h, xlo[2].e, xlo[2].u,
            xlo[2].v, DmE, DpE);
        // y faces: normal v, tangential u
        pvm(g, hdry, yhi[0].h, yhi[0].e, yhi[0].v, yhi[0].u, ylo[1].h, ylo[1].e, ylo[1].v,
            ylo[1].u, DmS, DpS);
        pvm(g, hdry, yhi[1].h, yhi[1].e, yhi[1].v, yhi[1].u, ylo[2].h, ylo[2].e, ylo[2].v,
            ylo[2].u, DmN, DpN);
        const St<T>& E = xhi[1]; const St<T>& W = xlo[1];
        const St<T>& N = yhi[1]; const St<T>& S = ylo[1];
        const T hc = cx[2].h;
        // inner-cell terms: convective flux difference + g h (eta_edge+ - eta_edge-)
        T Ix0 = E.h * E.u - W.h * W.u;
        T Ix1 = E.h * E.u * E.u - W.h * W.u * W.u + g * hc * (E.e - W.e);
        T Ix2 = E.h * E.u * E.v - W.h * W.u * W.v;
        T Iy0 = N.h * N.v - S.h * S.v;
        T Iy1 = N.h * N.u * N.v - S.h * S.u * S.v;
        T Iy2 = N.h * N.v * N.v - S.h * S.v * S.v + g * hc * (N.e - S.e);
        const size_t c = (size_t)idx;
        const T Hc = H[c];
        const T rx = dt / P.dx, ry = dt / P.dy;
        T en = eta[c] - rx * (DmE[0] + DpW[0] + Ix0) - ry * (DmN[0] + DpS[0] + Iy0);
        T an = q1[c] - rx * (DmE[1] + DpW[1] + Ix1) - ry * (DmN[2] + DpS[2] + Iy1);
        T bn = q2[c] - rx * (DmE[2] + DpW[2] + Ix2) - ry * (DmN[1] + DpS[1] + Iy2);
        T hn = en + Hc;
        if (P.manning > T(0) && hn > T(0)) {
            T u = desing(hn, an, d4), v = desing(hn, bn, d4);
            T hd = tmax(hn, P.delta);
            T fr = T(1) + dt * g * P.manning * P.manning * sqrt(u * u + v * v) / (hd * cbrt(hd));
            an /= fr;
            bn /= fr;
        }
        if (hn < T(0)) { en = -Hc; an = T(0); bn = T(0); ++nclamp; }
        if (a != T(0)) {
            en = a * etab[c] + b * en;
            an = a * q1b[c] + b * an;
            bn = a * q2b[c] + b * bn;
        }
        eo[c] = en; q1o[c] = an; q2o[c] = bn;
    }
    if (nclamp) atomicAdd(&st->clamped, nclamp);
}

// Face-based form of the hyperbolic update for a TX x TY cell tile: the block stages the
// tile plus a 2-cell halo (h, eta, u, v) in shared memory, then every face is evaluated
// once: it reconstructs the two cells next to it (minmod slopes of its side only) and
// stores, for the left cell, D^- + F_c(U^-) + (0, g h_L eta^-, 0) and, for the right cell,
// D^+ - F_c(U^+) - (0, g h_R eta^+, 0) (normal frame), i.e. the fluctuation plus that
// cell's half of the inner-cell term of Eq. (22) / (30).  A cell sums its four faces.
template <typename T, int TX, int TY>
__global__ void __launch_bounds__(256)
k_hyp2d_t(Prm<T> P, const T* __restrict__ eta, const T* __restrict__ q1,
          const T* __restrict__ q2, const T* __restrict__ etab, const T* __restrict__ q1b,
          const T* __restrict__ q2b, const T* __restrict__ H, T a, T b, T dt,
          T* __restrict__ eo, T* __restrict__ q1o, T* __restrict__ q2o, StepCtl* st)
{
    constexpr int LW = TX + 4, LH = TY + 4, LN = LW * LH;
    constexpr int NFX = (TX + 1) * TY, NFY = TX * (TY + 1);
    __shared__ T sh[LN], se[LN], su[LN], sv[LN];
    __shared__ T CLx[3][NFX], CRx[3][NFX], CLy[3][NFY], CRy[3][NFY];
    const T d2 = P.delta * P.delta, d4 = d2 * d2;
    const T g = P.g, hdry = P.hdry;
    const int i0 = blockIdx.x * TX, j0 = blockIdx.y * TY;
    const int tid = threadIdx.x, nt = blockDim.x;
    for (int t = tid; t < LN; t += nt) {
        const int li = t % LW, lj = t / LW;
        // cells more than 2 outside the domain only feed discarded faces: clamp them
        int ci = i0 + li - 2, cj = j0 + lj - 2;
        ci = ci > P.nx + 1 ? P.nx + 1 : ci;
        cj = cj > P.ny + 1 ? P.ny + 1 : cj;
        const St<T> c = load_st(P, eta, q1, q2, H, ci, cj, d4);
        sh[t] = c.h; se[t] = c.e; su[t] = c.u; sv[t] = c.v;
    }
    __syncthreads();
    auto L = [&](int i, int j) { return (j + 2) * LW + (i + 2); };   // local cell index
    // x faces f = 0..TX between local cells f-1 and f, rows 0..TY-1
    for (int t = tid; t < NFX + NFY; t += nt) {
        const bool xf = t < NFX;
        const int tt = xf ? t : t - NFX;
        const int f = xf ? tt % (TX + 1) : tt % TX;
        const int r = xf ? tt / (TX + 1) : tt / TX;
        // cells along the face normal: m2 = cell -2, m1 = -1 (left), p0 = right, p1 = +1
        const int s0 = xf ? 1 : LW;
        const int cl = xf ? L(f - 1, r) : L(f, r - 1);   // left cell (west / south)
        const int cr = cl + s0;                            // right cell
        const int cm = cl - s0, cp = cr + s0;
        // left cell: its high-side value; right cell: its low-side value
        const T uL = xf ? su[cl] : sv[cl], uR = xf ? su[cr] : sv[cr];
        const T tL = xf ? sv[cl] : su[cl], tR = xf ? sv[cr] : su[cr];
        const T unm = xf ? su[cm] : sv[cm], unp = xf ? su[cp] : sv[cp];
        const T utm = xf ? sv[cm] : su[cm], utp = xf ? sv[cp] : su[cp];
        const T sLh = minmod(sh[cl] - sh[cm], sh[cr] - sh[cl]);
        const T sLu = minmod(uL - unm, uR - uL);
        const T sLt = minmod(tL - utm, tR - tL);
        const bool dL = sh[cm] <= hdry || sh[cl] <= hdry || sh[cr] <= hdry;
        const T sLe = dL ? T(0) : minmod(se[cl] - se[cm], se[cr] - se[cl]);
        const T sRh = minmod(sh[cr] - sh[cl], sh[cp] - sh[cr]);
        const T sRu = minmod(uR - uL, unp - uR);
        const T sRt = minmod(tR - tL, utp - tR);
        const bool dR = sh[cl] <= hdry || sh[cr] <= hdry || sh[cp] <= hdry;
        const T sRe = dR ? T(0) : minmod(se[cr] - se[cl], se[cp] - se[cr]);
        const T hL = sh[cl] + T(0.5) * sLh, eL = se[cl] + T(0.5) * sLe;
        const T nL = uL + T(0.5) * sLu, tLv = tL + T(0.5) * sLt;
        const T hR = sh[cr] - T(0.5) * sRh, eR = se[cr] - T(0.5) * sRe;
        const T nR = uR - T(0.5) * sRu, tRv = tR - T(0.5) * sRt;
        T Dm[3], Dp[3];
        pvm(g, hdry, hL, eL, nL, tLv, hR, eR, nR, tRv, Dm, Dp);
        const T qL = hL * nL, qR = hR * nR;
        T* oL0 = xf ? &CLx[0][tt] : &CLy[0][tt];
        T* oR0 = xf ? &CRx[0][tt] : &CRy[0][tt];
        const int stride = xf ? NFX : NFY;
        oL0[0] = Dm[0] + qL;
        oL0[stride] = Dm[1] + qL * nL + g * sh[cl] * eL;
        oL0[2 * stride] = Dm[2] + qL * tLv;
        oR0[0] = Dp[0] - qR;
        oR0[stride] = Dp[1] - (qR * nR + g * sh[cr] * eR);
        oR0[2 * stride] = Dp[2] - qR * tRv;
    }
    __syncthreads();
    int nclamp = 0;
    for (int t = tid; t < TX * TY; t += nt) {
        const int li = t % TX, lj = t / TX;
        const int gi = i0 + li, gj = j0 + lj;
        if (gi >= P.nx || gj >= P.ny) continue;
        const int fe = lj * (TX + 1) + li + 1, fw = fe - 1;     // x faces east / west
        const int fn = (lj + 1) * TX + li, fs = lj * TX + li;   // y faces north / south
        const size_t c = (size_t)gj * P.nx + gi;
        const T Hc = H[c];
        const T rx = dt / P.dx, ry = dt / P.dy;
        T en = eta[c] - rx * (CLx[0][fe] + CRx[0][fw]) - ry * (CLy[0][fn] + CRy[0][fs]);
        T an = q1[c] - rx * (CLx[1][fe] + CRx[1][fw]) - ry * (CLy[2][fn] + CRy[2][fs]);
        T bn = q2[c] - rx * (CLx[2][fe] + CRx[2][fw]) - ry * (CLy[1][fn] + CRy[1][fs]);
        T hn = en + Hc;
        if (P.manning > T(0) && hn > T(0)) {
            T u = desing(hn, an, d4), v = desing(hn, bn, d4);
            T hd = tmax(hn, P.delta);
            T fr = T(1) + dt * g * P.manning * P.manning * sqrt(u * u + v * v) / (hd * cbrt(hd));
            an /= fr;
            bn /= fr;
        }
        if (hn < T(0)) { en = -Hc; an = T(0); bn = T(0); ++nclamp; }
        if (a != T(0)) {
            en = a * etab[c] + b * en;
            an = a * q1b[c] + b * an;
            bn = a * q2b[c] + b * bn;
        }
        eo[c] = en; q1o[c] = an; q2o[c] = bn;
    }
    if (nclamp) atomicAdd(&st->clamped, nclamp);
}

// Breaking terms at cells (Sec. 3 with q_x -> div q, u_x -> div u):
// q += de 2 nu (div u) grad H, centred differences.
template <typename T>
__global__ void __launch_bounds__(kThreads)
k_break2d(Prm<T> P, const T* __restrict__ eta, const T* __restrict__ q1,
          const T* __restrict__ q2, const T* __restrict__ H, T de, T* __restrict__ q1o,
          T* __restrict__ q2o)
{
    const T d2 = P.delta * P.delta, d4 = d2 * d2;
    GRID_STRIDE(idx, (long long)P.nx * P.ny)
    {
        const int i = (int)(idx % P.nx), j = (int)(idx / P.nx);
        // neighbours W, E, S, N with parity; velocities desingularised
        T qq[4], uu[4], HH[4];
        const int di[4] = {-1, 1, 0, 0}, dj[4] = {0, 0, -1, 1};
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            bool rx, ry;
            int ii = map_cell(i + di[k], P.nx, P.bcw, P.bce, rx);
            int jj = map_cell(j + dj[k], P.ny, P.bcs, P.bcn, ry);
            size_t m = (size_t)jj * P.nx + ii;
            T h = tmax(eta[m] + H[m], T(0));
            T a = q1[m], b = q2[m];
            if (rx) a = -a;
            if (ry) b = -b;
            qq[k] = k < 2 ? a : b;
            uu[k] = desing(h, qq[k], d4);
            HH[k] = H[m];
        }
        const size_t c = (size_t)idx;
        T h = tmax(eta[c] + H[c], T(0));
        T dq = (qq[1] - qq[0]) / (T(2) * P.dx) + (qq[3] - qq[2]) / (T(2) * P.dy);
        T du = (uu[1] - uu[0]) / (T(2) * P.dx) + (uu[3] - uu[2]) / (T(2) * P.dy);
        T Hx = (HH[1] - HH[0]) / (T(2) * P.dx), Hy = (HH[3] - HH[2]) / (T(2) * P.dy);
        T nu = nu_break(h, dq, P.g, P.B1, P.hdry);
        q1o[c] = q1[c] + de * T(2) * nu * du * Hx;
        q2o[c] = q2[c] + de * T(2) * nu * du * Hy;
    }
}

// Assembly at node (I, J) (App. A.2, Eqs. 36-41): w* (+ breaking), the five coefficients
// of the row scaled by 8 dx dy / de, and the right-hand side b = -(8 dx dy / de) B(q*, w*).
// Link (x) between nodes (I, J) and (I+1, J) carries alpha+- = 2 h~ + X~, X~ - 2 h~ (h~, X~
// averages over cells (I, J-1), (I, J)); node terms beta-+ = Xi -+ 2 h_c.
// With resid_form = 1 the kernel stores the defect r0 = b - M p0 for a correction solve
// M dp = r0 started from the warm start p0 (the solver's rounding floor then applies to dp,
// not to p); else b itself.
template <typename T>
__global__ void __launch_bounds__(kThreads)
k_asm2d(Prm<T> P, const T* __restrict__ eta, const T* __restrict__ H,
        const T* __restrict__ q1k, const T* __restrict__ q2k, const T* __restrict__ q1s,
        const T* __restrict__ q2s, const T* __restrict__ w_in, const T* __restrict__ w_b,
        T a, T b, T de, int with_coef, T* __restrict__ ws, T* __restrict__ cC,
        T* __restrict__ cW, T* __restrict__ cE, T* __restrict__ cS, T* __restrict__ cN,
        T* __restrict__ rhs, const T* __restrict__ p0, int resid_form, double* partials,
        SolveCtl* ctl, double tol2, int max_iter, int kpass)
{
    const T d2 = P.delta * P.delta, d4 = d2 * d2;
    const int nxn = P.nx + 1;
    const T inv2dx = T(1) / (T(2) * P.dx), inv2dy = T(1) / (T(2) * P.dy);
    const T scale = T(8) * P.dx * P.dy / de;
    double acc[3] = {0.0, 0.0, 0.0};   // ||b||^2, ||D^-1 b||^2, max Gershgorin radius
    GRID_STRIDE(idx, (long long)(P.nx + 1) * (P.ny + 1))
    {
        const int I = (int)(idx % nxn), J = (int)(idx / nxn);
        // s = 2 eta - h = eta - H on a 4x4 cross around the node; h at the 4 core cells.
        // sx[r][k]: rows J-1 (r=0), J (r=1), columns I-2 .. I+1
        // sy[c][k]: columns I-1 (c=0), I (c=1), rows J-2 .. J+1
        T sx[2][4], sy[2][4], hq[2][2];
#pragma unroll
        for (int r = 0; r < 2; ++r)
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                bool rx, ry;
                int ii = map_cell(I - 2 + k, P.nx, P.bcw, P.bce, rx);
                int jj = map_cell(J - 1 + r, P.ny, P.bcs, P.bcn, ry);
                size_t m = (size_t)jj * P.nx + ii;
                const T e = eta[m], Hm = H[m];
                sx[r][k] = e - Hm;
                if (k == 1 || k == 2) hq[r][k - 1] = tmax(e + Hm, T(0));
            }
#pragma unroll
        for (int cc = 0; cc < 2; ++cc)
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                bool rx, ry;
                int ii = map_cell(I - 1 + cc, P.nx, P.bcw, P.bce, rx);
                int jj = map_cell(J - 2 + k, P.ny, P.bcs, P.bcn, ry);
                size_t m = (size_t)jj * P.nx + ii;
                sy[cc][k] = eta[m] - H[m];
            }
        // core cells: a = (I-1, J-1), b = (I, J-1), d = (I-1, J), e = (I, J)
        const T ha = hq[0][0], hb = hq[0][1], hd = hq[1][0], he = hq[1][1];
        const T sa = sx[0][1], sb = sx[0][2], sd_ = sx[1][1], se = sx[1][2];
        // X (x-differences of s) at a, b, d, e; Y (y-differences) at a, b, d, e
        const T Xa = T(0.5) * (sx[0][2] - sx[0][0]), Xb = T(0.5) * (sx[0][3] - sx[0][1]);
        const T Xd = T(0.5) * (sx[1][2] - sx[1][0]), Xe = T(0.5) * (sx[1][3] - sx[1][1]);
        const T Ya = T(0.5) * (sy[0][2] - sy[0][0]), Yd = T(0.5) * (sy[0][3] - sy[0][1]);
        const T Yb = T(0.5) * (sy[1][2] - sy[1][0]), Ye = T(0.5) * (sy[1][3] - sy[1][1]);
        const T hc = T(0.25) * (ha + hb + hd + he);
        const T Xi = T(0.5) * (se + sb) - T(0.5) * (sd_ + sa);
        const T Yi = T(0.5) * (sd_ + se) - T(0.5) * (sa + sb);
        // discharges of the core cells (post-breaking) with boundary parity
        T Q1[4], Q2[4], P1[4], P2[4];
        const int ci[4] = {I - 1, I, I - 1, I}, cj[4] = {J - 1, J - 1, J, J};
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            bool rx, ry;
            int ii = map_cell(ci[k], P.nx, P.bcw, P.bce, rx);
            int jj = map_cell(cj[k], P.ny, P.bcs, P.bcn, ry);
            size_t m = (size_t)jj * P.nx + ii;
            Q1[k] = rx ? -q1k[m] : q1k[m];
            Q2[k] = ry ? -q2k[m] : q2k[m];
            if (P.breaking) {
                P1[k] = rx ? -q1s[m] : q1s[m];
                P2[k] = ry ? -q2s[m] : q2s[m];
            }
        }
        const size_t nidx = (size_t)idx;
        T wv = a != T(0) ? a * w_b[nidx] + b * w_in[nidx] : w_in[nidx];
        if (P.breaking) {
            const T hh[4] = {ha, hb, hd, he};
            T ua[4], va[4];
#pragma unroll
            for (int k = 0; k < 4; ++k) { ua[k] = desing(hh[k], P1[k], d4); va[k] = desing(hh[k], P2[k], d4); }
            T dq = (P1[1] + P1[3] - P1[0] - P1[2]) / (T(2) * P.dx)
                 + (P2[2] + P2[3] - P2[0] - P2[1]) / (T(2) * P.dy);
            T du = (ua[1] + ua[3] - ua[0] - ua[2]) / (T(2) * P.dx)
                 + (va[2] + va[3] - va[0] - va[1]) / (T(2) * P.dy);
            T nu = nu_break(hc, dq, P.g, P.B1, P.hdry);
            wv += de * T(2) * nu * du * desing(hc, T(1), d4);
        }
        ws[nidx] = wv;
        // B(q*, w*) (Eqs. 37-40) with the edge discharges of Eq. (41) at p = 0
        const T q1E = T(0.5) * (Q1[3] + Q1[1]), q1W = T(0.5) * (Q1[2] + Q1[0]);
        const T q2N = T(0.5) * (Q2[3] + Q2[2]), q2S = T(0.5) * (Q2[1] + Q2[0]);
        const T Bs = ((T(2) * hc - Xi) * q1E - (T(2) * hc + Xi) * q1W) * inv2dx
                   + ((T(2) * hc - Yi) * q2N - (T(2) * hc + Yi) * q2S) * inv2dy
                   + T(2) * hc * wv;
        const T bval = -scale * Bs;
        acc[0] += (double)bval * (double)bval;
        if (with_coef) {
            const T apE = T(2) * T(0.5) * (hb + he) + T(0.5) * (Xb + Xe);
            const T amE = T(0.5) * (Xb + Xe) - T(2) * T(0.5) * (hb + he);
            const T apW = T(2) * T(0.5) * (ha + hd) + T(0.5) * (Xa + Xd);
            const T amW = T(0.5) * (Xa + Xd) - T(2) * T(0.5) * (ha + hd);
            const T apN = T(2) * T(0.5) * (hd + he) + T(0.5) * (Yd + Ye);
            const T amN = T(0.5) * (Yd + Ye) - T(2) * T(0.5) * (hd + he);
            const T apS = T(2) * T(0.5) * (ha + hb) + T(0.5) * (Ya + Yb);
            const T amS = T(0.5) * (Ya + Yb) - T(2) * T(0.5) * (ha + hb);
            const T bmx = Xi - T(2) * hc, bpx = Xi + T(2) * hc;  // beta-, beta+ of the x links
            const T bmy = Yi - T(2) * hc, bpy = Yi + T(2) * hc;
            const T rxl = P.dy / P.dx, ryl = P.dx / P.dy;
            const T vE = rxl * bmx * apE, vW = rxl * bpx * amW;
            const T vN = ryl * bmy * apN, vS = ryl * bpy * amS;
            const T dC = T(16) * P.dx * P.dy + rxl * (bmx * amE + bpx * apW)
                       + ryl * (bmy * amN + bpy * apS);
            cE[nidx] = vE; cW[nidx] = vW; cN[nidx] = vN; cS[nidx] = vS; cC[nidx] = dC;
            const T id = T(1) / fabs(dC);
            const T bs = bval * id;
            acc[1] += (double)bs * (double)bs;
            acc[2] = fmax(acc[2], (double)((fabs(vE) + fabs(vW) + fabs(vN) + fabs(vS)) * id));
            if (resid_form) {
                const int Iw = map_node(I - 1, P.nx), Ie = map_node(I + 1, P.nx);
                const int Js = map_node(J - 1, P.ny), Jn = map_node(J + 1, P.ny);
                T mp = dC * p0[nidx];
                mp = fma(vW, p0[(size_t)J * nxn + Iw], mp);
                mp = fma(vE, p0[(size_t)J * nxn + Ie], mp);
                mp = fma(vS, p0[(size_t)Js * nxn + I], mp);
                mp = fma(vN, p0[(size_t)Jn * nxn + I], mp);
                rhs[nidx] = bval - mp;
            } else {
                rhs[nidx] = bval;
            }
        } else {
            rhs[nidx] = bval;
        }
    }
    if (grid_reduce<3, 4u>(acc, partials, &ctl->counter) && threadIdx.x == 0) {
        ctl->bb = acc[0];
        ctl->bdb = acc[1];
        ctl->gersh = acc[2];
        ctl->tol2 = tol2;
        ctl->max_iter = max_iter;
        ctl->iter = 0;
        ctl->sweeps = 0;
        ctl->done = 0;
        ctl->status = 0;
        // Chebyshev semi-iteration on D^-1 M with spectrum in [1 - g, 1 + g] (Gershgorin):
        // theta = 1, delta = g, sigma1 = 1 / g; sweep 0 is plain Jacobi (c1 = 0, c2 = 1).
        if (with_coef && kpass > 0) {
            if (!(acc[2] < 1.0)) {
                ctl->status = 4;   // no diagonal dominance: the caller switches solver
                ctl->done = 1;
            } else {
                const double dl = acc[2] > 1e-12 ? acc[2] : 1e-12;
                ctl->delta = dl;
                ctl->sigma1 = 1.0 / dl;
                double rp = dl;   // rho_0 = 1 / sigma1
                ctl->c1[0] = 0.0;
                ctl->c2[0] = 1.0;
                for (int k = 1; k < kpass; ++k) {
                    const double rn = 1.0 / (2.0 * ctl->sigma1 - rp);
                    ctl->c1[k] = rn * rp;
                    ctl->c2[k] = 2.0 * rn / dl;
                    rp = rn;
                }
                for (int k = 0; k < kpass; ++k) {
                    ctl->c1f[k] = (float)ctl->c1[k];
                    ctl->c2f[k] = (float)ctl->c2[k];
                }
                ctl->rho_prev = rp;
            }
        }
    }
}

// Tiled form of the assembly for a TX x TY node tile: the block stages s = eta - H and h of
// the cells around the tile (a 2-cell ring), computes the centred differences X, Y of every
// cell once, stages the discharges of the cells touching the tile's nodes, and then builds
// each node's row, right-hand side (or defect) and w* from shared memory.  Same arithmetic
// as k_asm2d per node.
template <typename T, int TX, int TY>
__global__ void __launch_bounds__(256)
k_asm2d_t(Prm<T> P, const T* __restrict__ eta, const T* __restrict__ H,
          const T* __restrict__ q1k, const T* __restrict__ q2k, const T* __restrict__ q1s,
          const T* __restrict__ q2s, const T* __restrict__ w_in, const T* __restrict__ w_b,
          T a, T b, T de, int with_coef, T* __restrict__ ws, T* __restrict__ cC,
          T* __restrict__ cW, T* __restrict__ cE, T* __restrict__ cS, T* __restrict__ cN,
          T* __restrict__ rhs, const T* __restrict__ p0, int resid_form, double* partials,
          SolveCtl* ctl, double tol2, int max_iter, int kpass)
{
    // staged cells: columns I0-2 .. I0+TX, rows J0-2 .. J0+TY  (SW x SH)
    constexpr int SW = TX + 3, SH = TY + 3, SN = SW * SH;
    // core cells (touching the tile's nodes): columns I0-1 .. I0+TX-1, rows J0-1 .. J0+TY-1
    constexpr int CW = TX + 1, CHh = TY + 1, CN = CW * CHh;
    __shared__ T ss[SN], hs[SN];
    __shared__ T Xc[CN], Yc[CN], Q1c[CN], Q2c[CN], U1c[CN], V1c[CN], P1c[CN], P2c[CN];
    const T d2 = P.delta * P.delta, d4 = d2 * d2;
    const int nxn = P.nx + 1;
    const int I0 = blockIdx.x * TX, J0 = blockIdx.y * TY;
    const int tid = threadIdx.x, nt = blockDim.x;
    for (int t = tid; t < SN; t += nt) {
        const int li = t % SW, lj = t / SW;
        int ci = I0 - 2 + li, cj = J0 - 2 + lj;
        ci = ci > P.nx + 1 ? P.nx + 1 : ci;
        cj = cj > P.ny + 1 ? P.ny + 1 : cj;
        bool rx, ry;
        const int ii = map_cell(ci, P.nx, P.bcw, P.bce, rx);
        const int jj = map_cell(cj, P.ny, P.bcs, P.bcn, ry);
        const size_t m = (size_t)jj * P.nx + ii;
        const T e = eta[m], Hm = H[m];
        ss[t] = e - Hm;
        hs[t] = tmax(e + Hm, T(0));
    }
    for (int t = tid; t < CN; t += nt) {
        const int li = t % CW, lj = t / CW;
        int ci = I0 - 1 + li, cj = J0 - 1 + lj;
        ci = ci > P.nx + 1 ? P.nx + 1 : ci;
        cj = cj > P.ny + 1 ? P.ny + 1 : cj;
        bool rx, ry;
        const int ii = map_cell(ci, P.nx, P.bcw, P.bce, rx);
        const int jj = map_cell(cj, P.ny, P.bcs, P.bcn, ry);
        const size_t m = (size_t)jj * P.nx + ii;
        Q1c[t] = rx ? -q1k[m] : q1k[m];
        Q2c[t] = ry ? -q2k[m] : q2k[m];
        if (P.breaking) {
            P1c[t] = rx ? -q1s[m] : q1s[m];
            P2c[t] = ry ? -q2s[m] : q2s[m];
        }
    }
    __syncthreads();
    for (int t = tid; t < CN; t += nt) {
        const int li = t % CW, lj = t / CW;
        const int sidx = (lj + 1) * SW + (li + 1);   // staged index of this core cell
        Xc[t] = T(0.5) * (ss[sidx + 1] - ss[sidx - 1]);
        Yc[t] = T(0.5) * (ss[sidx + SW] - ss[sidx - SW]);
        if (P.breaking) {
            U1c[t] = desing(hs[sidx], P1c[t], d4);
            V1c[t] = desing(hs[sidx], P2c[t], d4);
        }
    }
    __syncthreads();
    const T inv2dx = T(1) / (T(2) * P.dx), inv2dy = T(1) / (T(2) * P.dy);
    const T scale = T(8) * P.dx * P.dy / de;
    const T rxl = P.dy / P.dx, ryl = P.dx / P.dy;
    double acc[3] = {0.0, 0.0, 0.0};
    for (int t = tid; t < TX * TY; t += nt) {
        const int li = t % TX, lj = t / TX;
        const int I = I0 + li, J = J0 + lj;
        if (I > P.nx || J > P.ny) continue;
        // core-local indices of cells a (I-1,J-1), b (I,J-1), d (I-1,J), e (I,J)
        const int ka = lj * CW + li, kb = ka + 1, kd = ka + CW, ke = kd + 1;
        const int sa = (lj + 1) * SW + (li + 1), sb = sa + 1, sd = sa + SW, se = sd + 1;
        const T ha = hs[sa], hb = hs[sb], hd = hs[sd], he = hs[se];
        const T hc = T(0.25) * (ha + hb + hd + he);
        const T Xi = T(0.5) * (ss[se] + ss[sb]) - T(0.5) * (ss[sd] + ss[sa]);
        const T Yi = T(0.5) * (ss[sd] + ss[se]) - T(0.5) * (ss[sa] + ss[sb]);
        const size_t nidx = (size_t)J * nxn + I;
        T wv = a != T(0) ? a * w_b[nidx] + b * w_in[nidx] : w_in[nidx];
        if (P.breaking) {
            T dq = (P1c[kb] + P1c[ke] - P1c[ka] - P1c[kd]) * inv2dx
                 + (P2c[kd] + P2c[ke] - P2c[ka] - P2c[kb]) * inv2dy;
            T du = (U1c[kb] + U1c[ke] - U1c[ka] - U1c[kd]) * inv2dx
                 + (V1c[kd] + V1c[ke] - V1c[ka] - V1c[kb]) * inv2dy;
            T nu = nu_break(hc, dq, P.g, P.B1, P.hdry);
            wv += de * T(2) * nu * du * desing(hc, T(1), d4);
        }
        ws[nidx] = wv;
        const T q1E = T(0.5) * (Q1c[ke] + Q1c[kb]), q1W = T(0.5) * (Q1c[kd] + Q1c[ka]);
        const T q2N = T(0.5) * (Q2c[ke] + Q2c[kd]), q2S = T(0.5) * (Q2c[kb] + Q2c[ka]);
        const T Bs = ((T(2) * hc - Xi) * q1E - (T(2) * hc + Xi) * q1W) * inv2dx
                   + ((T(2) * hc - Yi) * q2N - (T(2) * hc + Yi) * q2S) * inv2dy
                   + T(2) * hc * wv;
        const T bval = -scale * Bs;
        acc[0] += (double)bval * (double)bval;
        if (with_coef) {
            const T Xa = Xc[ka], Xb = Xc[kb], Xd = Xc[kd], Xe = Xc[ke];
            const T Ya = Yc[ka], Yb = Yc[kb], Yd = Yc[kd], Ye = Yc[ke];
            const T apE = (hb + he) + T(0.5) * (Xb + Xe), amE = T(0.5) * (Xb + Xe) - (hb + he);
            const T apW = (ha + hd) + T(0.5) * (Xa + Xd), amW = T(0.5) * (Xa + Xd) - (ha + hd);
            const T apN = (hd + he) + T(0.5) * (Yd + Ye), amN = T(0.5) * (Yd + Ye) - (hd + he);
            const T apS = (ha + hb) + T(0.5) * (Ya + Yb), amS = T(0.5) * (Ya + Yb) - (ha + hb);
            const T bmx = Xi - T(2) * hc, bpx = Xi + T(2) * hc;
            const T bmy = Yi - T(2) * hc, bpy = Yi + T(2) * hc;
            const T vE = rxl * bmx * apE, vW = rxl * bpx * amW;
            const T vN = ryl * bmy * apN, vS = ryl * bpy * amS;
            const T dC = T(16) * P.dx * P.dy + rxl * (bmx * amE + bpx * apW)
                       + ryl * (bmy * amN + bpy * apS);
            cE[nidx] = vE; cW[nidx] = vW; cN[nidx] = vN; cS[nidx] = vS; cC[nidx] = dC;
            const T id = T(1) / fabs(dC);
            const T bs = bval * id;
            acc[1] += (double)bs * (double)bs;
            acc[2] = fmax(acc[2], (double)((fabs(vE) + fabs(vW) + fabs(vN) + fabs(vS)) * id));
            if (resid_form) {
                const int Iw = map_node(I - 1, P.nx), Ie = map_node(I + 1, P.nx);
                const int Js = map_node(J - 1, P.ny), Jn = map_node(J + 1, P.ny);
                T mp = dC * p0[nidx];
                mp = fma(vW, p0[(size_t)J * nxn + Iw], mp);
                mp = fma(vE, p0[(size_t)J * nxn + Ie], mp);
                mp = fma(vS, p0[(size_t)Js * nxn + I], mp);
                mp = fma(vN, p0[(size_t)Jn * nxn + I], mp);
                rhs[nidx] = bval - mp;
            } else {
                rhs[nidx] = bval;
            }
        } else {
            rhs[nidx] = bval;
        }
    }
    if (grid_reduce<3, 4u>(acc, partials, &ctl->counter) && tid == 0) {
        ctl->bb = acc[0];
        ctl->bdb = acc[1];
        ctl->gersh = acc[2];
        ctl->tol2 = tol2;
        ctl->max_iter = max_iter;
        ctl->iter = 0;
        ctl->sweeps = 0;
        ctl->done = 0;
        ctl->status = 0;
        if (with_coef && kpass > 0) {
            if (!(acc[2] < 1.0)) {
                ctl->status = 4;
                ctl->done = 1;
            } else {
                const double dl = acc[2] > 1e-12 ? acc[2] : 1e-12;
                ctl->delta = dl;
                ctl->sigma1 = 1.0 / dl;
                double rp = dl;
                ctl->c1[0] = 0.0;
                ctl->c2[0] = 1.0;
                for (int k = 1; k < kpass; ++k) {
                    const double rn = 1.0 / (2.0 * ctl->sigma1 - rp);
                    ctl->c1[k] = rn * rp;
                    ctl->c2[k] = 2.0 * rn / dl;
                    rp = rn;
                }
                for (int k = 0; k < kpass; ++k) {
                    ctl->c1f[k] = (float)ctl->c1[k];
                    ctl->c2f[k] = (float)ctl->c2[k];
                }
                ctl->rho_prev = rp;
            }
        }
    }
}

// (M x) at node (I, J) from the stored row and mirrored neighbours.
template <typename T>
struct Rows {
    const T *cC, *cW, *cE, *cS, *cN;
    int nx, ny;
};

template <typename T, typename F>
__device__ __forceinline__ T row_apply(const Rows<T>& R, int I, int J, T xc, F xat)
{
    const int nxn = R.nx + 1;
    const size_t k = (size_t)J * nxn + I;
    const int Iw = map_node(I - 1, R.nx), Ie = map_node(I + 1, R.nx);
    const int Js = map_node(J - 1, R.ny), Jn = map_node(J + 1, R.ny);
    return R.cC[k] * xc + R.cW[k] * xat((size_t)J * nxn + Iw) + R.cE[k] * xat((size_t)J * nxn + Ie)
         + R.cS[k] * xat((size_t)Js * nxn + I) + R.cN[k] * xat((size_t)Jn * nxn + I);
}

template <typename T>
__global__ void __launch_bounds__(kThreads)
k_matvec2d(Rows<T> R, const T* __restrict__ x, T* __restrict__ y)
{
    const int nxn = R.nx + 1;
    GRID_STRIDE(idx, (long long)(R.nx + 1) * (R.ny + 1))
    {
        const int I = (int)(idx % nxn), J = (int)(idx / nxn);
        y[idx] = row_apply(R, I, J, x[idx], [&](size_t m) { return x[m]; });
    }
}

// BiCGStab, right Jacobi preconditioning (y = D^-1 p^, z = D^-1 s), FP64 scalars.
// init: r = b - M x, rhat = r, p^ = v = 0; rho1 = r.r
template <typename T>
__global__ void __launch_bounds__(kThreads)
k_bicg_init(Rows<T> R, const T* __restrict__ b, T* __restrict__ x, T* __restrict__ r,
            T* __restrict__ rh, T* __restrict__ ph0, T* __restrict__ v0, double* partials,
            SolveCtl* ctl)
{
    const int nxn = R.nx + 1;
    const bool zero_rhs = ctl->bb == 0.0;
    double acc[1] = {0.0};
    GRID_STRIDE(idx, (long long)(R.nx + 1) * (R.ny + 1))
    {
        T rv;
        if (zero_rhs) {
            x[idx] = T(0);
            rv = T(0);
        } else {
            const int I = (int)(idx % nxn), J = (int)(idx / nxn);
            rv = b[idx] - row_apply(R, I, J, x[idx], [&](size_t m) { return x[m]; });
        }
        r[idx] = rv; rh[idx] = rv; ph0[idx] = T(0); v0[idx] = T(0);
        acc[0] += (double)rv * (double)rv;
    }
    if (grid_reduce<1, 0u>(acc, partials, &ctl->counter) && threadIdx.x == 0) {
        ctl->rho1 = acc[0];
        ctl->rr = acc[0];
        ctl->rho = 1.0; ctl->alpha = 1.0; ctl->omega = 1.0;
        const bool conv = zero_rhs || acc[0] <= ctl->tol2 * ctl->bb;
        ctl->done = conv ? 1 : 0;
        ctl->status = conv ? 1 : 0;
    }
}

// phase A: p^ = r + beta (p^ - omega v); v = M D^-1 p^; alpha = rho1 / (rhat . v)
template <typename T>
__global__ void __launch_bounds__(kThreads)
k_bicg_A(Rows<T> R, const T* __restrict__ r, const T* __restrict__ rh,
         const T* __restrict__ ph_old, const T* __restrict__ v_old, T* __restrict__ ph_new,
         T* __restrict__ v_new, double* partials, SolveCtl* ctl)
{
    if (ctl->done) return;
    const int nxn = R.nx + 1;
    const double beta_d = (ctl->rho1 / ctl->rho) * (ctl->alpha / ctl->omega);
    const T beta = (T)beta_d, om = (T)ctl->omega;
    double acc[1] = {0.0};
    GRID_STRIDE(idx, (long long)(R.nx + 1) * (R.ny + 1))
    {
        const int I = (int)(idx % nxn), J = (int)(idx / nxn);
        auto pnew = [&](size_t m) { return r[m] + beta * (ph_old[m] - om * v_old[m]); };
        const T pc = pnew((size_t)idx);
        const T vc = row_apply(R, I, J, pc / R.cC[idx],
                               [&](size_t m) { return pnew(m) / R.cC[m]; });
        ph_new[idx] = pc;
        v_new[idx] = vc;
        acc[0] += (double)rh[idx] * (double)vc;
    }
    if (grid_reduce<1, 0u>(acc, partials, &ctl->counter) && threadIdx.x == 0) {
        ctl->rv = acc[0];
        ctl->rho = ctl->rho1;
        if (acc[0] == 0.0 || !isfinite(acc[0])) {
            ctl->done = 1; ctl->status = 3;
        } else {
            ctl->alpha = ctl->rho1 / acc[0];
        }
    }
}

// phase B: s = r - alpha v; t = M D^-1 s; omega = (t . s) / (t . t)
template <typename T>
__global__ void __launch_bounds__(kThreads)
k_bicg_B(Rows<T> R, const T* __restrict__ r, const T* __restrict__ v, T* __restrict__ t,
         double* partials, SolveCtl* ctl)
{
    if (ctl->done) return;
    const int nxn = R.nx + 1;
    const T al = (T)ctl->alpha;
    double acc[2] = {0.0, 0.0};
    GRID_STRIDE(idx, (long long)(R.nx + 1) * (R.ny + 1))
    {
        const int I = (int)(idx % nxn), J = (int)(idx / nxn);
        auto sat = [&](size_t m) { return r[m] - al * v[m]; };
        const T sc = sat((size_t)idx);
        const T tc = row_apply(R, I, J, sc / R.cC[idx], [&](size_t m) { return sat(m) / R.cC[m]; });
        t[idx] = tc;
        acc[0] += (double)tc * (double)sc;
        acc[1] += (double)tc * (double)tc;
    }
    if (grid_reduce<2, 0u>(acc, partials, &ctl->counter) && threadIdx.x == 0) {
        ctl->ts = acc[0];
        ctl->tt = acc[1];
        ctl->omega = acc[1] > 0.0 ? acc[0] / acc[1] : 0.0;
    }
}

// phase C: x += alpha D^-1 p^ + omega D^-1 s; r = s - omega t; rho1 = rhat . r; test
template <typename T>
__global__ void __launch_bounds__(kThreads)
k_bicg_C(Rows<T> R, T* __restrict__ r, const T* __restrict__ rh, const T* __restrict__ ph,
         const T* __restrict__ v, const T* __restrict__ t, T* __restrict__ x, double* partials,
         SolveCtl* ctl)
{
    if (ctl->done) return;
    const T al = (T)ctl->alpha, om = (T)ctl->omega;
    double acc[2] = {0.0, 0.0};
    GRID_STRIDE(idx, (long long)(R.nx + 1) * (R.ny + 1))
    {
        const T s = r[idx] - al * v[idx];
        const T dinv = T(1) / R.cC[idx];
        x[idx] += (al * ph[idx] + om * s) * dinv;
        const T rn = s - om * t[idx];
        r[idx] = rn;
        acc[0] += (double)rh[idx] * (double)rn;
        acc[1] += (double)rn * (double)rn;
    }
    if (grid_reduce<2, 0u>(acc, partials, &ctl->counter) && threadIdx.x == 0) {
        ctl->rho1 = acc[0];
        ctl->rr = acc[1];
        ctl->iter += 1;
        if (acc[1] <= ctl->tol2 * ctl->bb) { ctl->done = 1; ctl->status = 1; }
        else if (ctl->iter >= ctl->max_iter) { ctl->done = 1; ctl->status = 2; }
        else if (ctl->omega == 0.0 || acc[0] == 0.0 || !isfinite(acc[1])) {
            ctl->done = 1; ctl->status = 3;
        }
    }
}

// Jacobi with Chebyshev-scheduled relaxation (the "scheduled relaxation" of Sec. 5 with
// the Chebyshev weights of the Gershgorin interval [1 - g, 1 + g] of D^-1 M), K sweeps per
// launch with temporal blocking: each block loads a tile plus a K-node halo into shared
// memory, sweeps K times there (the valid region shrinking by one node per sweep) and
// writes the tile back.  Sweep k: x_{k+1} = x_k + c1 (x_k - x_{k-1}) + c2 r_k with
// r_k = D^-1 (b - M x_k).  The last sweep accumulates ||r||^2 (Jacobi-scaled) and
// max |x_{k+1} - x_k|; the last block tests convergence and prepares the next K weights.
// A (32, BY) thread block owns a fixed set of region
// nodes per thread (columns tx + 32 a, rows ty + 8 b), so the sweep loop has no index
// arithmetic beyond constant offsets.  The region is the tile plus a K-node halo on every
// side; outside the domain the halo holds mirror images (values, and coefficients with
// W <-> E or S <-> N swapped), which evolve exactly as the nodes they mirror, so tiles at
// the boundary are no different from interior ones.  x_{k-1} lives in registers.
template <typename T, int NA, int NB, int BY, int K>
__global__ void __launch_bounds__(32 * BY, 2)
k_cheb_pass2(Rows<T> R, const T* __restrict__ b, T* __restrict__ x, T* __restrict__ xp,
             double* partials, SolveCtl* ctl)
{
    if (ctl->done) return;
    constexpr int RW = 32 * NA, RH = BY * NB, RN = RW * RH;
    constexpr int TX = RW - 2 * K, TY = RH - 2 * K;
    extern __shared__ unsigned char cheb2_smem[];
    T* xs0 = reinterpret_cast<T*>(cheb2_smem);
    T* xs1 = xs0 + RN;
    T* bd = xs1 + RN;
    T* wW = bd + RN;
    T* wE = wW + RN;
    T* wS = wE + RN;
    T* wN = wS + RN;
    const int nx = R.nx, ny = R.ny, NX = nx + 1;
    const int I0 = (int)blockIdx.x * TX - K, J0 = (int)blockIdx.y * TY - K;
    const int tx = threadIdx.x, ty = threadIdx.y;
    T xa[NA * NB];
#pragma unroll
    for (int bb = 0; bb < NB; ++bb)
#pragma unroll
        for (int aa = 0; aa < NA; ++aa) {
            const int li = tx + 32 * aa, lj = ty + BY * bb;
            const int gI = I0 + li, gJ = J0 + lj;
            int mI = gI < 0 ? -gI : (gI > nx ? 2 * nx - gI : gI);
            int mJ = gJ < 0 ? -gJ : (gJ > ny ? 2 * ny - gJ : gJ);
            const bool fx = mI != gI, fy = mJ != gJ;
            mI = mI < 0 ? 0 : (mI > nx ? nx : mI);   // far outside: any finite value
            mJ = mJ < 0 ? 0 : (mJ > ny ? ny : mJ);
            const size_t g = (size_t)mJ * NX + mI;
            const int sidx = lj * RW + li;
            const T ic = T(1) / R.cC[g];
            xs0[sidx] = x[g];
            xa[bb * NA + aa] = xp[g];
            bd[sidx] = b[g] * ic;
            const T cw = R.cW[g] * ic, ce = R.cE[g] * ic;
            const T cs = R.cS[g] * ic, cn = R.cN[g] * ic;
            wW[sidx] = fx ? ce : cw;
            wE[sidx] = fx ? cw : ce;
            wS[sidx] = fy ? cn : cs;
            wN[sidx] = fy ? cs : cn;
        }
    T c1s[K], c2s[K];
#pragma unroll
    for (int k = 0; k < K; ++k) {
        if (sizeof(T) == 4) { c1s[k] = (T)ctl->c1f[k]; c2s[k] = (T)ctl->c2f[k]; }
        else { c1s[k] = (T)ctl->c1[k]; c2s[k] = (T)ctl->c2[k]; }
    }
    __syncthreads();
    T* cur = xs0;
    T* nxt = xs1;
    T rsum = T(0), dmax = T(0);   // per-thread (few terms): native precision is enough
#pragma unroll
    for (int sw = 0; sw < K; ++sw) {
        const T c1 = c1s[sw], c2 = c2s[sw];
#pragma unroll
        for (int bb = 0; bb < NB; ++bb)
#pragma unroll
            for (int aa = 0; aa < NA; ++aa) {
                const int li = tx + 32 * aa, lj = ty + BY * bb;
                if (li > sw && li < RW - 1 - sw && lj > sw && lj < RH - 1 - sw) {
                    const int sidx = lj * RW + li;
                    const T xc = cur[sidx];
                    const T r = bd[sidx] - xc -
                                (wW[sidx] * cur[sidx - 1] + wE[sidx] * cur[sidx + 1] +
                                 wS[sidx] * cur[sidx - RW] + wN[sidx] * cur[sidx + RW]);
                    const T xn = xc + c1 * (xc - xa[bb * NA + aa]) + c2 * r;
                    nxt[sidx] = xn;
                    xa[bb * NA + aa] = xc;
                    if (sw == K - 1 && li >= K && li < RW - K && lj >= K && lj < RH - K &&
                        I0 + li <= nx && J0 + lj <= ny) {
                        rsum = fma(r, r, rsum);
                        dmax = tmax(dmax, T(fabs(xn - xc)));
                    }
                }
            }
        __syncthreads();
        T* tmp = cur; cur = nxt; nxt = tmp;
    }
#pragma unroll
    for (int bb = 0; bb < NB; ++bb)
#pragma unroll
        for (int aa = 0; aa < NA; ++aa) {
            const int li = tx + 32 * aa, lj = ty + BY * bb;
            const int gI = I0 + li, gJ = J0 + lj;
            if (li >= K && li < RW - K && lj >= K && lj < RH - K && gI <= nx && gJ <= ny) {
                const size_t g = (size_t)gJ * NX + gI;
                x[g] = cur[lj * RW + li];
                xp[g] = xa[bb * NA + aa];
            }
        }
    double acc[2];
    if (grid_reduce_sum_max_f((float)rsum, (float)dmax, partials, &ctl->counter, acc) &&
        tx == 0 && ty == 0) {
        ctl->rr = acc[0];
        ctl->dpmax = acc[1];
        ctl->sweeps += K;
        ctl->iter = ctl->sweeps;
        const bool conv = ctl->eps_dp > 0.0 ? acc[1] < ctl->eps_dp
                                            : acc[0] <= ctl->tol2 * ctl->bdb;
        if (conv) { ctl->done = 1; ctl->status = 1; }
        else if (!isfinite(acc[0])) { ctl->done = 1; ctl->status = 3; }
        else if (ctl->sweeps >= ctl->max_iter) { ctl->done = 1; ctl->status = 2; }
        double rp = ctl->rho_prev;
        for (int k = 0; k < K; ++k) {
            const double rn = 1.0 / (2.0 * ctl->sigma1 - rp);
            ctl->c1[k] = rn * rp;
            ctl->c2[k] = 2.0 * rn / ctl->delta;
            ctl->c1f[k] = (float)ctl->c1[k];
            ctl->c2f[k] = (float)ctl->c2[k];
            rp = rn;
        }
        ctl->rho_prev = rp;
    }
}

// Correction (Eq. 36 and the w update of Eq. 41) at node (I, J) and cell (I, J):
// q1 += de (T^Hor_N + T^Hor_S)/2, q2 += de (T^Ver_E + T^Ver_W)/2, w += de p / h_c;
// dry cells (h <= hdry) keep q = 0, as App. B A.2 assumes where the depth vanishes.
// In the final stage also the Eq. (23) rate max((|u|+c)/dx + (|v|+c)/dy).
template <typename T>
__global__ void __launch_bounds__(kThreads)
k_corr2d(Prm<T> P, const T* __restrict__ eta, const T* __restrict__ H,
         const T* __restrict__ q1k, const T* __restrict__ q2k, const T* __restrict__ ws,
         const T* __restrict__ p, const T* __restrict__ dp, T* __restrict__ pout, T de,
         int with_p, T* __restrict__ eo, T* __restrict__ q1o,
         T* __restrict__ q2o, T* __restrict__ wo, int final_stage, double* partials,
         StepCtl* st)
{
    const T d2 = P.delta * P.delta, d4 = d2 * d2;
    const int nxn = P.nx + 1;
    double acc[1] = {0.0};
    int bad = 0;
    GRID_STRIDE(idx, (long long)(P.nx + 1) * (P.ny + 1))
    {
        const int I = (int)(idx % nxn), J = (int)(idx / nxn);
        // node
        T pc = T(0);
        if (with_p) {
            pc = p[idx] + dp[idx];
            T hs = T(0);
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                bool rx, ry;
                int ii = map_cell(I - 1 + (k & 1), P.nx, P.bcw, P.bce, rx);
                int jj = map_cell(J - 1 + (k >> 1), P.ny, P.bcs, P.bcn, ry);
                size_t m = (size_t)jj * P.nx + ii;
                hs += tmax(eta[m] + H[m], T(0));
            }
            const T hc = T(0.25) * hs;
            const T wn = ws[idx] + de * pc * desing(hc, T(1), d4);
            wo[idx] = wn;
            pout[idx] = pc;
            if (!isfinite(wn) || !isfinite(pc)) bad = 1;
        } else {
            wo[idx] = ws[idx];
            pout[idx] = T(0);
        }
        // cell
        if (I < P.nx && J < P.ny) {
            const int i = I, j = J;
            const size_t c = (size_t)j * P.nx + i;
            const T e = eta[c], Hc = H[c];
            const T h = tmax(e + Hc, T(0));
            T a1 = q1k[c], a2 = q2k[c];
            if (with_p) {
                bool rx, ry;
                int iw = map_cell(i - 1, P.nx, P.bcw, P.bce, rx);
                int ie = map_cell(i + 1, P.nx, P.bcw, P.bce, rx);
                int js = map_cell(j - 1, P.ny, P.bcs, P.bcn, ry);
                int jn = map_cell(j + 1, P.ny, P.bcs, P.bcn, ry);
                const size_t mw = (size_t)j * P.nx + iw, me = (size_t)j * P.nx + ie;
                const size_t ms = (size_t)js * P.nx + i, mn = (size_t)jn * P.nx + i;
                const T X = T(0.5) * ((eta[me] - H[me]) - (eta[mw] - H[mw]));
                const T Y = T(0.5) * ((eta[mn] - H[mn]) - (eta[ms] - H[ms]));
                auto pat = [&](size_t m) { return p[m] + dp[m]; };
                const T pSW = pat((size_t)J * nxn + I), pSE = pat((size_t)J * nxn + I + 1);
                const T pNW = pat((size_t)(J + 1) * nxn + I), pNE = pat((size_t)(J + 1) * nxn + I + 1);
                const T TN = -T(0.5) * h * (pNE - pNW) / P.dx - T(0.25) * (pNE + pNW) * X / P.dx;
                const T TS = -T(0.5) * h * (pSE - pSW) / P.dx - T(0.25) * (pSE + pSW) * X / P.dx;
                const T TE = -T(0.5) * h * (pNE - pSE) / P.dy - T(0.25) * (pNE + pSE) * Y / P.dy;
                const T TW = -T(0.5) * h * (pNW - pSW) / P.dy - T(0.25) * (pNW + pSW) * Y / P.dy;
                a1 += de * T(0.5) * (TN + TS);
                a2 += de * T(0.5) * (TE + TW);
            }
            if (h <= P.hdry) { a1 = T(0); a2 = T(0); }   // dry cells carry no discharge
            eo[c] = e; q1o[c] = a1; q2o[c] = a2;
            if (!isfinite(e) || !isfinite(a1) || !isfinite(a2)) bad = 1;
            if (final_stage) {
                const T u = desing(h, a1, d4), v = desing(h, a2, d4), cw = sqrt(P.g * h);
                acc[0] = fmax(acc[0], (double)((fabs(u) + cw) / P.dx + (fabs(v) + cw) / P.dy));
            }
        }
    }
    if (bad) atomicOr(&st->nonfinite, 1);
    if (final_stage) {
        if (grid_reduce<1, 1u>(acc, partials, &st->counter) && threadIdx.x == 0) st->lam = acc[0];
    }
}

// ================================================================ batched 1D kernels
// Row r of the ny rows is an independent channel: cells (i, r), nodes (k, r) with
// row stride nx + 1.

template <typename T>
__device__ __forceinline__ St<T> load_st1(const Prm<T>& P, const T* __restrict__ eta,
                                          const T* __restrict__ q, const T* __restrict__ H,
                                          int i, int row, T d4)
{
    bool rx;
    int ii = map_cell(i, P.nx, P.bcw, P.bce, rx);
    size_t k = (size_t)row * P.nx + ii;
    T e = eta[k];
    T h = tmax(e + H[k], T(0));
    T a = rx ? -q[k] : q[k];
    St<T> s;
    s.h = h; s.e = e; s.u = desing(h, a, d4); s.v = T(0);
    return s;
}

// Hyperbolic update of one cell of a 1D channel (Eqs. 18-22), friction, clamp, combination.
template <typename T>
__global__ void __launch_bounds__(kThreads)
k_hyp1d(Prm<T> P, const T* __restrict__ eta, const T* __restrict__ q,
        const T* __restrict__ etab, const T* __restrict__ qb, const T* __restrict__ H, T a,
        T b, T dt, T* __restrict__ eo, T* __restrict__ qo, StepCtl* st)
{
    const T d2 = P.delta * P.delta, d4 = d2 * d2;
    const T g = P.g, hdry = P.hdry;
    int nclamp = 0;
    GRID_STRIDE(idx, (long long)P.nx * P.ny)
    {
        const int i = (int)(idx % P.nx), row = (int)(idx / P.nx);
        St<T> cx[5];
#pragma unroll
        for (int k = 0; k < 5; ++k) cx[k] = load_st1(P, eta, q, H, i - 2 + k, row, d4);
        St<T> lo[3], hi[3];
#pragma unroll
        for (int k = 1; k <= 3; ++k) recon(cx, k, hdry, lo[k - 1], hi[k - 1]);
        T DmW[3], DpW[3], DmE[3], DpE[3];
        pvm(g, hdry, hi[0].h, hi[0].e, hi[0].u, T(0), lo[1].h, lo[1].e, lo[1].u, T(0), DmW, DpW);
        pvm(g, hdry, hi[1].h, hi[1].e, hi[1].u, T(0), lo[2].h, lo[2].e, lo[2].u, T(0), DmE, DpE);
        const St<T>& E = hi[1]; const St<T>& W = lo[1];
        const T hc = cx[2].h;
        T I0 = E.h * E.u - W.h * W.u;
        T I1 = E.h * E.u * E.u - W.h * W.u * W.u + g * hc * (E.e - W.e);
        const size_t c = (size_t)idx;
        const T Hc = H[c];
        const T rx = dt / P.dx;
        T en = eta[c] - rx * (DmE[0] + DpW[0] + I0);
        T qn = q[c] - rx * (DmE[1] + DpW[1] + I1);
        T hn = en + Hc;
        if (P.manning > T(0) && hn > T(0)) {
            T u = desing(hn, qn, d4);
            T hd = tmax(hn, P.delta);
            qn /= T(1) + dt * g * P.manning * P.manning * fabs(u) / (hd * cbrt(hd));
        }
        if (hn < T(0)) { en = -Hc; qn = T(0); ++nclamp; }
        if (a != T(0)) {
            en = a * etab[c] + b * en;
            qn = a * qb[c] + b * qn;
        }
        eo[c] = en; qo[c] = qn;
    }
    if (nclamp) atomicAdd(&st->clamped, nclamp);
}

// 1D breaking terms at cells: q += de 2 nu u_x H_x (centred differences, Sec. 4.3).
template <typename T>
__global__ void __launch_bounds__(kThreads)
k_break1d(Prm<T> P, const T* __restrict__ eta, const T* __restrict__ q,
          const T* __restrict__ H, T de, T* __restrict__ qo)
{
    const T d2 = P.delta * P.delta, d4 = d2 * d2;
    GRID_STRIDE(idx, (long long)P.nx * P.ny)
    {
        const int i = (int)(idx % P.nx), row = (int)(idx / P.nx);
        T qq[2], uu[2], HH[2];
#pragma unroll
        for (int k = 0; k < 2; ++k) {
            bool rx;
            int ii = map_cell(i - 1 + 2 * k, P.nx, P.bcw, P.bce, rx);
            size_t m = (size_t)row * P.nx + ii;
            T h = tmax(eta[m] + H[m], T(0));
            qq[k] = rx ? -q[m] : q[m];
            uu[k] = desing(h, qq[k], d4);
            HH[k] = H[m];
        }
        const size_t c = (size_t)idx;
        T h = tmax(eta[c] + H[c], T(0));
        T qx = (qq[1] - qq[0]) / (T(2) * P.dx);
        T ux = (uu[1] - uu[0]) / (T(2) * P.dx);
        T Hx = (HH[1] - HH[0]) / (T(2) * P.dx);
        T nu = nu_break(h, qx, P.g, P.B1, P.hdry);
        qo[c] = q[c] + de * T(2) * nu * ux * Hx;
    }
}

// Tridiagonal row of App. B, Eq. (43) at node k of a channel (cells k-1, k), outside
// neighbours folded onto their mirrors, rhs = -(8 dx^2 / de) B(q*, w*); also w*.
template <typename T>
__global__ void __launch_bounds__(kThreads)
k_asm1d(Prm<T> P, const T* __restrict__ eta, const T* __restrict__ H,
        const T* __restrict__ qpre, const T* __restrict__ qk, const T* __restrict__ w_in,
        const T* __restrict__ w_b, T a, T b, T de, T* __restrict__ ws, T* __restrict__ A,
        T* __restrict__ Bd, T* __restrict__ Cc, T* __restrict__ rhs)
{
    const T d2 = P.delta * P.delta, d4 = d2 * d2;
    const int nxn = P.nx + 1;
    const T dx = P.dx;
    GRID_STRIDE(idx, (long long)nxn * P.ny)
    {
        const int k = (int)(idx % nxn), row = (int)(idx / nxn);
        // s = eta - H at cells k-3 .. k+0 shifted: s[m] is cell k-2+m, m = 0..3
        T s[4], hv[2], qv[2], qp[2];
#pragma unroll
        for (int m = 0; m < 4; ++m) {
            bool rx;
            int ii = map_cell(k - 2 + m, P.nx, P.bcw, P.bce, rx);
            size_t c = (size_t)row * P.nx + ii;
            s[m] = eta[c] - H[c];
            if (m == 1 || m == 2) {
                hv[m - 1] = tmax(eta[c] + H[c], T(0));
                qv[m - 1] = rx ? -qk[c] : qk[c];
                qp[m - 1] = rx ? -qpre[c] : qpre[c];
            }
        }
        const T hL = hv[0], hR = hv[1];
        const T xiL = T(0.5) * (s[2] - s[0]), xiR = T(0.5) * (s[3] - s[1]);
        const T xin = s[2] - s[1];
        const T hn = T(0.5) * (hL + hR);
        T ak = (xiL - T(2) * hL) * (xin + T(2) * hn);
        T bk = T(16) * dx * dx + xin * (xiL + xiR + T(2) * hL - T(2) * hR)
             + T(2) * hn * (xiL - xiR + T(4) * hn);
        T ck = (xiR + T(2) * hR) * (xin - T(2) * hn);
        if (k == 0) { ck += ak; ak = T(0); }
        if (k == P.nx) { ak += ck; ck = T(0); }
        const size_t nidx = (size_t)idx;
        T wv = a != T(0) ? a * w_b[nidx] + b * w_in[nidx] : w_in[nidx];
        if (P.breaking) {
            T qx = (qp[1] - qp[0]) / dx;
            T ux = (desing(hR, qp[1], d4) - desing(hL, qp[0], d4)) / dx;
            T nu = nu_break(hn, qx, P.g, P.B1, P.hdry);
            wv += de * T(2) * nu * ux * desing(hn, T(1), d4);
        }
        ws[nidx] = wv;
        const T Bs = hn * (qv[1] - qv[0]) / dx - T(0.5) * (qv[1] + qv[0]) * xin / dx
                   + T(2) * hn * wv;
        A[nidx] = ak; Bd[nidx] = bk; Cc[nidx] = ck;
        rhs[nidx] = -(T(8) * dx * dx / de) * Bs;
    }
}

// Parallel cyclic reduction of one channel's system per block, in shared memory.
template <typename T, int PER>
__global__ void __launch_bounds__(1024)
k_pcr(int n, const T* __restrict__ A, const T* __restrict__ Bd, const T* __restrict__ Cc,
      const T* __restrict__ D, T* __restrict__ x)
{
    extern __shared__ unsigned char smraw[];
    T* a = reinterpret_cast<T*>(smraw);
    T* b = a + n;
    T* c = b + n;
    T* d = c + n;
    const size_t off = (size_t)blockIdx.x * n;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        a[i] = A[off + i]; b[i] = Bd[off + i]; c[i] = Cc[off + i]; d[i] = D[off + i];
    }
    __syncthreads();
    for (int s = 1; s < n; s <<= 1) {
        T na[PER], nb[PER], nc[PER], nd[PER];
#pragma unroll
        for (int r = 0; r < PER; ++r) {
            const int i = threadIdx.x + r * blockDim.x;
            if (i < n) {
                const int im = i - s, ip = i + s;
                T k1 = im >= 0 ? a[i] / b[im] : T(0);
                T k2 = ip < n ? c[i] / b[ip] : T(0);
                na[r] = im >= 0 ? -a[im] * k1 : T(0);
                nc[r] = ip < n ? -c[ip] * k2 : T(0);
                nb[r] = b[i] - (im >= 0 ? c[im] * k1 : T(0)) - (ip < n ? a[ip] * k2 : T(0));
                nd[r] = d[i] - (im >= 0 ? d[im] * k1 : T(0)) - (ip < n ? d[ip] * k2 : T(0));
            }
        }
        __syncthreads();
#pragma unroll
        for (int r = 0; r < PER; ++r) {
            const int i = threadIdx.x + r * blockDim.x;
            if (i < n) { a[i] = na[r]; b[i] = nb[r]; c[i] = nc[r]; d[i] = nd[r]; }
        }
        __syncthreads();
    }
    for (int i = threadIdx.x; i < n; i += blockDim.x) x[off + i] = d[i] / b[i];
}

// Thomas algorithm, one thread per channel, for systems too long for shared memory;
// cp / dp are scratch node arrays.
template <typename T>
__global__ void k_thomas(int n, int rows, const T* __restrict__ A, const T* __restrict__ Bd,
                         const T* __restrict__ Cc, const T* __restrict__ D, T* __restrict__ cp,
                         T* __restrict__ dp, T* __restrict__ x)
{
    const int row = blockIdx.x * blockDim.x + threadIdx.x;
    if (row >= rows) return;
    const size_t o = (size_t)row * n;
    cp[o] = Cc[o] / Bd[o];
    dp[o] = D[o] / Bd[o];
    for (int i = 1; i < n; ++i) {
        const T m = Bd[o + i] - A[o + i] * cp[o + i - 1];
        cp[o + i] = Cc[o + i] / m;
        dp[o + i] = (D[o + i] - A[o + i] * dp[o + i - 1]) / m;
    }
    x[o + n - 1] = dp[o + n - 1];
    for (int i = n - 2; i >= 0; --i) x[o + i] = dp[o + i] - cp[o + i] * x[o + i + 1];
}

template <typename T>
__global__ void __launch_bounds__(kThreads)
k_tri_apply(int n, long long total, const T* __restrict__ A, const T* __restrict__ Bd,
            const T* __restrict__ Cc, const T* __restrict__ x, T* __restrict__ y)
{
    GRID_STRIDE(idx, total)
    {
        const int k = (int)(idx % n);
        T v = Bd[idx] * x[idx];
        if (k > 0) v += A[idx] * x[idx - 1];
        if (k < n - 1) v += Cc[idx] * x[idx + 1];
        y[idx] = v;
    }
}

// 1D correction (Eqs. 26-28): q += de T_NH(p), w += de p / h; Eq. (23) rate when final.
template <typename T>
__global__ void __launch_bounds__(kThreads)
k_corr1d(Prm<T> P, const T* __restrict__ eta, const T* __restrict__ H,
         const T* __restrict__ qk, const T* __restrict__ ws, T* __restrict__ p, T de,
         int with_p, T* __restrict__ eo, T* __restrict__ qo, T* __restrict__ wo,
         int final_stage, double* partials, StepCtl* st)
{
    const T d2 = P.delta * P.delta, d4 = d2 * d2;
    const int nxn = P.nx + 1;
    double acc[1] = {0.0};
    int bad = 0;
    GRID_STRIDE(idx, (long long)nxn * P.ny)
    {
        const int k = (int)(idx % nxn), row = (int)(idx / nxn);
        if (with_p) {
            T hs = T(0);
#pragma unroll
            for (int m = 0; m < 2; ++m) {
                bool rx;
                int ii = map_cell(k - 1 + m, P.nx, P.bcw, P.bce, rx);
                size_t c = (size_t)row * P.nx + ii;
                hs += tmax(eta[c] + H[c], T(0));
            }
            const T wn = ws[idx] + de * p[idx] * desing(T(0.5) * hs, T(1), d4);
            wo[idx] = wn;
            if (!isfinite(wn)) bad = 1;
        } else {
            wo[idx] = ws[idx];
            p[idx] = T(0);
        }
        if (k < P.nx) {
            const int i = k;
            const size_t c = (size_t)row * P.nx + i;
            const T e = eta[c];
            const T h = tmax(e + H[c], T(0));
            T qn = qk[c];
            if (with_p) {
                bool rx;
                const size_t mw = (size_t)row * P.nx + map_cell(i - 1, P.nx, P.bcw, P.bce, rx);
                const size_t me = (size_t)row * P.nx + map_cell(i + 1, P.nx, P.bcw, P.bce, rx);
                const T xi = T(0.5) * ((eta[me] - H[me]) - (eta[mw] - H[mw]));
                const T pw = p[idx], pe = p[idx + 1];
                const T Tn = -T(0.5) * (h * (pe - pw) / P.dx + T(0.5) * (pe + pw) * xi / P.dx);
                qn += de * Tn;
            }
            if (h <= P.hdry) qn = T(0);   // dry cells carry no discharge
            eo[c] = e; qo[c] = qn;
            if (!isfinite(e) || !isfinite(qn)) bad = 1;
            if (final_stage) {
                const T u = desing(h, qn, d4);
                acc[0] = fmax(acc[0], (double)((fabs(u) + sqrt(P.g * h)) / P.dx));
            }
        }
    }
    if (bad) atomicOr(&st->nonfinite, 1);
    if (final_stage) {
        if (grid_reduce<1, 1u>(acc, partials, &st->counter) && threadIdx.x == 0) st->lam = acc[0];
    }
}

// ================================================================ shared small kernels

template <typename T>
__global__ void __launch_bounds__(kThreads)
k_mass(long long n, const T* __restrict__ eta, const T* __restrict__ H, double* partials,
       StepCtl* st)
{
    double acc[1] = {0.0};
    GRID_STRIDE(idx, n) acc[0] += (double)tmax(eta[idx] + H[idx], T(0));
    if (grid_reduce<1, 0u>(acc, partials, &st->counter) && threadIdx.x == 0) st->mass = acc[0];
}

template <typename T>
__global__ void __launch_bounds__(kThreads)
k_lambda(Prm<T> P, int dim, const T* __restrict__ eta, const T* __restrict__ q1,
         const T* __restrict__ q2, const T* __restrict__ H, double* partials, StepCtl* st)
{
    const T d2 = P.delta * P.delta, d4 = d2 * d2;
    double acc[1] = {0.0};
    GRID_STRIDE(idx, (long long)P.nx * P.ny)
    {
        const T h = tmax(eta[idx] + H[idx], T(0));
        const T cw = sqrt(P.g * h);
        const T u = desing(h, q1[idx], d4);
        double l = (fabs(u) + cw) / P.dx;
        if (dim == 2) l += (fabs(desing(h, q2[idx], d4)) + cw) / P.dy;
        acc[0] = fmax(acc[0], l);
    }
    if (grid_reduce<1, 1u>(acc, partials, &st->counter) && threadIdx.x == 0) st->lam = acc[0];
}

template <typename T>
__global__ void k_fill(T* x, long long n, T v)
{
    GRID_STRIDE(idx, n) x[idx] = v;
}

template <typename T>
__global__ void k_from_double(const double* src, T* dst, long long n)
{
    GRID_STRIDE(idx, n) dst[idx] = (T)src[idx];
}

template <typename T>
Rows<T> rows_of(const Prm<T>& P, const Bufs<T>& B)
{
    Rows<T> R;
    R.cC = B.cC; R.cW = B.cW; R.cE = B.cE; R.cS = B.cS; R.cN = B.cN;
    R.nx = P.nx; R.ny = P.ny;
    return R;
}

}  // namespace

// ================================================================ launchers

template <typename T>
void launch_hyp2d(const Prm<T>& P, const Launch& L, const T* eta, const T* q1, const T* q2,
                  const T* etab, const T* q1b, const T* q2b, const T* H, T a, T b, T dt,
                  T* eo, T* q1o, T* q2o, StepCtl* st)
{
    constexpr int TX = 32, TY = sizeof(T) == 4 ? 16 : 8;
    dim3 grid((P.nx + TX - 1) / TX, (P.ny + TY - 1) / TY);
    k_hyp2d_t<T, TX, TY><<<grid, kThreads, 0, L.s>>>(P, eta, q1, q2, etab, q1b, q2b, H, a, b, dt,
                                                    eo, q1o, q2o, st);
}

template <typename T>
void launch_break2d(const Prm<T>& P, const Launch& L, const T* eta, const T* q1, const T* q2,
                    const T* H, T de, T* q1o, T* q2o)
{
    k_break2d<T><<<L.nblk, kThreads, 0, L.s>>>(P, eta, q1, q2, H, de, q1o, q2o);
}

template <typename T>
void launch_asm2d(const Prm<T>& P, const Launch& L, const Bufs<T>& B, const T* w_in,
                  const T* w_base, T a, T b, T de, int with_coef, int resid_form, double tol2,
                  int max_iter, int kpass, double* partials, SolveCtl* ctl)
{
    constexpr int TX = 32, TY = 16;
    dim3 grid((P.nx + 1 + TX - 1) / TX, (P.ny + 1 + TY - 1) / TY);
    k_asm2d_t<T, TX, TY><<<grid, kThreads, 0, L.s>>>(P, B.etas, B.H, B.q1k, B.q2k, B.q1s, B.q2s,
                                                    w_in, w_base, a, b, de, with_coef, B.ws,
                                                    B.cC, B.cW, B.cE, B.cS, B.cN, B.rhs, B.p,
                                                    resid_form, partials, ctl, tol2, max_iter,
                                                    kpass);
}

template <typename T> struct ChebCfg;
// region 128 x 32 nodes (FP32) / 64 x 32 (FP64), 512 threads, 8 nodes per thread, 4 sweeps
template <> struct ChebCfg<float> { static constexpr int NA = 4, NB = 2, BY = 16, K = 4; };
template <> struct ChebCfg<double> { static constexpr int NA = 2, NB = 2, BY = 16, K = 4; };

template <typename T>
int cheb_sweeps_per_pass() { return ChebCfg<T>::K; }

template <typename T>
size_t asm_tiles(const Prm<T>& P)
{
    return (size_t)((P.nx + 1 + 31) / 32) * ((P.ny + 1 + 15) / 16);
}

template <typename T>
size_t cheb_tiles(const Prm<T>& P)
{
    using C = ChebCfg<T>;
    constexpr int TX = 32 * C::NA - 2 * C::K, TY = C::BY * C::NB - 2 * C::K;
    return (size_t)((P.nx + 1 + TX - 1) / TX) * ((P.ny + 1 + TY - 1) / TY);
}

template <typename T>
int launch_cheb_pass(const Prm<T>& P, cudaStream_t s, const Bufs<T>& B, T* xprev,
                     double* partials)
{
    using C = ChebCfg<T>;
    constexpr int TX = 32 * C::NA - 2 * C::K, TY = C::BY * C::NB - 2 * C::K;
    constexpr size_t smem = 7 * (size_t)(32 * C::NA) * (C::BY * C::NB) * sizeof(T);
    static bool attr_set = false;
    if (!attr_set) {
        if (cudaFuncSetAttribute(k_cheb_pass2<T, C::NA, C::NB, C::BY, C::K>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
            cudaSuccess)
            return -1;
        attr_set = true;
    }
    dim3 grid((P.nx + 1 + TX - 1) / TX, (P.ny + 1 + TY - 1) / TY);
    k_cheb_pass2<T, C::NA, C::NB, C::BY, C::K><<<grid, dim3(32, C::BY), smem, s>>>(
        rows_of(P, B), B.rhs, B.dp, xprev, partials, B.sctl);
    return 0;
}

template <typename T>
void launch_matvec2d(const Prm<T>& P, const Launch& L, const Bufs<T>& B, const T* x, T* y)
{
    k_matvec2d<T><<<L.nblk, kThreads, 0, L.s>>>(rows_of(P, B), x, y);
}

template <typename T>
void launch_bicg_init(const Prm<T>& P, const Launch& L, const Bufs<T>& B, double* partials)
{
    k_bicg_init<T><<<L.nblk, kThreads, 0, L.s>>>(rows_of(P, B), B.rhs, B.dp, B.r, B.rh, B.ph[0],
                                                 B.v[0], partials, B.sctl);
}

template <typename T>
void launch_bicg_phase(const Prm<T>& P, const Launch& L, const Bufs<T>& B, int parity, int phase,
                       double* partials)
{
    const Rows<T> R = rows_of(P, B);
    T* pho = B.ph[parity];
    T* vo = B.v[parity];
    T* phn = B.ph[parity ^ 1];
    T* vn = B.v[parity ^ 1];
    if (phase == 0)
        k_bicg_A<T><<<L.nblk, kThreads, 0, L.s>>>(R, B.r, B.rh, pho, vo, phn, vn, partials, B.sctl);
    else if (phase == 1)
        k_bicg_B<T><<<L.nblk, kThreads, 0, L.s>>>(R, B.r, vn, B.t, partials, B.sctl);
    else
        k_bicg_C<T><<<L.nblk, kThreads, 0, L.s>>>(R, B.r, B.rh, phn, vn, B.t, B.dp, partials,
                                                  B.sctl);
}

template <typename T>
void launch_corr2d(const Prm<T>& P, const Launch& L, const Bufs<T>& B, const T* q1k,
                   const T* q2k, T de, int with_p, T* eo, T* q1o, T* q2o, T* wo, int final_stage,
                   double* partials, StepCtl* st)
{
    k_corr2d<T><<<L.nblk, kThreads, 0, L.s>>>(P, B.etas, B.H, q1k, q2k, B.ws, B.p, B.dp, B.palt,
                                              de, with_p, eo, q1o, q2o, wo, final_stage, partials,
                                              st);
}

template <typename T>
void launch_hyp1d(const Prm<T>& P, const Launch& L, const T* eta, const T* q, const T* etab,
                  const T* qb, const T* H, T a, T b, T dt, T* eo, T* qo, StepCtl* st)
{
    k_hyp1d<T><<<L.nblk, kThreads, 0, L.s>>>(P, eta, q, etab, qb, H, a, b, dt, eo, qo, st);
}

template <typename T>
void launch_break1d(const Prm<T>& P, const Launch& L, const T* eta, const T* q, const T* H,
                    T de, T* qo)
{
    k_break1d<T><<<L.nblk, kThreads, 0, L.s>>>(P, eta, q, H, de, qo);
}

template <typename T>
void launch_asm1d(const Prm<T>& P, const Launch& L, const Bufs<T>& B, const T* q_pre,
                  const T* qk, const T* w_in, const T* w_base, T a, T b, T de)
{
    k_asm1d<T><<<L.nblk, kThreads, 0, L.s>>>(P, B.etas, B.H, q_pre, qk, w_in, w_base, a, b, de,
                                             B.ws, B.cW, B.cC, B.cE, B.rhs);
}

int pcr_max_n(int elem_bytes) { return elem_bytes == 8 ? 4096 : 8192; }

template <typename T>
int launch_tridiag1d(const Prm<T>& P, cudaStream_t s, const Bufs<T>& B, T* x)
{
    const int n = P.nx + 1;
    if (n <= pcr_max_n((int)sizeof(T))) {
        const size_t smem = 4 * (size_t)n * sizeof(T);
        const int thr = n >= 1024 ? 1024 : ((n + 31) / 32) * 32;
        const int per = (n + thr - 1) / thr;
        cudaError_t e = cudaSuccess;
#define NH_PCR(PERV)                                                                        \
    do {                                                                                    \
        e = cudaFuncSetAttribute(k_pcr<T, PERV>, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                                 (int)smem);                                                \
        if (e == cudaSuccess)                                                               \
            k_pcr<T, PERV><<<P.ny, thr, smem, s>>>(n, B.cW, B.cC, B.cE, B.rhs, x);          \
    } while (0)
        if (per <= 1) NH_PCR(1);
        else if (per <= 2) NH_PCR(2);
        else if (per <= 4) NH_PCR(4);
        else NH_PCR(8);
#undef NH_PCR
        return e == cudaSuccess ? 0 : -1;
    }
    k_thomas<T><<<(P.ny + 127) / 128, 128, 0, s>>>(n, P.ny, B.cW, B.cC, B.cE, B.rhs, B.r, B.rh, x);
    return 0;
}

template <typename T>
int launch_tridiag_raw(int n, int rows, const T* a, const T* b, const T* c, const T* d, T* x,
                       T* cp, T* dp, cudaStream_t s)
{
    if (n <= pcr_max_n((int)sizeof(T))) {
        const size_t smem = 4 * (size_t)n * sizeof(T);
        const int thr = n >= 1024 ? 1024 : ((n + 31) / 32) * 32;
        const int per = (n + thr - 1) / thr;
        cudaError_t e = cudaSuccess;
#define NH_PCR_RAW(PERV)                                                                    \
    do {                                                                                    \
        e = cudaFuncSetAttribute(k_pcr<T, PERV>, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                                 (int)smem);                                                \
        if (e == cudaSuccess) k_pcr<T, PERV><<<rows, thr, smem, s>>>(n, a, b, c, d, x);     \
    } while (0)
        if (per <= 1) NH_PCR_RAW(1);
        else if (per <= 2) NH_PCR_RAW(2);
        else if (per <= 4) NH_PCR_RAW(4);
        else NH_PCR_RAW(8);
#undef NH_PCR_RAW
        return e == cudaSuccess ? 0 : -1;
    }
    if (!cp || !dp) return -2;
    k_thomas<T><<<(rows + 127) / 128, 128, 0, s>>>(n, rows, a, b, c, d, cp, dp, x);
    return 0;
}

template <typename T>
void launch_tridiag_apply1d(const Prm<T>& P, const Launch& L, const Bufs<T>& B, const T* x,
                            T* y)
{
    k_tri_apply<T><<<L.nblk, kThreads, 0, L.s>>>(P.nx + 1, (long long)(P.nx + 1) * P.ny, B.cW,
                                                 B.cC, B.cE, x, y);
}

template <typename T>
void launch_corr1d(const Prm<T>& P, const Launch& L, const Bufs<T>& B, const T* qk, T de,
                   int with_p, T* eo, T* qo, T* wo, int final_stage, double* partials,
                   StepCtl* st)
{
    k_corr1d<T><<<L.nblk, kThreads, 0, L.s>>>(P, B.etas, B.H, qk, B.ws, B.p, de, with_p, eo, qo,
                                              wo, final_stage, partials, st);
}

template <typename T>
void launch_mass(const Prm<T>& P, const Launch& L, const T* eta, const T* H, double* partials,
                 StepCtl* st)
{
    k_mass<T><<<L.nblk, kThreads, 0, L.s>>>((long long)P.nx * P.ny, eta, H, partials, st);
}

template <typename T>
void launch_lambda(const Prm<T>& P, const Launch& L, const T* eta, const T* q1, const T* q2,
                   const T* H, int dim, double* partials, StepCtl* st)
{
    k_lambda<T><<<L.nblk, kThreads, 0, L.s>>>(P, dim, eta, q1, q2, H, partials, st);
}

template <typename T>
void launch_fill(const Launch& L, T* x, size_t n, T v)
{
    k_fill<T><<<L.nblk, kThreads, 0, L.s>>>(x, (long long)n, v);
}

template <typename T>
void launch_convert_from_double(const Launch& L, const double* src, T* dst, size_t n)
{
    k_from_double<T><<<L.nblk, kThreads, 0, L.s>>>(src, dst, (long long)n);
}

#define NH_INSTANTIATE(T)                                                                       \
    template void launch_hyp2d<T>(const Prm<T>&, const Launch&, const T*, const T*, const T*,  \
                                  const T*, const T*, const T*, const T*, T, T, T, T*, T*, T*, \
                                  StepCtl*);                                                   \
    template void launch_break2d<T>(const Prm<T>&, const Launch&, const T*, const T*, const T*,\
                                    const T*, T, T*, T*);                                      \
    template void launch_asm2d<T>(const Prm<T>&, const Launch&, const Bufs<T>&, const T*,      \
                                  const T*, T, T, T, int, int, double, int, int, double*,      \
                                  SolveCtl*);                                                  \
    template int cheb_sweeps_per_pass<T>();                                                    \
    template size_t cheb_tiles<T>(const Prm<T>&);                                              \
    template size_t asm_tiles<T>(const Prm<T>&);                                               \
    template int launch_cheb_pass<T>(const Prm<T>&, cudaStream_t, const Bufs<T>&, T*, double*);\
    template void launch_matvec2d<T>(const Prm<T>&, const Launch&, const Bufs<T>&, const T*,   \
                                     T*);                                                      \
    template void launch_bicg_init<T>(const Prm<T>&, const Launch&, const Bufs<T>&, double*);  \
    template void launch_bicg_phase<T>(const Prm<T>&, const Launch&, const Bufs<T>&, int, int, \
                                       double*);                                               \
    template void launch_corr2d<T>(const Prm<T>&, const Launch&, const Bufs<T>&, const T*,     \
                                   const T*, T, int, T*, T*, T*, T*, int, double*, StepCtl*);  \
    template void launch_hyp1d<T>(const Prm<T>&, const Launch&, const T*, const T*, const T*,  \
                                  const T*, const T*, T, T, T, T*, T*, StepCtl*);              \
    template void launch_break1d<T>(const Prm<T>&, const Launch&, const T*, const T*, const T*,\
                                    T, T*);                                                    \
    template void launch_asm1d<T>(const Prm<T>&, const Launch&, const Bufs<T>&, const T*,      \
                                  const T*, const T*, const T*, T, T, T);                      \
    template int launch_tridiag1d<T>(const Prm<T>&, cudaStream_t, const Bufs<T>&, T*);         \
    template int launch_tridiag_raw<T>(int, int, const T*, const T*, const T*, const T*, T*, T*, \
                                       T*, cudaStream_t);                                      \
    template void launch_tridiag_apply1d<T>(const Prm<T>&, const Launch&, const Bufs<T>&,      \
                                            const T*, T*);                                     \
    template void launch_corr1d<T>(const Prm<T>&, const Launch&, const Bufs<T>&, const T*, T,  \
                                   int, T*, T*, T*, int, double*, StepCtl*);                   \
    template void launch_mass<T>(const Prm<T>&, const Launch&, const T*, const T*, double*,    \
                                 StepCtl*);                                                    \
    template void launch_lambda<T>(const Prm<T>&, const Launch&, const T*, const T*, const T*, \
                                   const T*, int, double*, StepCtl*);                          \
    template void launch_fill<T>(const Launch&, T*, size_t, T);                                \
    template void launch_convert_from_double<T>(const Launch&, const double*, T*, size_t);

NH_INSTANTIATE(float)
NH_INSTANTIATE(double)

}  // namespace nh
