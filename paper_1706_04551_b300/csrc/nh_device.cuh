// nh_device.cuh -- device-side building blocks of the non-hydrostatic shallow-water step
// (Escalante, Morales de Luna & Castro, arXiv:1706.04551), shared by the single-domain
// kernels (nh_kernels.cu) and the batched ensemble kernels (nh_batch.cu).
//
// Boundary conditions are applied by index mapping at load time (walls: mirror, normal
// discharge odd; outflow: copy), so no ghost arrays exist.  The tile and element bodies
// below take their tile coordinates (or element index) as arguments; a kernel maps its
// blocks to the tiles of one domain (blockIdx) or of many (a work list).  Global sums
// (FP64) use per-block partials and a last-block-done finish with a fixed summation order.
// State precision T is float or double.
#pragma once

#include "nh_internal.h"

#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

namespace nh {
namespace dev {

constexpr int kThreads = 256;
constexpr int kCorrThreads = 256;   // threads of a correction tile block

template <typename T> __device__ __forceinline__ T tmin(T a, T b) { return a < b ? a : b; }
template <typename T> __device__ __forceinline__ T tmax(T a, T b) { return a > b ? a : b; }

// minmod slope limiter of the MUSCL reconstruction (Sec. 4.1).
// Branch-free: sign(a) max(0, min(|a|, sign(a) b)) is the smaller of a, b in magnitude when
// they have one sign and zero otherwise.
template <typename T>
__device__ __forceinline__ T minmod(T a, T b)
{
    const T s = copysign(T(1), a);
    return s * tmax(T(0), tmin(fabs(a), s * b));
}

// Square root and quotient of the hot FP32 paths: the hardware approximations
// (sqrt.approx, __fdividef; a few ulp, flush-to-zero), which the FP32 form's tolerance
// covers; FP64 keeps the correctly rounded operations.
__device__ __forceinline__ float qsqrt(float x)
{
    float y;
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ double qsqrt(double x) { return sqrt(x); }
__device__ __forceinline__ float qdiv(float a, float b) { return __fdividef(a, b); }
__device__ __forceinline__ double qdiv(double a, double b) { return a / b; }

// Desingularised q / h (Sec. 4.5): sqrt(2) h q / sqrt(h^4 + max(h^4, delta^4)); d4 = delta^4.
template <typename T>
__device__ __forceinline__ T desing(T h, T q, T d4)
{
    T h2 = h * h;
    T h4 = h2 * h2;
    return qdiv(T(1.4142135623730951) * h * q, qsqrt(h4 + tmax(h4, d4)));
}

// Cell index under the boundary condition of each side: wall = mirror (refl = true),
// outflow = copy of the first interior cell, periodic (1D channels) = the cell n away.
// Valid for up to n cells outside.
__device__ __forceinline__ int map_cell(int i, int n, int bclo, int bchi, bool& refl)
{
    refl = false;
    if (i < 0) {
        if (bclo == 0) { refl = true; return -1 - i; }
        return bclo == 2 ? i + n : 0;
    }
    if (i >= n) {
        if (bchi == 0) { refl = true; return 2 * n - 1 - i; }
        return bchi == 2 ? i - n : n - 1;
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
// sg = sqrt(g): the one-sided celerities sqrt(g h_L), sqrt(g h_R) reuse sqrt(h_L), sqrt(h_R).
template <typename T>
__device__ __forceinline__ void pvm(T g, T sg, T hdry, T hL, T eL, T unL, T utL, T hR, T eR,
                                    T unR, T utR, T Dm[3], T Dp[3])
{
    T qnL = hL * unL, qnR = hR * unR, qtL = hL * utL, qtR = hR * utR;
    T hb = T(0.5) * (hL + hR);
    T sL = qsqrt(hL), sR = qsqrt(hR), ss = sL + sR;
    T ub = ss > T(0) ? qdiv(unL * sL + unR * sR, ss) : T(0);   // Roe velocity
    T cb = qsqrt(g * hb);
    T SL = tmin(ub - cb, unL - sg * sL);
    T SR = tmax(ub + cb, unR + sg * sR);
    // emerging bottom (Sec. 4.5): dry side's bed at or above the wet free surface
    T de = eR - eL;
    if (hR <= hdry && (eR - hR) >= eL) de = T(0);
    if (hL <= hdry && (eL - hL) >= eR) de = T(0);
    T span = SR - SL;
    if (!(span > T(0))) {
        Dm[0] = Dm[1] = Dm[2] = Dp[0] = Dp[1] = Dp[2] = T(0);
        return;
    }
    const T isp = qdiv(T(1), span);
    T a0 = (SR * fabs(SL) - SL * fabs(SR)) * isp;
    T a1 = (fabs(SR) - fabs(SL)) * isp;
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
    T U1 = B1 * qsqrt(g * h);
    if (!(fabs(d) >= U1) || !(U1 > T(0))) return T(0);
    T B = T(1) - qdiv(d, U1);
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

// Write this block's partials (block `bid` of `nblocks` sharing `partials` and `counter`),
// then return true in the last block to finish; that block receives the totals (fixed
// summation order) in v.  The grid form numbers blocks linearly over a 1D or 2D grid; the
// batched kernels pass a domain-local id so that each domain reduces on its own.
template <int NV, unsigned MAXMASK>
__device__ __forceinline__ bool dom_reduce(double (&v)[NV], double* partials, unsigned* counter,
                                           unsigned bid, unsigned nblocks)
{
    block_reduce<NV, MAXMASK>(v);
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

// Publish a block's totals for `cnt` items of a domain at once (the pooled form of
// dom_reduce): the block reduces v, thread 0 writes the totals to slot `slot` (the block
// has written zeros to the slots of its other cnt - 1 items) and counts cnt arrivals.
// Returns true, in every thread, in the block whose arrivals complete the domain's nitems;
// that block receives the totals (fixed order over the slots) in v.  Maxima must be
// non-negative (a zero slot is neutral).
template <int NV, unsigned MAXMASK>
__device__ __forceinline__ bool dom_publish(double (&v)[NV], double* partials,
                                            unsigned* counter, unsigned slot, unsigned cnt,
                                            unsigned nitems)
{
    block_reduce<NV, MAXMASK>(v);
    const unsigned tid = threadIdx.x + blockDim.x * threadIdx.y;
    const unsigned nthr = blockDim.x * blockDim.y;
    __shared__ bool last;
    if (tid == 0) {
#pragma unroll
        for (int k = 0; k < NV; ++k) partials[(size_t)slot * NV + k] = v[k];
        __threadfence();
        last = atomicAdd(counter, cnt) + cnt == nitems;
    }
    __syncthreads();
    if (!last) return false;
    __threadfence();
    double acc[NV];
#pragma unroll
    for (int k = 0; k < NV; ++k) acc[k] = ((MAXMASK >> k) & 1u) ? -1.0e300 : 0.0;
    for (unsigned bb = tid; bb < nitems; bb += nthr)
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

template <int NV, unsigned MAXMASK>
__device__ __forceinline__ bool grid_reduce(double (&v)[NV], double* partials,
                                            unsigned* counter)
{
    return dom_reduce<NV, MAXMASK>(v, partials, counter, blockIdx.y * gridDim.x + blockIdx.x,
                                   gridDim.x * gridDim.y);
}

// Sum (and max) of a pass's per-thread scaled squared-residual sums over the block, thread
// 0 receiving the totals.  FP32 passes: every sum -- a thread's over its regions, a warp's,
// the block's over its warps -- is a double-single pair (float hi + lo kept exact by Knuth's
// TwoSum, about 44 significant bits), converted to FP64 once per block: FP64-class sums
// without FP64 additions, which B300 runs at 1/64 of its FP32 rate.  The thread values are scaled by rsc^2 (an exact power
// of two, see SolveCtl), so they lie far inside the FP32 range.  FP64 passes add in FP64.
// The max is exact in either precision.
__device__ __forceinline__ void two_sum_add(float& hi, float& lo, float x)
{
    const float s = hi + x;
    const float bp = s - hi;
    const float e = (hi - (s - bp)) + (x - bp);
    hi = s;
    lo += e;
}

// Per-thread accumulator of the scaled squares: a double-single pair in FP32 passes, a
// double in FP64 passes.
struct SumDS {
    float hi, lo;
};
template <typename T>
using NormAcc = typename std::conditional<sizeof(T) == 4, SumDS, double>::type;
__device__ __forceinline__ void norm_zero(SumDS& a) { a.hi = 0.f; a.lo = 0.f; }
__device__ __forceinline__ void norm_zero(double& a) { a = 0.0; }
__device__ __forceinline__ void norm_add(SumDS& a, float x) { two_sum_add(a.hi, a.lo, x); }
__device__ __forceinline__ void norm_add(double& a, double x) { a += x; }

// one level of a double-single shuffle tree
__device__ __forceinline__ void ds_shfl_add(float& hi, float& lo, int o)
{
    const float h2 = __shfl_xor_sync(0xffffffffu, hi, o);
    const float l2 = __shfl_xor_sync(0xffffffffu, lo, o);
    two_sum_add(hi, lo, h2);
    lo += l2;
}

template <typename T>
__device__ __forceinline__ void block_sum_max_scaled(NormAcc<T> s, double m, double& out_s,
                                                     double& out_m)
{
    if constexpr (sizeof(T) == 8) {
        double v[2] = {s, m};
        block_reduce<2, 2u>(v);
        out_s = v[0];
        out_m = v[1];
    } else {
        __shared__ float wh[32], wl[32], wm[32];
        const int tid = threadIdx.x + blockDim.x * threadIdx.y;
        const int lane = tid & 31, wid = tid >> 5, nw = (blockDim.x * blockDim.y + 31) >> 5;
        float hi = s.hi, lo = s.lo, mx = (float)m;
        for (int o = 16; o > 0; o >>= 1) {
            ds_shfl_add(hi, lo, o);
            mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        }
        if (lane == 0) { wh[wid] = hi; wl[wid] = lo; wm[wid] = mx; }
        __syncthreads();
        if (wid == 0) {
            hi = lane < nw ? wh[lane] : 0.f;
            lo = lane < nw ? wl[lane] : 0.f;
            mx = lane < nw ? wm[lane] : 0.f;
            for (int o = 16; o > 0; o >>= 1) {
                ds_shfl_add(hi, lo, o);
                mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
            }
            out_s = (double)hi + (double)lo;
            out_m = (double)mx;
        }
        __syncthreads();
    }
}

// The pass's grid reduction: block totals of (scaled sum, max) by block_sum_max_scaled, the
// sum times `scale` (1 / rsc^2) written as this block's FP64 partial, and the last block
// (fixed order over the partials) receives the totals in out (thread 0).
template <typename T>
__device__ __forceinline__ bool dom_reduce_sum_max(NormAcc<T> s, double m, double scale,
                                                   double* partials, unsigned* counter,
                                                   double out[2], unsigned bid,
                                                   unsigned nblocks)
{
    double bs = 0.0, bm = 0.0;
    block_sum_max_scaled<T>(s, m, bs, bm);
    const unsigned tid = threadIdx.x + blockDim.x * threadIdx.y;
    const unsigned nthr = blockDim.x * blockDim.y;
    __shared__ bool last;
    if (tid == 0) {
        partials[(size_t)bid * 2] = bs * scale;
        partials[(size_t)bid * 2 + 1] = bm;
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

// Publish a block's (sum, max) for `cnt` items of a domain at once: thread 0 writes it to
// partial slot `slot` (the block has written zeros to the slots of its other `cnt - 1`
// items) and counts `cnt` arrivals.  Returns true, in every thread, in the block whose
// arrivals complete the domain's `nitems`; that block receives the totals (fixed order over
// the slots) in out.  Non-negative maxima only (a zero slot is neutral).
__device__ __forceinline__ bool dom_publish_sum_max(double s, double m, double* partials,
                                                    unsigned* counter, unsigned slot,
                                                    unsigned cnt, unsigned nitems,
                                                    double out[2])
{
    const unsigned tid = threadIdx.x + blockDim.x * threadIdx.y;
    const unsigned nthr = blockDim.x * blockDim.y;
    __shared__ bool last;
    if (tid == 0) {
        partials[(size_t)slot * 2] = s;
        partials[(size_t)slot * 2 + 1] = m;
        __threadfence();
        last = atomicAdd(counter, cnt) + cnt == nitems;
    }
    __syncthreads();
    if (!last) return false;
    __threadfence();
    double acc[2] = {0.0, 0.0};
    for (unsigned bb = tid; bb < nitems; bb += nthr) {
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

// ================================================================ 2D bodies

// Faces per run of the hyperbolic tile: the shortest run for which the x-face runs (padded
// to whole warps) and the y-face runs of a TX x TY tile take one round of NTHR threads.
__host__ __device__ constexpr int hyp_run_len(int TX, int TY, int NTHR)
{
    int r = 1;
    while (r < TX + 1 &&
           ((TX + r) / r * TY + 31) / 32 * 32 + (TY + r) / r * TX > NTHR)
        ++r;
    return r;
}

// Face-based form of the hyperbolic update for a TX x TY cell tile: the block stages the
// tile plus a 2-cell halo (h, eta, u, v) in shared memory, then every face is evaluated
// once from the edge states of the two cells next to it (each cell's minmod slopes along
// the face normal are computed once per run of faces) and stores, for the left cell, D^- + F_c(U^-) + (0, g h_L eta^-, 0) and, for the right cell,
// D^+ - F_c(U^+) - (0, g h_R eta^+, 0) (normal frame), i.e. the fluctuation plus that
// cell's half of the inner-cell term of Eq. (22) / (30).  A cell sums its four faces.
// fmx / fmy (or null): every face's mass flux F_h(U^-) + D^-_h (its left cell's output)
// into [ny][nx+1] / [ny+1][nx]; the faces a tile shares with its east / north neighbour
// are written by that neighbour.  Returns this thread's count of depth clamps.
template <typename T, int TX, int TY>
__device__ __forceinline__ int
hyp_tile(const Prm<T>& P, const T* __restrict__ eta, const T* __restrict__ q1,
          const T* __restrict__ q2, const T* __restrict__ etab, const T* __restrict__ q1b,
          const T* __restrict__ q2b, const T* __restrict__ H, T a, T b, T dt,
          T* __restrict__ eo, T* __restrict__ q1o, T* __restrict__ q2o, int bx, int by,
          T* __restrict__ fmx = nullptr, T* __restrict__ fmy = nullptr)
{
    constexpr int LW = TX + 4, LH = TY + 4, LN = LW * LH;
    constexpr int NFX = (TX + 1) * TY, NFY = TX * (TY + 1);
    __shared__ T sh[LN], se[LN], su[LN], sv[LN];
    __shared__ T CLx[3][NFX], CRx[3][NFX], CLy[3][NFY], CRy[3][NFY];
    const T d2 = P.delta * P.delta, d4 = d2 * d2;
    const T g = P.g, hdry = P.hdry;
    const int i0 = bx * TX, j0 = by * TY;
    const int tid = threadIdx.x, nt = blockDim.x;
    if (i0 >= 2 && j0 >= 2 && i0 + TX + 2 <= P.nx && j0 + TY + 2 <= P.ny) {
        // the tile and its 2-cell halo inside the grid: no boundary mapping
        for (int t = tid; t < LN; t += nt) {
            const int li = t % LW, lj = t / LW;
            const size_t k = (size_t)(j0 + lj - 2) * P.nx + (i0 + li - 2);
            const T e = eta[k];
            const T h = tmax(e + H[k], T(0));
            sh[t] = h; se[t] = e; su[t] = desing(h, q1[k], d4); sv[t] = desing(h, q2[k], d4);
        }
    } else {
        for (int t = tid; t < LN; t += nt) {
            const int li = t % LW, lj = t / LW;
            // cells more than 2 outside the domain only feed discarded faces: clamp them
            int ci = i0 + li - 2, cj = j0 + lj - 2;
            ci = ci > P.nx + 1 ? P.nx + 1 : ci;
            cj = cj > P.ny + 1 ? P.ny + 1 : cj;
            const St<T> c = load_st(P, eta, q1, q2, H, ci, cj, d4);
            sh[t] = c.h; se[t] = c.e; su[t] = c.u; sv[t] = c.v;
        }
    }
    __syncthreads();
    auto L = [&](int i, int j) { return (j + 2) * LW + (i + 2); };   // local cell index
    const T sg = qsqrt(g);
    // A thread walks a run of up to RUN consecutive faces along their normal (stride s0 in
    // the staged tile; un, ut: the staged normal and tangential velocities).  Each cell's
    // minmod slopes and edge states are computed once and carried from one face to the
    // next.  Face m of the run lies between cells k0 + m s0 and k0 + (m + 1) s0; it writes
    // its left cell's output to oL + m fs and its right cell's to oR + m fs (stride `stride`
    // between the three components).
    struct Cv { T h, e, n, t; };
    auto ld = [&](int k, const T* un, const T* ut) { return Cv{sh[k], se[k], un[k], ut[k]}; };
    // minmod slopes of cell b from its neighbours a, c and its low / high edge states
    auto recon = [&](const Cv& a, const Cv& b, const Cv& c, Cv& lo, Cv& hi) {
        const T s_h = minmod(b.h - a.h, c.h - b.h);
        const T s_n = minmod(b.n - a.n, c.n - b.n);
        const T s_t = minmod(b.t - a.t, c.t - b.t);
        const bool dry = (a.h <= hdry) | (b.h <= hdry) | (c.h <= hdry);
        const T s_e = dry ? T(0) : minmod(b.e - a.e, c.e - b.e);
        lo.h = b.h - T(0.5) * s_h; lo.e = b.e - T(0.5) * s_e;
        lo.n = b.n - T(0.5) * s_n; lo.t = b.t - T(0.5) * s_t;
        hi.h = b.h + T(0.5) * s_h; hi.e = b.e + T(0.5) * s_e;
        hi.n = b.n + T(0.5) * s_n; hi.t = b.t + T(0.5) * s_t;
    };
    constexpr int RUN = hyp_run_len(TX, TY, kThreads);
    auto run = [&](int k0, int s0, const T* un, const T* ut, int nf, T* oL, T* oR, int fs,
                   int stride) {
        Cv b = ld(k0, un, ut), c = ld(k0 + s0, un, ut), blo, bhi;
        recon(ld(k0 - s0, un, ut), b, c, blo, bhi);
#pragma unroll
        for (int m = 0; m < RUN; ++m) {
            if (m >= nf) break;
            const Cv d = ld(k0 + (m + 2) * s0, un, ut);
            Cv clo, chi;
            recon(b, c, d, clo, chi);
            T Dm[3], Dp[3];
            pvm(g, sg, hdry, bhi.h, bhi.e, bhi.n, bhi.t, clo.h, clo.e, clo.n, clo.t, Dm, Dp);
            const T qL = bhi.h * bhi.n, qR = clo.h * clo.n;
            T* o = oL + m * fs;
            o[0] = Dm[0] + qL;
            o[stride] = Dm[1] + qL * bhi.n + g * b.h * bhi.e;
            o[2 * stride] = Dm[2] + qL * bhi.t;
            o = oR + m * fs;
            o[0] = Dp[0] - qR;
            o[stride] = Dp[1] - (qR * clo.n + g * c.h * clo.e);
            o[2 * stride] = Dp[2] - qR * clo.t;
            b = c; c = d; bhi = chi;
        }
    };
    // x faces f = 0..TX between local cells f-1 and f of rows 0..TY-1, in runs of RUN faces
    // (lanes over rows); then y faces f = 0..TY between local rows f-1 and f of columns
    // 0..TX-1 (lanes over columns); the y runs start on a warp boundary
    constexpr int NRX = (TX + 1 + RUN - 1) / RUN, NRY = (TY + 1 + RUN - 1) / RUN;
    constexpr int NTX = NRX * TY, NTX32 = (NTX + 31) / 32 * 32, NT = NTX32 + NRY * TX;
    for (int t = tid; t < NT; t += nt) {
        if (t < NTX) {
            const int r = t % TY, f0 = (t / TY) * RUN;
            const int nf = TX + 1 - f0 < RUN ? TX + 1 - f0 : RUN;
            const int e = r * (TX + 1) + f0;
            run(L(f0 - 1, r), 1, su, sv, nf, &CLx[0][e], &CRx[0][e], 1, NFX);
        } else if (t >= NTX32) {
            const int u = t - NTX32, col = u % TX, f0 = (u / TX) * RUN;
            const int nf = TY + 1 - f0 < RUN ? TY + 1 - f0 : RUN;
            const int e = f0 * TX + col;
            run(L(col, f0 - 1), LW, sv, su, nf, &CLy[0][e], &CRy[0][e], TX, NFY);
        }
    }
    __syncthreads();
    if (fmx != nullptr) {
        for (int t = tid; t < NFX; t += nt) {
            const int f = t % (TX + 1), r = t / (TX + 1);
            const int I = i0 + f, j = j0 + r;
            if (j < P.ny && I <= P.nx && (f < TX || I == P.nx))
                fmx[(size_t)j * (P.nx + 1) + I] = CLx[0][t];
        }
        for (int t = tid; t < NFY; t += nt) {
            const int f = t % TX, r = t / TX;
            const int i = i0 + f, J = j0 + r;
            if (i < P.nx && J <= P.ny && (r < TY || J == P.ny))
                fmy[(size_t)J * P.nx + i] = CLy[0][t];
        }
    }
    int nclamp = 0;
    const T rx = dt / P.dx, ry = dt / P.dy;
    const T fric = dt * g * P.manning * P.manning;
    for (int t = tid; t < TX * TY; t += nt) {
        const int li = t % TX, lj = t / TX;
        const int gi = i0 + li, gj = j0 + lj;
        if (gi >= P.nx || gj >= P.ny) continue;
        const int fe = lj * (TX + 1) + li + 1, fw = fe - 1;     // x faces east / west
        const int fn = (lj + 1) * TX + li, fs = lj * TX + li;   // y faces north / south
        const size_t c = (size_t)gj * P.nx + gi;
        const T Hc = H[c];
        T en = eta[c] - rx * (CLx[0][fe] + CRx[0][fw]) - ry * (CLy[0][fn] + CRy[0][fs]);
        T an = q1[c] - rx * (CLx[1][fe] + CRx[1][fw]) - ry * (CLy[2][fn] + CRy[2][fs]);
        T bn = q2[c] - rx * (CLx[2][fe] + CRx[2][fw]) - ry * (CLy[1][fn] + CRy[1][fs]);
        T hn = en + Hc;
        if (P.manning > T(0) && hn > T(0)) {
            T u = desing(hn, an, d4), v = desing(hn, bn, d4);
            T hd = tmax(hn, P.delta);
            if constexpr (sizeof(T) == 4) {
                // FP32: hd^(-4/3) and 1 / fr from the hardware exp2 / log2 / reciprocal
                // approximations (relative error ~1e-6 at hd = delta, inside the FP32 bar)
                const float fr = 1.f + fric * qsqrt(u * u + v * v) * __powf(hd, -4.f / 3.f);
                const float ifr = qdiv(1.f, fr);
                an *= ifr;
                bn *= ifr;
            } else {
                T fr = T(1) + fric * sqrt(u * u + v * v) / (hd * cbrt(hd));
                an /= fr;
                bn /= fr;
            }
        }
        if (hn < T(0)) { en = -Hc; an = T(0); bn = T(0); ++nclamp; }
        if (a != T(0)) {
            en = a * etab[c] + b * en;
            an = a * q1b[c] + b * an;
            bn = a * q2b[c] + b * bn;
        }
        eo[c] = en; q1o[c] = an; q2o[c] = bn;
    }
    return nclamp;
}

// Breaking terms at a cell (Sec. 3 with q_x -> div q, u_x -> div u): q** = q* + de 2 nu
// (div u) grad H, centred differences, velocities desingularised, nu of Eq. (9) -- for the
// staged cell sm of a tile whose staged q* (mirror / copy ghosts with the side's parity),
// h and H (row stride SW) hold the cell and its four neighbours.
template <typename T>
__device__ __forceinline__ void break_staged(const Prm<T>& P, const T* sq1, const T* sq2,
                                             const T* hs, const T* sHH, int sm, int SW, T de,
                                             T d4, T& q1o, T& q2o)
{
    const int nb[4] = {sm - 1, sm + 1, sm - SW, sm + SW};   // W, E, S, N
    T qq[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) qq[k] = k < 2 ? sq1[nb[k]] : sq2[nb[k]];
    const T h = hs[sm];
    const T i2x = T(1) / (T(2) * P.dx), i2y = T(1) / (T(2) * P.dy);
    T dq = (qq[1] - qq[0]) * i2x + (qq[3] - qq[2]) * i2y;
    T nu = nu_break(h, dq, P.g, P.B1, P.hdry);
    q1o = sq1[sm];
    q2o = sq2[sm];
    if (nu == T(0)) return;   // no breaking here (most cells): q** = q* (up to the sign of a zero)
    T uu[4], HH[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        uu[k] = desing(hs[nb[k]], qq[k], d4);
        HH[k] = sHH[nb[k]];
    }
    T du = (uu[1] - uu[0]) * i2x + (uu[3] - uu[2]) * i2y;
    T Hx = (HH[1] - HH[0]) * i2x, Hy = (HH[3] - HH[2]) * i2y;
    q1o += de * T(2) * nu * du * Hx;
    q2o += de * T(2) * nu * du * Hy;
}
// Tiled form of the assembly for a TX x TY node tile: the block stages s = eta - H and h of
// the cells around the tile (a 2-cell ring), computes the centred differences X, Y of every
// cell once, stages the discharges of the cells touching the tile's nodes, and then builds
// each node's row, right-hand side (or defect) and w* from shared memory.  Same arithmetic
// as k_asm2d per node.
// Accumulates (||b||^2, ||D^-1 b||^2, max Gershgorin radius) of this thread's nodes in acc.
template <typename T, int TX, int TY>
__device__ __forceinline__ void
asm_tile(const Prm<T>& P, const T* __restrict__ eta, const T* __restrict__ H,
          const T* __restrict__ q1k, const T* __restrict__ q2k, const T* __restrict__ q1s,
          const T* __restrict__ q2s, const T* __restrict__ w_in, const T* __restrict__ w_b,
          T a, T b, T de, int with_coef, T* __restrict__ ws, T* __restrict__ cC,
          T* __restrict__ cW, T* __restrict__ cE, T* __restrict__ cS, T* __restrict__ cN,
          T* __restrict__ rhs, const T* __restrict__ p0, int resid_form, int bx, int by,
          double (&acc)[3], T* __restrict__ q1k_out = nullptr, T* __restrict__ q2k_out = nullptr)
{
    // staged cells: columns I0-2 .. I0+TX, rows J0-2 .. J0+TY  (SW x SH)
    constexpr int SW = TX + 3, SH = TY + 3, SN = SW * SH;
    // core cells (touching the tile's nodes): columns I0-1 .. I0+TX-1, rows J0-1 .. J0+TY-1
    constexpr int CW = TX + 1, CHh = TY + 1, CN = CW * CHh;
    __shared__ T ss[SN], hs[SN];
    // fused breaking (q1k_out set): q*, H of the staged cells; the core cells' q** are
    // computed here (break_staged) and the tile's own cells written to q1k_out / q2k_out
    const bool fuse = P.breaking && q1k_out != nullptr;
    __shared__ T sq1[SN], sq2[SN], sHH[SN];
    __shared__ T Xc[CN], Yc[CN], Q1c[CN], Q2c[CN], P1c[CN], P2c[CN];
    // previous pressure of the tile's nodes and a 1-node ring (residual form)
    constexpr int PW = TX + 2, PN = PW * (TY + 2);
    __shared__ T P0s[PN];
    const T d2 = P.delta * P.delta, d4 = d2 * d2;
    const int nxn = P.nx + 1;
    const int I0 = bx * TX, J0 = by * TY;
    const int tid = threadIdx.x, nt = blockDim.x;
    // staged cells (and the previous pressure ring, PN < SN) in rounds of NS entries per
    // thread: every load of a round is issued before its first shared store, so a 256-thread
    // block waits on one round of memory latency instead of one per loop
    constexpr int NS = 3;
    // the staged cells (and the pressure ring) all inside the grid: no boundary mapping
    const bool inner = I0 >= 2 && J0 >= 2 && I0 + TX + 1 <= P.nx && J0 + TY + 1 <= P.ny;
    for (int base = tid; base < SN; base += NS * nt) {
        T ve[NS], vH[NS], v1[NS], v2[NS], vp[NS];
        bool fx[NS], fy[NS];
#pragma unroll
        for (int k = 0; k < NS; ++k) {
            const int t = base + k * nt;
            ve[k] = vH[k] = v1[k] = v2[k] = vp[k] = T(0);
            fx[k] = fy[k] = false;
            if (t < SN) {
                const int li = t % SW, lj = t / SW;
                int ci = I0 - 2 + li, cj = J0 - 2 + lj;
                if (!inner) {
                    ci = ci > P.nx + 1 ? P.nx + 1 : ci;
                    cj = cj > P.ny + 1 ? P.ny + 1 : cj;
                    ci = map_cell(ci, P.nx, P.bcw, P.bce, fx[k]);
                    cj = map_cell(cj, P.ny, P.bcs, P.bcn, fy[k]);
                }
                const size_t m = (size_t)cj * P.nx + ci;
                ve[k] = eta[m];
                vH[k] = H[m];
                if (fuse) {
                    v1[k] = q1s[m];
                    v2[k] = q2s[m];
                }
            }
            if (resid_form && t < PN) {
                int I = I0 - 1 + t % PW, J = J0 - 1 + t / PW;
                if (!inner) {
                    I = I > P.nx + 1 ? P.nx + 1 : I;   // beyond the mirror: feeds no node of the tile
                    J = J > P.ny + 1 ? P.ny + 1 : J;
                    I = map_node(I, P.nx);
                    J = map_node(J, P.ny);
                }
                vp[k] = p0[(size_t)J * nxn + I];
            }
        }
#pragma unroll
        for (int k = 0; k < NS; ++k) {
            const int t = base + k * nt;
            if (t < SN) {
                ss[t] = ve[k] - vH[k];
                hs[t] = tmax(ve[k] + vH[k], T(0));
                if (fuse) {
                    sHH[t] = vH[k];
                    sq1[t] = fx[k] ? -v1[k] : v1[k];
                    sq2[t] = fy[k] ? -v2[k] : v2[k];
                }
            }
            if (resid_form && t < PN) P0s[t] = vp[k];
        }
    }
    if (!fuse)
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
    static_assert(PN < SN, "the pressure ring is staged with the cells");
    __syncthreads();
    for (int t = tid; t < CN; t += nt) {
        const int li = t % CW, lj = t / CW;
        const int sidx = (lj + 1) * SW + (li + 1);   // staged index of this core cell
        Xc[t] = T(0.5) * (ss[sidx + 1] - ss[sidx - 1]);
        Yc[t] = T(0.5) * (ss[sidx + SW] - ss[sidx - SW]);
        if (fuse) {
            P1c[t] = sq1[sidx];
            P2c[t] = sq2[sidx];
            const int ci = I0 - 1 + li, cj = J0 - 1 + lj;
            T b1 = T(0), b2 = T(0);
            bool rx = false, ry = false;
            if (ci <= P.nx && cj <= P.ny) {   // cells beyond the first ghost feed no node
                // a ghost cell holds its real cell's q** under the side's mirror / copy
                const int mi = inner ? ci : map_cell(ci, P.nx, P.bcw, P.bce, rx);
                const int mj = inner ? cj : map_cell(cj, P.ny, P.bcs, P.bcn, ry);
                const int sm = (mj - (J0 - 2)) * SW + (mi - (I0 - 2));
                break_staged(P, sq1, sq2, hs, sHH, sm, SW, de, d4, b1, b2);
                if (li >= 1 && lj >= 1 && ci < P.nx && cj < P.ny) {   // this tile's own cells
                    const size_t c = (size_t)cj * P.nx + ci;
                    q1k_out[c] = b1;
                    q2k_out[c] = b2;
                }
            }
            Q1c[t] = rx ? -b1 : b1;
            Q2c[t] = ry ? -b2 : b2;
        }
    }
    __syncthreads();
    const T inv2dx = T(1) / (T(2) * P.dx), inv2dy = T(1) / (T(2) * P.dy);
    const T scale = T(8) * P.dx * P.dy / de;
    const T rxl = P.dy / P.dx, ryl = P.dx / P.dy;
    // norms of the right-hand side (plain and Jacobi-scaled) summed in FP64 from the first
    // square on; the Gershgorin ratio is a max (exact in T)
    double s0 = 0.0, s1 = 0.0;
    T s2 = T(0);
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
            T nu = nu_break(hc, dq, P.g, P.B1, P.hdry);
            if (nu != T(0)) {   // the velocities only where the eddy viscosity acts
                auto u1 = [&](int k, int sx) { return desing(hs[sx], P1c[k], d4); };
                auto v1 = [&](int k, int sx) { return desing(hs[sx], P2c[k], d4); };
                T du = (u1(kb, sb) + u1(ke, se) - u1(ka, sa) - u1(kd, sd)) * inv2dx
                     + (v1(kd, sd) + v1(ke, se) - v1(ka, sa) - v1(kb, sb)) * inv2dy;
                wv += de * T(2) * nu * du * desing(hc, T(1), d4);
            }
        }
        ws[nidx] = wv;
        const T q1E = T(0.5) * (Q1c[ke] + Q1c[kb]), q1W = T(0.5) * (Q1c[kd] + Q1c[ka]);
        const T q2N = T(0.5) * (Q2c[ke] + Q2c[kd]), q2S = T(0.5) * (Q2c[kb] + Q2c[ka]);
        const T Bs = ((T(2) * hc - Xi) * q1E - (T(2) * hc + Xi) * q1W) * inv2dx
                   + ((T(2) * hc - Yi) * q2N - (T(2) * hc + Yi) * q2S) * inv2dy
                   + T(2) * hc * wv;
        const T bval = -scale * Bs;
        s0 = fma((double)bval, (double)bval, s0);
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
            const T id = qdiv(T(1), fabs(dC));
            const T bs = bval * id;
            s1 = fma((double)bs, (double)bs, s1);
            s2 = tmax(s2, (fabs(vE) + fabs(vW) + fabs(vN) + fabs(vS)) * id);
            if (resid_form) {
                const int pc = (lj + 1) * PW + li + 1;
                T mp = dC * P0s[pc];
                mp = fma(vW, P0s[pc - 1], mp);
                mp = fma(vE, P0s[pc + 1], mp);
                mp = fma(vS, P0s[pc - PW], mp);
                mp = fma(vN, P0s[pc + PW], mp);
                rhs[nidx] = bval - mp;
            } else {
                rhs[nidx] = bval;
            }
        } else {
            rhs[nidx] = bval;
        }
    }
    acc[0] += s0;
    acc[1] += s1;
    acc[2] = fmax(acc[2], (double)s2);
}

// Last block of an assembly: store the reductions, reset the solve and, for the
// Chebyshev-scheduled Jacobi, check the Gershgorin bound and prepare the first pass's weights.
__device__ __forceinline__ void asm_finish(SolveCtl* ctl, const double (&acc)[3], double tol2,
                                           int max_iter, int kpass, int with_coef)
{
    ctl->bb = acc[0];
    ctl->bdb = acc[1];
    ctl->gersh = acc[2];
    {
        int e = acc[1] > 0.0 ? ilogb(sqrt(acc[1])) : 0;
        e = e < -100 ? -100 : (e > 100 ? 100 : e);
        ctl->rscd = ldexp(1.0, -e);
        ctl->rscf = (float)ctl->rscd;
        ctl->rinv2 = ldexp(1.0, 2 * e);
    }
    ctl->tol2 = tol2;
    ctl->max_iter = max_iter;
    ctl->iter = 0;
    ctl->sweeps = 0;
    ctl->done = 0;
    ctl->status = 0;
    ctl->best = 1.0e300;
    ctl->stale = 0;
    ctl->fb = 0;
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


// One node of a Chebyshev-scheduled Jacobi sweep with every rounding fixed by explicit fused
// multiply-adds, so that all kernel forms of the pass give the same bits: the scaled
// residual r = D^-1 b - x - D^-1 (M - D) x from the node's four weights and neighbours,
// and the update x_new = x + c1 (x - x_prev) + c2 r.
template <typename T>
__device__ __forceinline__ T cheb_resid(T rb, T xc, T wW, T xW, T wE, T xE, T wS, T xS, T wN,
                                        T xN)
{
    T s = fma(wE, xE, wW * xW);
    s = fma(wS, xS, s);
    s = fma(wN, xN, s);
    return (rb - xc) - s;
}

template <typename T>
__device__ __forceinline__ T cheb_next(T xc, T xa, T c1, T c2, T r)
{
    return fma(c2, r, fma(c1, xc - xa, xc));
}

// Product that the compiler may not fuse into a later addition (the Jacobi scaling of b
// and of the weights), so that every form rounds it alike.
__device__ __forceinline__ float mul_rn(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double mul_rn(double a, double b) { return __dmul_rn(a, b); }
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
// One tile (bx, by): reads x, x_{k-1} of the tile and its halo from (xi, xpi) and writes the
// tile's new values to (xo, xpo) -- separate buffers, so that no block reads a halo that
// another block of the same pass has already advanced.  Returns the last sweep's per-thread
// sum of r^2 and max |dx| in rsum, dmax.  The Jacobi-scaled right-hand side and the four off-diagonal weights of a node are
// read only by the thread that owns the node, so they live either in shared memory (REGW =
// false: smem holds 7 region arrays) or in that thread's registers (REGW = true: smem holds
// only the two x buffers).  Both forms do the same arithmetic in the same order.
template <typename T, int NA, int NB, int BY, int K, bool REGW>
__device__ __forceinline__ void
cheb_tile(const Rows<T>& R, const T* __restrict__ b, const T* __restrict__ xi,
          const T* __restrict__ xpi, T* __restrict__ xo, T* __restrict__ xpo,
          const SolveCtl* ctl, int bx, int by, T* smem, NormAcc<T>& rsum, T& dmax)
{
    constexpr int RW = 32 * NA, RH = BY * NB, RN = RW * RH, NN = NA * NB;
    constexpr int TX = RW - 2 * K, TY = RH - 2 * K;
    T* xs0 = smem;
    T* xs1 = xs0 + RN;
    T* bd = xs1 + RN;   // (REGW = false only)
    T* wW = bd + RN;
    T* wE = wW + RN;
    T* wS = wE + RN;
    T* wN = wS + RN;
    T rbd[REGW ? NN : 1], rwW[REGW ? NN : 1], rwE[REGW ? NN : 1], rwS[REGW ? NN : 1],
        rwN[REGW ? NN : 1];
    const int nx = R.nx, ny = R.ny, NX = nx + 1;
    const int I0 = bx * TX - K, J0 = by * TY - K;
    const int tx = threadIdx.x, ty = threadIdx.y;
    T xa[NN];
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
            const int q = bb * NA + aa;
            const T ic = qdiv(T(1), R.cC[g]);
            xs0[sidx] = xi[g];
            xa[q] = xpi[g];
            const T bv = mul_rn(b[g], ic);
            const T cw = mul_rn(R.cW[g], ic), ce = mul_rn(R.cE[g], ic);
            const T cs = mul_rn(R.cS[g], ic), cn = mul_rn(R.cN[g], ic);
            if constexpr (REGW) {
                rbd[q] = bv;
                rwW[q] = fx ? ce : cw;
                rwE[q] = fx ? cw : ce;
                rwS[q] = fy ? cn : cs;
                rwN[q] = fy ? cs : cn;
            } else {
                bd[sidx] = bv;
                wW[sidx] = fx ? ce : cw;
                wE[sidx] = fx ? cw : ce;
                wS[sidx] = fy ? cn : cs;
                wN[sidx] = fy ? cs : cn;
            }
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
    // squared scaled residuals: a T partial over the thread's nodes, then FP64
    const T rsc = sizeof(T) == 4 ? (T)ctl->rscf : (T)ctl->rscd;
    T part = T(0);
    dmax = T(0);
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
                    const int q = bb * NA + aa;
                    const T xc = cur[sidx];
                    T r;
                    if constexpr (REGW)
                        r = cheb_resid(rbd[q], xc, rwW[q], cur[sidx - 1], rwE[q], cur[sidx + 1],
                                       rwS[q], cur[sidx - RW], rwN[q], cur[sidx + RW]);
                    else
                        r = cheb_resid(bd[sidx], xc, wW[sidx], cur[sidx - 1], wE[sidx],
                                       cur[sidx + 1], wS[sidx], cur[sidx - RW], wN[sidx],
                                       cur[sidx + RW]);
                    const T xn = cheb_next(xc, xa[q], c1, c2, r);
                    nxt[sidx] = xn;
                    xa[q] = xc;
                    if (sw == K - 1 && li >= K && li < RW - K && lj >= K && lj < RH - K &&
                        I0 + li <= nx && J0 + lj <= ny) {
                        {
                        const T rs = r * rsc;
                        part = fma(rs, rs, part);
                    }
                        dmax = tmax(dmax, T(fabs(xn - xc)));
                    }
                }
            }
        __syncthreads();
        T* tmp = cur; cur = nxt; nxt = tmp;
    }
    norm_zero(rsum);
    norm_add(rsum, part);   // scaled; the block applies 1 / rsc^2
#pragma unroll
    for (int bb = 0; bb < NB; ++bb)
#pragma unroll
        for (int aa = 0; aa < NA; ++aa) {
            const int li = tx + 32 * aa, lj = ty + BY * bb;
            const int gI = I0 + li, gJ = J0 + lj;
            if (li >= K && li < RW - K && lj >= K && lj < RH - K && gI <= nx && gJ <= ny) {
                const size_t g = (size_t)gJ * NX + gI;
                xo[g] = cur[lj * RW + li];
                xpo[g] = xa[bb * NA + aa];
            }
        }
}

// The zero ring around a padded (PW = RW + 2) x (RH + 2) region, for both buffers of the
// pair (the second starts PN = PW (RH + 2) elements after the first): slot t < 2 (PW + RH)
// zeroes two elements -- rows 0 and RH + 1 for t % (PW + RH) < PW, else columns 0 and
// RW + 1 of row t % (PW + RH) - PW + 1.
struct RingPair { int a, b; };

template <int RW, int RH>
__host__ __device__ constexpr RingPair pad_ring_slots(int t)
{
    constexpr int PW = RW + 2, PN = PW * (RH + 2);
    const int k = t % (PW + RH);
    const int base = t < PW + RH ? 0 : PN;
    if (k < PW) return RingPair{base + k, base + (RH + 1) * PW + k};
    const int r = k - PW + 1;
    return RingPair{base + r * PW, base + r * PW + RW + 1};
}

// every slot inside [0, 2 PN), evaluated at compile time for each region form
template <int RW, int RH>
__host__ __device__ constexpr bool pad_ring_in_bounds()
{
    constexpr int PW = RW + 2, PN = PW * (RH + 2);
    for (int t = 0; t < 2 * (PW + RH); ++t) {
        const RingPair z = pad_ring_slots<RW, RH>(t);
        if (z.a < 0 || z.b < 0 || z.a >= 2 * PN || z.b >= 2 * PN) return false;
    }
    return true;
}

// Form of cheb_tile with the weights in registers and the two x buffers padded by one node
// on every side (zeros): every sweep updates all of the thread's region nodes without
// bounds tests (values near the region edge go stale, one node per sweep, and never reach
// the tile interior within the K sweeps).  Same arithmetic for the interior nodes.
template <typename T, int NA, int NB, int BY, int K>
__device__ __forceinline__ void
cheb_tile_pad(const Rows<T>& R, const T* __restrict__ b, const T* __restrict__ xi,
              const T* __restrict__ xpi, T* __restrict__ xo, T* __restrict__ xpo,
              const SolveCtl* ctl, int bx, int by, T* smem, NormAcc<T>& rsum, T& dmax)
{
    constexpr int RW = 32 * NA, RH = BY * NB, NN = NA * NB;
    constexpr int PW = RW + 2, PN = PW * (RH + 2);
    constexpr int TX = RW - 2 * K, TY = RH - 2 * K;
    T* xs0 = smem;
    T* xs1 = xs0 + PN;
    T rbd[NN], rwW[NN], rwE[NN], rwS[NN], rwN[NN], xa[NN];
    const int nx = R.nx, ny = R.ny, NX = nx + 1;
    const int I0 = bx * TX - K, J0 = by * TY - K;
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int tid = ty * 32 + tx, nthr = 32 * BY;
    static_assert(pad_ring_in_bounds<RW, RH>(), "pad ring outside the two shared buffers");
    for (int t = tid; t < 2 * (PW + RH); t += nthr) {
        const RingPair z = pad_ring_slots<RW, RH>(t);
        xs0[z.a] = T(0);
        xs0[z.b] = T(0);
    }
#pragma unroll
    for (int bb = 0; bb < NB; ++bb)
#pragma unroll
        for (int aa = 0; aa < NA; ++aa) {
            const int li = tx + 32 * aa, lj = ty + BY * bb;
            const int gI = I0 + li, gJ = J0 + lj;
            int mI = gI < 0 ? -gI : (gI > nx ? 2 * nx - gI : gI);
            int mJ = gJ < 0 ? -gJ : (gJ > ny ? 2 * ny - gJ : gJ);
            const bool fx = mI != gI, fy = mJ != gJ;
            mI = mI < 0 ? 0 : (mI > nx ? nx : mI);
            mJ = mJ < 0 ? 0 : (mJ > ny ? ny : mJ);
            const size_t g = (size_t)mJ * NX + mI;
            const int q = bb * NA + aa;
            const T ic = qdiv(T(1), R.cC[g]);
            xs0[(lj + 1) * PW + li + 1] = xi[g];
            xa[q] = xpi[g];
            rbd[q] = mul_rn(b[g], ic);
            const T cw = mul_rn(R.cW[g], ic), ce = mul_rn(R.cE[g], ic);
            const T cs = mul_rn(R.cS[g], ic), cn = mul_rn(R.cN[g], ic);
            rwW[q] = fx ? ce : cw;
            rwE[q] = fx ? cw : ce;
            rwS[q] = fy ? cn : cs;
            rwN[q] = fy ? cs : cn;
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
    const T rsc = sizeof(T) == 4 ? (T)ctl->rscf : (T)ctl->rscd;
    T part = T(0);
    dmax = T(0);
#pragma unroll
    for (int sw = 0; sw < K; ++sw) {
        const T c1 = c1s[sw], c2 = c2s[sw];
#pragma unroll
        for (int bb = 0; bb < NB; ++bb)
#pragma unroll
            for (int aa = 0; aa < NA; ++aa) {
                const int li = tx + 32 * aa, lj = ty + BY * bb;
                const int p = (lj + 1) * PW + li + 1;
                const int q = bb * NA + aa;
                const T xc = cur[p];
                const T r = cheb_resid(rbd[q], xc, rwW[q], cur[p - 1], rwE[q], cur[p + 1], rwS[q],
                                       cur[p - PW], rwN[q], cur[p + PW]);
                const T xn = cheb_next(xc, xa[q], c1, c2, r);
                nxt[p] = xn;
                xa[q] = xc;
                if (sw == K - 1 && li >= K && li < RW - K && lj >= K && lj < RH - K &&
                    I0 + li <= nx && J0 + lj <= ny) {
                    {
                        const T rs = r * rsc;
                        part = fma(rs, rs, part);
                    }
                    dmax = tmax(dmax, T(fabs(xn - xc)));
                }
            }
        __syncthreads();
        T* tmp = cur; cur = nxt; nxt = tmp;
    }
    norm_zero(rsum);
    norm_add(rsum, part);   // scaled; the block applies 1 / rsc^2
#pragma unroll
    for (int bb = 0; bb < NB; ++bb)
#pragma unroll
        for (int aa = 0; aa < NA; ++aa) {
            const int li = tx + 32 * aa, lj = ty + BY * bb;
            const int gI = I0 + li, gJ = J0 + lj;
            if (li >= K && li < RW - K && lj >= K && lj < RH - K && gI <= nx && gJ <= ny) {
                const size_t g = (size_t)gJ * NX + gI;
                xo[g] = cur[(lj + 1) * PW + li + 1];
                xpo[g] = xa[bb * NA + aa];
            }
        }
}

// ---- Chebyshev pass with the sweeps in registers (persistent blocks, prefetched inputs)
// A region of RW = 32 C by RH = R NW nodes is swept by NW warps: warp w holds rows
// R w .. R w + R - 1, lane l columns C l .. C l + C - 1 of each, with x, x_prev, D^-1 b and
// the four off-diagonal weights of D^-1 M in registers.  Per sweep the west / east
// neighbours come from the neighbouring lanes (shuffles), the south / north ones from the
// thread's own rows, and the two rows next to another warp from a small exchange buffer
// (one barrier per sweep).  The eight input planes of the next region (x, x_prev, b and the
// five coefficients) are copied into shared memory while the current region is swept: one
// bulk copy (TMA engine, completion on an mbarrier) per plane row where the region's
// columns lie inside the grid, element copies (cp.async) with mirrored columns at the west
// and east edges.  Nodes on the region's rim use their own value for a missing neighbour:
// like every node within K of the rim they go stale, and none of them reaches the tile
// interior within K sweeps.  The node arithmetic (cheb_resid / cheb_next) is the one of
// every other form, so the iterates are the same bits.

__device__ __forceinline__ unsigned smem_u32(const void* p)
{
    return static_cast<unsigned>(__cvta_generic_to_shared(p));
}

template <int BYTES>
__device__ __forceinline__ void cp_async_elem(unsigned dst, const void* src)
{
    static_assert(BYTES == 4 || BYTES == 8, "4- or 8-byte elements");
    if constexpr (BYTES == 4)
        asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(dst), "l"(src) : "memory");
    else
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(dst), "l"(src) : "memory");
}

__device__ __forceinline__ void cp_async_commit()
{
    asm volatile("cp.async.commit_group;\n" ::: "memory");
}

__device__ __forceinline__ void cp_async_wait_all()
{
    asm volatile("cp.async.wait_group 0;\n" ::: "memory");
}

__device__ __forceinline__ void mbar_init(unsigned long long* bar, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(count)
                 : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
}

// One arrival on `bar` that also announces `bytes` of bulk copies completing on it.
__device__ __forceinline__ void mbar_arrive_expect_tx(unsigned long long* bar, unsigned bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_test_parity(unsigned long long* bar, unsigned parity)
{
    unsigned ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Wait for phase `parity` of `bar` to complete, at most `limit` polls; false on timeout.
__device__ __forceinline__ bool mbar_wait_bounded(unsigned long long* bar, unsigned parity,
                                                  unsigned limit)
{
    for (unsigned k = 0; k < limit; ++k)
        if (mbar_test_parity(bar, parity)) return true;
    return false;
}

// After a wait on `bar` ran out: wait, in bounded rounds whose length does not depend on
// the (settable) poll limit of the first wait, for bulk copies already issued on phase
// `parity` (issued = false: none were), so that the block never leaves while copies into
// its shared memory are in flight.  True in every thread when that phase completed (or
// nothing was issued); false if the drain ran out as well.
__device__ __forceinline__ bool cheb_drain(unsigned long long* bar, unsigned parity,
                                           bool issued)
{
    bool done = !issued;
    for (int round = 0; round < 8 && !done; ++round)
        done = mbar_wait_bounded(bar, parity, 1u << 22);
    cp_async_wait_all();
    return __syncthreads_and(done) != 0;
}

__device__ __forceinline__ void bulk_copy_g2s(void* dst, const void* src, unsigned bytes,
                                              unsigned long long* bar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n"
        ::"r"(smem_u32(dst)), "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

// Order this thread's shared-memory reads before later bulk copies into the same memory.
__device__ __forceinline__ void fence_proxy_async_smem()
{
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
}

// Planes of a staged region (row-major, x fastest).
enum { kPlX = 0, kPlXp, kPlB, kPlC, kPlW, kPlE, kPlS, kPlN, kPlanes };

// Staged region of RW x RH nodes: each plane row has SP = RW + A elements (A = elements per
// 16 bytes).  A row copied in bulk starts at the 16-byte boundary at or below its first node,
// which then sits at offset (first node's index mod A) of the shared row; rows staged by
// element copies start at offset 0.
template <typename T, int RW, int RH>
struct RegionGeom {
    static constexpr int A = 16 / (int)sizeof(T);
    static constexpr int SP = RW + A;
    static constexpr int PLN = SP * RH;
    static constexpr unsigned ROWB = SP * sizeof(T);   // bytes of one bulk row copy
    static_assert(ROWB % 16 == 0, "bulk copies move multiples of 16 bytes");
    // every row of a region starting at column I0 is one bulk copy inside the node array
    __device__ static bool bulk(int I0, int NX) { return I0 >= 0 && I0 + SP <= NX; }
};

template <typename T, int C, int R, int NW>
constexpr size_t cheb_reg_smem()
{
    using G = RegionGeom<T, 32 * C, R * NW>;
    return ((size_t)kPlanes * G::PLN + (size_t)2 * NW * 2 * (32 * C)) * sizeof(T);
}

__device__ __forceinline__ int mirror_node(int g, int n)
{
    int m = g < 0 ? -g : (g > n ? 2 * n - g : g);
    return m < 0 ? 0 : (m > n ? n : m);   // far outside: any node (a finite value)
}

// Offset of node row lj of region (I0, J0) in its shared row.
template <typename T, int RW, int RH>
__device__ __forceinline__ int region_row_off(int I0, int J0, int lj, int nx, int ny)
{
    using G = RegionGeom<T, RW, RH>;
    const int NX = nx + 1;
    if (!G::bulk(I0, NX)) return 0;
    return (int)(((size_t)mirror_node(J0 + lj, ny) * NX + I0) & (size_t)(G::A - 1));
}

// The same for a region inside the grid (node row J0 + lj itself, no mirror).
template <typename T, int RW, int RH>
__device__ __forceinline__ int region_row_off_in(int I0, int J, int nx)
{
    using G = RegionGeom<T, RW, RH>;
    const int NX = nx + 1;
    if (!G::bulk(I0, NX)) return 0;
    return (int)(((size_t)J * NX + I0) & (size_t)(G::A - 1));
}

// Bytes the bulk copies of region (I0, J0)'s NP planes will complete on the mbarrier (0:
// element copies).
template <typename T, int RW, int RH, int NP = kPlanes>
__device__ __forceinline__ unsigned region_bulk_bytes(int I0, int nx)
{
    using G = RegionGeom<T, RW, RH>;
    return G::bulk(I0, nx + 1) ? (unsigned)NP * RH * G::ROWB : 0u;
}

// Issue the copies of region (I0, J0)'s NP planes (nodes outside the grid read their
// mirror image, as the wall and outflow rows of M prescribe).  bases: the NP source
// arrays in plane order; planes p0 .. p1 - 1 only.  Bulk copies complete on `bar` (whose expected bytes the caller
// announced); element copies are committed as one cp.async group.
template <typename T, int RW, int RH, int NTHR, int NP = kPlanes>
__device__ __forceinline__ void cheb_stage_region(const T* const* bases, int nx, int ny,
                                                  int I0, int J0, T* planes,
                                                  unsigned long long* bar, int p0 = 0,
                                                  int p1 = NP)
{
    using G = RegionGeom<T, RW, RH>;
    const int NX = nx + 1;
    const int tid = threadIdx.x;
    if (G::bulk(I0, NX)) {
        for (int c = p0 * RH + tid; c < p1 * RH; c += NTHR) {
            const int p = c / RH, lj = c - p * RH;
            const size_t e0 = (size_t)mirror_node(J0 + lj, ny) * NX + I0;
            const size_t a0 = e0 & ~(size_t)(G::A - 1);
            bulk_copy_g2s(planes + p * G::PLN + lj * G::SP, bases[p] + a0, G::ROWB, bar);
        }
        return;
    }
    const unsigned s0 = smem_u32(planes);
    constexpr unsigned PB = G::PLN * sizeof(T);
    for (int t = tid; t < RW * RH; t += NTHR) {
        const int li = t % RW, lj = t / RW;
        const size_t g = (size_t)mirror_node(J0 + lj, ny) * NX + mirror_node(I0 + li, nx);
        const unsigned s = s0 + (unsigned)((lj * G::SP + li) * sizeof(T));
#pragma unroll
        for (int p = p0; p < p1; ++p) cp_async_elem<sizeof(T)>(s + p * PB, bases[p] + g);
    }
    cp_async_commit();
}

// One staged region (I0, J0): registers from the planes, then `stage_next(-1)` (before the
// barrier that frees the planes: fences and announces the next region's copies), then K
// sweeps, the first preceded by `stage_next(0)` (issues the next region's copies); writes
// the tile interior's x and x_prev and adds the last sweep's squared scaled residuals and
// largest change over the interior nodes to rsum / dmax.  c1s / c2s: the K sweep weights.
template <typename T, int C, int R, int NW, int K, typename F>
__device__ __forceinline__ void cheb_region_reg(const Rows<T>& Rw, const T* planes, T* exch,
                                                const T* c1s, const T* c2s, T rsc,
                                                int I0, int J0, T* __restrict__ xo,
                                                T* __restrict__ xpo, NormAcc<T>& rsum, T& dmax,
                                                F stage_next)
{
    constexpr int RW = 32 * C, RH = R * NW;
    using G = RegionGeom<T, RW, RH>;
    const int nx = Rw.nx, ny = Rw.ny, NX = nx + 1;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    T x[R][C], xa[R][C], rb[R][C], wW[R][C], wE[R][C], wS[R][C], wN[R][C];
    // registers from the planes; nodes outside the grid hold mirror images, whose W / E and
    // S / N weights swap (tested only in regions that reach past the grid)
    auto load = [&](auto edge) {
        constexpr bool E = decltype(edge)::value;
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const int lj = R * w + r, gJ = J0 + lj;
            const bool fy = E && (gJ < 0 || gJ > ny);
            const int row = lj * G::SP + (E ? region_row_off<T, RW, RH>(I0, J0, lj, nx, ny)
                                            : region_row_off_in<T, RW, RH>(I0, gJ, nx));
#pragma unroll
            for (int c = 0; c < C; ++c) {
                const int li = C * lane + c, gI = I0 + li;
                const bool fx = E && (gI < 0 || gI > nx);
                const int t = row + li;
                const T ic = qdiv(T(1), planes[kPlC * G::PLN + t]);
                x[r][c] = planes[kPlX * G::PLN + t];
                xa[r][c] = planes[kPlXp * G::PLN + t];
                rb[r][c] = mul_rn(planes[kPlB * G::PLN + t], ic);
                const T cw = mul_rn(planes[kPlW * G::PLN + t], ic);
                const T ce = mul_rn(planes[kPlE * G::PLN + t], ic);
                const T cs = mul_rn(planes[kPlS * G::PLN + t], ic);
                const T cn = mul_rn(planes[kPlN * G::PLN + t], ic);
                wW[r][c] = fx ? ce : cw;
                wE[r][c] = fx ? cw : ce;
                wS[r][c] = fy ? cn : cs;
                wN[r][c] = fy ? cs : cn;
            }
        }
    };
    if (I0 >= 0 && I0 + RW - 1 <= nx && J0 >= 0 && J0 + RH - 1 <= ny)
        load(std::false_type{});
    else
        load(std::true_type{});
    // the tile interior inside the grid (the nodes this region writes and measures)
    bool okc[C], okr[R];
#pragma unroll
    for (int c = 0; c < C; ++c) {
        const int li = C * lane + c;
        okc[c] = li >= K && li < RW - K && I0 + li <= nx;
    }
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int lj = R * w + r;
        okr[r] = lj >= K && lj < RH - K && J0 + lj <= ny;
    }
    // exchange rows of the warps above and below (the first and last warps read their own
    // edge rows back: the region's edge rows are halo)
    const int lo_row = (w > 0 ? 2 * w - 1 : 2 * w) * RW, hi_row = (w < NW - 1 ? 2 * w + 2 : 2 * w + 1) * RW;
    stage_next(-1);
    __syncthreads();   // every warp has its registers: the planes may be refilled
    stage_next(0);
    // One sweep from the iterate `cur` (and the one before it, `prv`): each node's new
    // value overwrites its own `prv` entry, which no other node reads, so the sweeps
    // alternate the two arrays' roles and no copy is made; K is even, so x ends as the
    // latest iterate and xa as the one before.
    static_assert(K % 2 == 0, "sweeps alternate the two iterate arrays");
    T part = T(0);   // squared scaled residuals of this thread's nodes (rsc: exact 2^-e)
    auto sweep = [&](T (&cur)[R][C], T (&prv)[R][C], int sw) {
        T* e = exch + (sw & 1) * (NW * 2 * RW);
        T lo[C], hi[C];
        if constexpr (sizeof(T) == 4 && C == 3) {
            // an exchange row holds the lanes' (c0, c1) pairs, then their c2 values
            auto put = [&](int row, const T (&v)[C]) {
                reinterpret_cast<float2*>(e + row)[lane] = make_float2(v[0], v[1]);
                e[row + 64 + lane] = v[2];
            };
            auto get = [&](int row, T (&v)[C]) {
                const float2 q = reinterpret_cast<const float2*>(e + row)[lane];
                v[0] = q.x;
                v[1] = q.y;
                v[2] = e[row + 64 + lane];
            };
            put((2 * w) * RW, cur[0]);
            put((2 * w + 1) * RW, cur[R - 1]);
            __syncthreads();
            get(lo_row, lo);
            get(hi_row, hi);
        } else {
#pragma unroll
            for (int c = 0; c < C; ++c) {
                e[(2 * w) * RW + C * lane + c] = cur[0][c];
                e[(2 * w + 1) * RW + C * lane + c] = cur[R - 1][c];
            }
            __syncthreads();
#pragma unroll
            for (int c = 0; c < C; ++c) {
                lo[c] = e[lo_row + C * lane + c];
                hi[c] = e[hi_row + C * lane + c];
            }
        }
        const T c1 = c1s[sw], c2 = c2s[sw];
#pragma unroll
        for (int r = 0; r < R; ++r) {
            // (lanes 0 and 31 read their own values: halo columns of the region, whose
            // errors do not reach the interior within the K sweeps)
            const T left = __shfl_up_sync(0xffffffffu, cur[r][C - 1], 1);
            const T right = __shfl_down_sync(0xffffffffu, cur[r][0], 1);
#pragma unroll
            for (int c = 0; c < C; ++c) {
                const T xc = cur[r][c];
                const T xw = c == 0 ? left : cur[r][c - 1];
                const T xe = c == C - 1 ? right : cur[r][c + 1];
                const T xs = r == 0 ? lo[c] : cur[r - 1][c];
                const T xnn = r == R - 1 ? hi[c] : cur[r + 1][c];
                const T res = cheb_resid(rb[r][c], xc, wW[r][c], xw, wE[r][c], xe, wS[r][c], xs,
                                         wN[r][c], xnn);
                const T v = cheb_next(xc, prv[r][c], c1, c2, res);
                prv[r][c] = v;
                if (sw == K - 1) {
                    if (okr[r] && okc[c]) {
                        const T rs = res * rsc;
                        part = fma(rs, rs, part);
                        dmax = tmax(dmax, T(fabs(v - xc)));
                    }
                }
            }
        }
    };
#pragma unroll
    for (int sw = 0; sw < K; sw += 2) {
        sweep(x, xa, sw);
        sweep(xa, x, sw + 1);
    }
    norm_add(rsum, part);   // scaled; the block applies 1 / rsc^2
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int gJ = J0 + R * w + r;
#pragma unroll
        for (int c = 0; c < C; ++c) {
            const int gI = I0 + C * lane + c;
            if (okr[r] && okc[c]) {
                const size_t g = (size_t)gJ * NX + gI;
                xo[g] = x[r][c];
                xpo[g] = xa[r][c];
            }
        }
    }
}

// Packed FP32 form of cheb_region_reg for C = 2: a lane's two columns are one float2 and
// every sweep operation acts on both with one Blackwell packed instruction (FFMA2 / FMUL2;
// differences as fma(a, -1, b), which rounds like b - a).  Each packed lane rounds like the
// scalar code, so the iterates are the same bits as every other form's.
template <int R, int NW, int K, typename F>
__device__ __forceinline__ void cheb_region_reg2(const Rows<float>& Rw, const float* planes,
                                                 float* exch, const float* c1s,
                                                 const float* c2s, float rsc,
                                                 int I0, int J0, float* __restrict__ xo,
                                                 float* __restrict__ xpo, SumDS& rsum,
                                                 float& dmax, F stage_next)
{
    constexpr int RW = 64, RH = R * NW;
    using G = RegionGeom<float, RW, RH>;
    const int nx = Rw.nx, ny = Rw.ny, NX = nx + 1;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const float2 m1 = make_float2(-1.f, -1.f);
    float2 x[R], xa[R], rb[R], wW[R], wE[R], wS[R], wN[R];
    const int gI0 = I0 + 2 * lane, gI1 = gI0 + 1;
    const bool fx0 = gI0 < 0 || gI0 > nx, fx1 = gI1 < 0 || gI1 > nx;
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int lj = R * w + r, gJ = J0 + lj;
        const bool fy = gJ < 0 || gJ > ny;
        const int off = region_row_off<float, RW, RH>(I0, J0, lj, nx, ny);
        const int t = lj * G::SP + off + 2 * lane;
        // an odd row offset leaves the pair 4-byte aligned only
        auto ld = [&](int plane) {
            const float* q = planes + plane * G::PLN + t;
            return (off & 1) ? make_float2(q[0], q[1]) : *reinterpret_cast<const float2*>(q);
        };
        const float2 cc = ld(kPlC);
        const float2 ic = make_float2(qdiv(1.f, cc.x), qdiv(1.f, cc.y));
        x[r] = ld(kPlX);
        xa[r] = ld(kPlXp);
        rb[r] = __fmul2_rn(ld(kPlB), ic);
        const float2 cw = __fmul2_rn(ld(kPlW), ic), ce = __fmul2_rn(ld(kPlE), ic);
        const float2 cs = __fmul2_rn(ld(kPlS), ic), cn = __fmul2_rn(ld(kPlN), ic);
        wW[r] = make_float2(fx0 ? ce.x : cw.x, fx1 ? ce.y : cw.y);
        wE[r] = make_float2(fx0 ? cw.x : ce.x, fx1 ? cw.y : ce.y);
        wS[r] = fy ? cn : cs;
        wN[r] = fy ? cs : cn;
    }
    stage_next(-1);
    __syncthreads();   // every warp has its registers: the planes may be refilled
    stage_next(0);
    // sweeps alternate the roles of x and xa, as in cheb_region_reg (no copies)
    static_assert(K % 2 == 0, "sweeps alternate the two iterate arrays");
    float part = 0.f;   // squared scaled residuals of this thread's nodes (rsc: exact 2^-e)
    auto sweep = [&](float2 (&cur)[R], float2 (&prv)[R], int sw) {
        float* e = exch + (sw & 1) * (NW * 2 * RW);
        *reinterpret_cast<float2*>(e + (2 * w) * RW + 2 * lane) = cur[0];
        *reinterpret_cast<float2*>(e + (2 * w + 1) * RW + 2 * lane) = cur[R - 1];
        __syncthreads();
        const float2 lo = w > 0 ? *reinterpret_cast<const float2*>(e + (2 * w - 1) * RW + 2 * lane)
                                : cur[0];
        const float2 hi = w < NW - 1
                              ? *reinterpret_cast<const float2*>(e + (2 * w + 2) * RW + 2 * lane)
                              : cur[R - 1];
        const float2 c1 = make_float2(c1s[sw], c1s[sw]), c2 = make_float2(c2s[sw], c2s[sw]);
#pragma unroll
        for (int r = 0; r < R; ++r) {
            float left = __shfl_up_sync(0xffffffffu, cur[r].y, 1);
            float right = __shfl_down_sync(0xffffffffu, cur[r].x, 1);
            if (lane == 0) left = cur[r].x;
            if (lane == 31) right = cur[r].y;
            const float2 xw = make_float2(left, cur[r].x), xe = make_float2(cur[r].y, right);
            const float2 xs = r == 0 ? lo : cur[r - 1];
            const float2 xnn = r == R - 1 ? hi : cur[r + 1];
            float2 s = __ffma2_rn(wE[r], xe, __fmul2_rn(wW[r], xw));
            s = __ffma2_rn(wS[r], xs, s);
            s = __ffma2_rn(wN[r], xnn, s);
            const float2 res = __ffma2_rn(s, m1, __ffma2_rn(cur[r], m1, rb[r]));
            const float2 v =
                __ffma2_rn(c2, res, __ffma2_rn(c1, __ffma2_rn(prv[r], m1, cur[r]), cur[r]));
            if (sw == K - 1) {
                const int lj = R * w + r;
                if (lj >= K && lj < RH - K && J0 + lj <= ny) {
                    const int li = 2 * lane;
                    if (li >= K && li < RW - K && gI0 <= nx) {
                        const float rs = res.x * rsc;
                        part = fmaf(rs, rs, part);
                        dmax = fmaxf(dmax, fabsf(v.x - cur[r].x));
                    }
                    if (li + 1 >= K && li + 1 < RW - K && gI1 <= nx) {
                        const float rs = res.y * rsc;
                        part = fmaf(rs, rs, part);
                        dmax = fmaxf(dmax, fabsf(v.y - cur[r].y));
                    }
                }
            }
            prv[r] = v;
        }
    };
#pragma unroll
    for (int sw = 0; sw < K; sw += 2) {
        sweep(x, xa, sw);
        sweep(xa, x, sw + 1);
    }
    norm_add(rsum, part);   // scaled; the block applies 1 / rsc^2
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int lj = R * w + r, gJ = J0 + lj;
        if (lj < K || lj >= RH - K || gJ > ny) continue;
        const int li = 2 * lane;
        const size_t g = (size_t)gJ * NX + gI0;
        if (li >= K && li < RW - K && gI0 <= nx) { xo[g] = x[r].x; xpo[g] = xa[r].x; }
        if (li + 1 >= K && li + 1 < RW - K && gI1 <= nx) { xo[g + 1] = x[r].y; xpo[g + 1] = xa[r].y; }
    }
}

// Planes of a region staged for the cyclic form of the pass (one iterate, no x_prev).
// The coefficient planes come first: a region reads them into registers and releases them
// (planes 0 .. kRbRows - 1) before it reads x and b.
enum { kRbC = 0, kRbW, kRbE, kRbS, kRbN, kRbRows, kRbX = kRbRows, kRbB, kRbPlanes };

template <typename T, int R, int NW>
constexpr size_t cheb_rb_smem()
{
    using G = RegionGeom<T, 64, R * NW>;
    static_assert((kRbPlanes * G::PLN * sizeof(T)) % 16 == 0, "exchange rows 16-byte aligned");
    return ((size_t)kRbPlanes * G::PLN + (size_t)2 * NW * 2 * 64) * sizeof(T);
}

template <typename T> struct Pair2;
template <> struct Pair2<float> { using V = float2; };
template <> struct Pair2<double> { using V = double2; };

// Cyclic form of the Chebyshev-scheduled Jacobi pass: regions of 64 x (R NW) nodes, two
// columns per lane, R rows per warp (R even), K steps per pass (K even).
//   A row of M couples a node with its four neighbours only, and they have the other colour
// (I + J) mod 2 (so do mirror images: a node and its image lie an even number of nodes
// apart), so D^-1 (M - D) maps each colour to the other.  The Chebyshev interval
// [1 - g, 1 + g] is centred at 1, so the weights satisfy c1 = c2 - 1 and the step
// x_{k+1} = x_k + c1 (x_k - x_{k-1}) + c2 r_k equals c2 (D^-1 b - D^-1 (M - D) x_k) +
// (1 - c2) x_{k-1}: a node at step k + 1 needs its neighbours at step k and itself at step
// k - 1 only.  One colour at the odd steps and the other at the even steps therefore form a
// closed recurrence (the cyclic Chebyshev semi-iterative method of Golub and Varga, 1961),
// computed here in place: step s of a solve updates the nodes of colour s mod 2 by
// x <- x + c2 r, r = D^-1 b - x - D^-1 (M - D) x their scaled residual.  A step touches
// half the nodes of a Jacobi sweep and the pass carries one iterate; every node takes the
// values of the full iteration at the steps of its colour (up to rounding).
//   K is even, so each pass starts with colour 1.  The pass writes x of the tile interior
// (colour 0 at step K, colour 1 at step K - 1) and measures the vector of colour 0 at step
// K - 2 and colour 1 at step K - 1, whose scaled residual is (1 - c2) r at the colour-1
// nodes of step K - 1 and r at the colour-0 nodes of step K.
//   stage_next(-1): fence this thread's plane reads and announce the next region's bytes
// (before the barrier that releases the coefficient planes); stage_next(1): issue the copies
// of those planes; stage_next(-2): fence the reads of x and b; stage_next(2), after the
// first step's barrier: issue the copies of the x and b planes.
template <typename T, int R, int NW, int K, typename F>
__device__ __forceinline__ void cheb_region_rb(const Rows<T>& Rw, const T* planes, T* exch,
                                               const T* c2s, T rsc, int I0, int J0,
                                               T* __restrict__ xo, NormAcc<T>& rsum, T& dmax,
                                               F stage_next)
{
    constexpr int RW = 64, RH = R * NW;
    static_assert(R % 2 == 0 && K % 2 == 0, "colours uniform over the block; passes of even length");
    using G = RegionGeom<T, RW, RH>;
    using V2 = typename Pair2<T>::V;
    const int nx = Rw.nx, ny = Rw.ny, NX = nx + 1;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    T x[R][2], rb[R][2], wW[R][2], wE[R][2], wS[R][2], wN[R][2];
    // registers from the planes in two groups, the coefficients first (their planes are
    // released, and the next region's copies into them issued, while x and b are read);
    // nodes outside the grid hold mirror images, whose W / E and S / N weights swap (tested
    // only in regions that reach past the grid).  rb holds 1 / cC until b is read.
    const bool edge = !(I0 >= 0 && I0 + RW - 1 <= nx && J0 >= 0 && J0 + RH - 1 <= ny);
    auto rows = [&](auto e, auto body) {
        constexpr bool E = decltype(e)::value;
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const int lj = R * w + r, gJ = J0 + lj;
            const bool fy = E && (gJ < 0 || gJ > ny);
            const int row = lj * G::SP + (E ? region_row_off<T, RW, RH>(I0, J0, lj, nx, ny)
                                            : region_row_off_in<T, RW, RH>(I0, gJ, nx));
#pragma unroll
            for (int c = 0; c < 2; ++c) {
                const int gI = I0 + 2 * lane + c;
                body(r, c, row + 2 * lane + c, E && (gI < 0 || gI > nx), fy);
            }
        }
    };
    auto coef = [&](int r, int c, int t, bool fx, bool fy) {
        const T ic = qdiv(T(1), planes[kRbC * G::PLN + t]);
        rb[r][c] = ic;
        const T cw = mul_rn(planes[kRbW * G::PLN + t], ic);
        const T ce = mul_rn(planes[kRbE * G::PLN + t], ic);
        const T cs = mul_rn(planes[kRbS * G::PLN + t], ic);
        const T cn = mul_rn(planes[kRbN * G::PLN + t], ic);
        wW[r][c] = fx ? ce : cw;
        wE[r][c] = fx ? cw : ce;
        wS[r][c] = fy ? cn : cs;
        wN[r][c] = fy ? cs : cn;
    };
    auto state = [&](int r, int c, int t, bool, bool) {
        x[r][c] = planes[kRbX * G::PLN + t];
        rb[r][c] = mul_rn(planes[kRbB * G::PLN + t], rb[r][c]);
    };
    if (edge) rows(std::true_type{}, coef); else rows(std::false_type{}, coef);
    stage_next(-1);
    __syncthreads();   // the coefficient planes may be refilled
    stage_next(1);
    if (edge) rows(std::true_type{}, state); else rows(std::false_type{}, state);
    bool okc[2], okr[R];   // the tile interior inside the grid
#pragma unroll
    for (int c = 0; c < 2; ++c) {
        const int li = 2 * lane + c;
        okc[c] = li >= K && li < RW - K && I0 + li <= nx;
    }
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int lj = R * w + r;
        okr[r] = lj >= K && lj < RH - K && J0 + lj <= ny;
    }
    const int lo_row = (w > 0 ? 2 * w - 1 : 2 * w) * RW, hi_row = (w < NW - 1 ? 2 * w + 2 : 2 * w + 1) * RW;
    stage_next(-2);   // this thread's reads of x and b are done: the first step's barrier
                      // releases those planes
    T part = T(0);   // squared scaled residuals of this thread's nodes (rsc: exact 2^-e)
    // node (r, c) of this thread has colour (I0 + J0 + R w + r + c) mod 2; R is even, so
    // the block's colours are fixed by Q = (I0 + J0) mod 2
    auto steps = [&](auto qc) {
        constexpr int Q = decltype(qc)::value;
#pragma unroll
        for (int sw = 0; sw < K; ++sw) {
            T* e = exch + (sw & 1) * (NW * 2 * RW);
            reinterpret_cast<V2*>(e + (2 * w) * RW)[lane] = V2{x[0][0], x[0][1]};
            reinterpret_cast<V2*>(e + (2 * w + 1) * RW)[lane] = V2{x[R - 1][0], x[R - 1][1]};
            __syncthreads();
            if (sw == 0) stage_next(2);   // the x and b planes of the next region
            const V2 lo2 = reinterpret_cast<const V2*>(e + lo_row)[lane];
            const V2 hi2 = reinterpret_cast<const V2*>(e + hi_row)[lane];
            const T lo[2] = {lo2.x, lo2.y}, hi[2] = {hi2.x, hi2.y};
            const T c2 = c2s[sw];
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const int cu = (Q + r + sw + 1) & 1;   // the column of colour (sw + 1) mod 2
                // (lanes 0 and 31 read their own values: halo columns of the region, whose
                // errors do not reach the interior within the K steps)
                T xw, xe;
                if (cu == 0) {
                    xw = __shfl_up_sync(0xffffffffu, x[r][1], 1);
                    xe = x[r][1];
                } else {
                    xw = x[r][0];
                    xe = __shfl_down_sync(0xffffffffu, x[r][0], 1);
                }
                const T xs = r == 0 ? lo[cu] : x[r - 1][cu];
                const T xn = r == R - 1 ? hi[cu] : x[r + 1][cu];
                const T xc = x[r][cu];
                const T res = cheb_resid(rb[r][cu], xc, wW[r][cu], xw, wE[r][cu], xe,
                                         wS[r][cu], xs, wN[r][cu], xn);
                const T v = fma(c2, res, xc);
                x[r][cu] = v;
                if (sw >= K - 2) {
                    if (okr[r] && okc[cu]) {
                        const T rz = (sw == K - 2 ? (T(1) - c2) * res : res) * rsc;
                        part = fma(rz, rz, part);
                        dmax = tmax(dmax, T(fabs(v - xc)));
                    }
                }
            }
        }
    };
    if (((I0 + J0) & 1) == 0)
        steps(std::integral_constant<int, 0>{});
    else
        steps(std::integral_constant<int, 1>{});
    norm_add(rsum, part);   // scaled; the block applies 1 / rsc^2
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int gJ = J0 + R * w + r;
#pragma unroll
        for (int c = 0; c < 2; ++c) {
            const int gI = I0 + 2 * lane + c;
            if (okr[r] && okc[c]) xo[(size_t)gJ * NX + gI] = x[r][c];
        }
    }
}

// Last block of a pass: residual test (or criterion (32) on max |dx|), and the next K weights.
__device__ __forceinline__ void cheb_finish(SolveCtl* ctl, const double (&acc)[2], int K)
{
    if (ctl->status >= 6) {   // a block of the register form gave up waiting for its copies
        ctl->done = 1;
        return;
    }
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

// cheb_finish plus the stall test of the passes: 8 passes without a 0.81 reduction of the
// best residual (0.99 under criterion (32), where only a residual that no longer falls at
// all counts) end the relaxation with status 5 (the rounding floor of the precision, or a
// spectrum the Gershgorin interval does not describe); BiCGStab then continues from the
// current iterate.
__device__ __forceinline__ void cheb_finish_stall(SolveCtl* ctl, const double (&acc)[2], int K)
{
    cheb_finish(ctl, acc, K);
    if (!ctl->done) {
        const double fall = ctl->eps_dp > 0.0 ? 0.99 : 0.81;
        if (acc[0] < fall * ctl->best) { ctl->best = acc[0]; ctl->stale = 0; }
        else if (++ctl->stale >= 8) { ctl->done = 1; ctl->status = 5; }
    }
}

// Correction (Eq. 36 and the w update of Eq. 41) at node (I, J) and cell (I, J):
// q1 += de (T^Hor_N + T^Hor_S)/2, q2 += de (T^Ver_E + T^Ver_W)/2, w += de p / h_c;
// with P.dry_zero, dry cells (h <= hdry) keep q = 0, as App. B A.2 assumes where the depth
// vanishes; without it the correction acts on every cell, as Sec. 4.5 states.
// In the final stage also the Eq. (23) rate max((|u|+c)/dx + (|v|+c)/dy); lam and bad
// accumulate the final-stage rate and the non-finite flag.
// Tiled for a TX x TY tile of nodes (and the cells with the same (i, j)): the block stages
// eta and H of the cells around the tile (a 1-cell ring) and p + dp of the tile's nodes
// plus one row and column, so each value is loaded once per tile.
template <typename T, int TX, int TY>
__device__ __forceinline__ void
corr_tile(const Prm<T>& P, const T* __restrict__ eta, const T* __restrict__ H,
          const T* __restrict__ q1k, const T* __restrict__ q2k, const T* __restrict__ ws,
          const T* __restrict__ p, const T* __restrict__ dp, T* __restrict__ pout, T de,
          int with_p, T* __restrict__ eo, T* __restrict__ q1o, T* __restrict__ q2o,
          T* __restrict__ wo, int final_stage, int bx, int by, T& lam, int& bad)
{
    constexpr int CW = TX + 2, CH = TY + 2, CN = CW * CH;   // cells I0-1 .. I0+TX
    constexpr int NW = TX + 1, NH = TY + 1, NNd = NW * NH;  // nodes I0 .. I0+TX
    __shared__ T se[CN], sH[CN], pn[NNd];
    const T d2 = P.delta * P.delta, d4 = d2 * d2;
    const int nx = P.nx, ny = P.ny, nxn = nx + 1;
    const int I0 = bx * TX, J0 = by * TY;
    const int tid = threadIdx.x, nt = blockDim.x;
    // the thread's own node / cell operands (node t = tid + k nt), loaded before the staging
    // so that their latency overlaps it (nt = kCorrThreads)
    constexpr int NPT = (TX * TY + kCorrThreads - 1) / kCorrThreads;
    T wsv[NPT], a1v[NPT], a2v[NPT];
#pragma unroll
    for (int k = 0; k < NPT; ++k) {
        const int t = tid + k * kCorrThreads;
        const int I = I0 + t % TX, J = J0 + t / TX;
        wsv[k] = a1v[k] = a2v[k] = T(0);
        if (t < TX * TY && I <= nx && J <= ny) {
            wsv[k] = ws[(size_t)J * nxn + I];
            if (I < nx && J < ny) {
                a1v[k] = q1k[(size_t)J * nx + I];
                a2v[k] = q2k[(size_t)J * nx + I];
            }
        }
    }
    // staged cells and nodes (NNd < CN) in rounds of NS entries per thread, all loads of a
    // round issued before its first shared store (one round of memory latency per tile)
    static_assert(NNd < CN, "the nodes are staged with the cells");
    constexpr int NS = 2;
    // the staged cells and nodes all inside the grid: no boundary mapping
    const bool inner = I0 >= 1 && J0 >= 1 && I0 + TX + 1 <= nx && J0 + TY + 1 <= ny;
    for (int base = tid; base < CN; base += NS * nt) {
        T ve[NS], vH[NS], vp[NS], vd[NS];
#pragma unroll
        for (int k = 0; k < NS; ++k) {
            const int t = base + k * nt;
            ve[k] = vH[k] = vp[k] = vd[k] = T(0);
            if (t < CN) {
                const int li = t % CW, lj = t / CW;
                int ci = I0 - 1 + li, cj = J0 - 1 + lj;
                if (!inner) {
                    ci = ci > nx + 1 ? nx + 1 : ci;
                    cj = cj > ny + 1 ? ny + 1 : cj;
                    bool rx, ry;
                    ci = map_cell(ci, nx, P.bcw, P.bce, rx);
                    cj = map_cell(cj, ny, P.bcs, P.bcn, ry);
                }
                const size_t m = (size_t)cj * nx + ci;
                ve[k] = eta[m];
                vH[k] = H[m];
            }
            if (with_p && t < NNd) {
                const int I = I0 + t % NW, J = J0 + t / NW;
                const size_t m = inner ? (size_t)J * nxn + I
                                       : (size_t)(J > ny ? ny : J) * nxn + (I > nx ? nx : I);
                vp[k] = p[m];
                vd[k] = dp[m];
            }
        }
#pragma unroll
        for (int k = 0; k < NS; ++k) {
            const int t = base + k * nt;
            if (t < CN) {
                se[t] = ve[k];
                sH[t] = vH[k];
            }
            if (with_p && t < NNd) pn[t] = vp[k] + vd[k];
        }
    }
    __syncthreads();
    const T idx_ = T(1) / P.dx, idy_ = T(1) / P.dy;
#pragma unroll
    for (int k = 0; k < NPT; ++k) {
        const int t = tid + k * kCorrThreads;
        const int li = t % TX, lj = t / TX;
        const int I = I0 + li, J = J0 + lj;
        if (t >= TX * TY || I > nx || J > ny) continue;
        const size_t nidx = (size_t)J * nxn + I;
        const int ca = lj * CW + li;   // staged cell (I-1, J-1); b = ca + 1, d = ca + CW, e = d + 1
        // node
        T pc = T(0);
        if (with_p) {
            pc = pn[lj * NW + li];
            const T hs = tmax(se[ca] + sH[ca], T(0)) + tmax(se[ca + 1] + sH[ca + 1], T(0)) +
                         tmax(se[ca + CW] + sH[ca + CW], T(0)) +
                         tmax(se[ca + CW + 1] + sH[ca + CW + 1], T(0));
            const T hc = T(0.25) * hs;
            const T wn = wsv[k] + de * pc * desing(hc, T(1), d4);
            wo[nidx] = wn;
            pout[nidx] = pc;
            if (!isfinite(wn) || !isfinite(pc)) bad = 1;
        } else {
            wo[nidx] = wsv[k];
            pout[nidx] = T(0);
        }
        // cell (i, j) = (I, J)
        if (I < nx && J < ny) {
            const size_t c = (size_t)J * nx + I;
            const int ce = ca + CW + 1;   // staged cell (I, J)
            const T e = se[ce], Hc = sH[ce];
            const T h = tmax(e + Hc, T(0));
            T a1 = a1v[k], a2 = a2v[k];
            if (with_p) {
                const T X = T(0.5) * ((se[ce + 1] - sH[ce + 1]) - (se[ce - 1] - sH[ce - 1]));
                const T Y = T(0.5) * ((se[ce + CW] - sH[ce + CW]) - (se[ce - CW] - sH[ce - CW]));
                const int nsw = lj * NW + li;
                const T pSW = pn[nsw], pSE = pn[nsw + 1];
                const T pNW = pn[nsw + NW], pNE = pn[nsw + NW + 1];
                const T TN = (-T(0.5) * h * (pNE - pNW) - T(0.25) * (pNE + pNW) * X) * idx_;
                const T TS = (-T(0.5) * h * (pSE - pSW) - T(0.25) * (pSE + pSW) * X) * idx_;
                const T TE = (-T(0.5) * h * (pNE - pSE) - T(0.25) * (pNE + pSE) * Y) * idy_;
                const T TW = (-T(0.5) * h * (pNW - pSW) - T(0.25) * (pNW + pSW) * Y) * idy_;
                a1 += de * T(0.5) * (TN + TS);
                a2 += de * T(0.5) * (TE + TW);
            }
            if (P.dry_zero && h <= P.hdry) { a1 = T(0); a2 = T(0); }   // dry cells: no discharge
            eo[c] = e; q1o[c] = a1; q2o[c] = a2;
            if (!isfinite(e) || !isfinite(a1) || !isfinite(a2)) bad = 1;
            if (final_stage) {
                const T u = desing(h, a1, d4), v = desing(h, a2, d4), cw = qsqrt(P.g * h);
                lam = tmax(lam, (fabs(u) + cw) * (T(1) / P.dx) + (fabs(v) + cw) * (T(1) / P.dy));
            }
        }
    }
}

// Eq. (23) rate of cell idx: (|u| + c)/dx, plus (|v| + c)/dy in 2D.
template <typename T>
__device__ __forceinline__ double lambda_cell(const Prm<T>& P, int dim, const T* __restrict__ eta,
                                              const T* __restrict__ q1, const T* __restrict__ q2,
                                              const T* __restrict__ H, long long idx)
{
    const T d2 = P.delta * P.delta, d4 = d2 * d2;
    const T h = tmax(eta[idx] + H[idx], T(0));
    const T cw = sqrt(P.g * h);
    const T u = desing(h, q1[idx], d4);
    double lv = (fabs(u) + cw) / P.dx;
    if (dim == 2) lv += (fabs(desing(h, q2[idx], d4)) + cw) / P.dy;
    return lv;
}

}  // namespace dev
}  // namespace nh
