// nh_kernels.cu -- sm_103a kernels of one non-hydrostatic shallow-water time step
// (Escalante, Morales de Luna & Castro, arXiv:1706.04551).
//
// Single-domain kernels: the tile and element bodies of nh_device.cuh mapped to blockIdx
// (tiled kernels) or to a grid-stride loop over cells or nodes on a grid sized to a multiple
// of the SM count (element kernels), plus the 1D, BiCGStab and utility kernels.  State
// precision T is float or double.
#include "nh_device.cuh"

#include <cuda_runtime.h>
#include <stdint.h>

namespace nh {
namespace {

using namespace dev;

// ================================================================ 2D kernels

template <typename T, int TX, int TY>
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? 5 : 2)
k_hyp2d_t(Prm<T> P, const T* __restrict__ eta, const T* __restrict__ q1,
          const T* __restrict__ q2, const T* __restrict__ etab, const T* __restrict__ q1b,
          const T* __restrict__ q2b, const T* __restrict__ H, T a, T b, T dt,
          T* __restrict__ eo, T* __restrict__ q1o, T* __restrict__ q2o, StepCtl* st,
          T* __restrict__ fmx, T* __restrict__ fmy, const double* dtd)
{
    if (dtd) dt = (T)*dtd;   // captured steps: the step's dt from device memory
    const int nclamp = hyp_tile<T, TX, TY>(P, eta, q1, q2, etab, q1b, q2b, H, a, b, dt, eo, q1o,
                                           q2o, blockIdx.x, blockIdx.y, fmx, fmy);
    if (nclamp) atomicAdd(&st->clamped, nclamp);
}

// w* of the energy-consistent w equation (hw)_t + div(hw u) = p (Sec. 2, the system of
// the paper's reference [7]) for a TX x TY tile of nodes.  Node (I, J) owns the dual cell
// [x_I - dx/2, x_I + dx/2] x [y_J - dy/2, y_J + dy/2] clipped to the domain (area fraction
// ax * ay), a quarter of each cell around it.  Its east face runs along the centre lines
// of the cells (I, J-1), (I, J) inside the grid, through half of each, where the x mass
// flux is the mean of the cell's two x-face fluxes; on the domain boundary the dual face
// is the boundary face.  w is taken upwind (the node's own at boundary faces), and
//   (hw)* = a h_b w_b + b (h w - dt div(F w)),   w* = (hw)* / h*  (desingularised),
// with the node depths (mean of the four cells, outside cells mapped onto their wall /
// outflow images) of the base, input and combined states.  Those dual fluxes move the
// dual depth exactly as the cell depths move, so a uniform w stays uniform.  The block
// stages the depths of the cells around the tile, the face fluxes next to it and w of
// the tile with a 1-node ring.
template <typename T, int TX, int TY, int NT>
__global__ void __launch_bounds__(NT)
k_wtrans2d_t(Prm<T> P, const T* __restrict__ etab, const T* __restrict__ etain,
             const T* __restrict__ etas, const T* __restrict__ H, const T* __restrict__ wb,
             const T* __restrict__ win, const T* __restrict__ fmx, const T* __restrict__ fmy,
             T a, T b, T dt, T* __restrict__ wo, const double* dtd)
{
    if (dtd) dt = (T)*dtd;
    constexpr int CW = TX + 1, CN = CW * (TY + 1);          // cells I0-1.., J0-1..
    constexpr int XW = TX + 2, XN = XW * (TY + 1);          // x faces I0-1..I0+TX
    constexpr int YW = TX + 1, YN = YW * (TY + 2);          // y faces J0-1..J0+TY
    constexpr int WW = TX + 2, WN = WW * (TY + 2);          // nodes with a 1-node ring
    // every thread stages at most NS entries of each array and issues all its loads
    // before the first store, so the block waits on one round of memory latency
    constexpr int NS = (WN + NT - 1) / NT;
    static_assert(CN <= NS * NT && XN <= NS * NT && YN <= NS * NT, "staging slots");
    static_assert((TX * TY) % NT == 0, "whole nodes per thread");
    __shared__ T hB[CN], hI[CN], hS[CN], sx[XN], sy[YN], sw[WN];
    const T d2 = P.delta * P.delta, d4 = d2 * d2;
    const int nx = P.nx, ny = P.ny, nxn = nx + 1;
    const int I0 = blockIdx.x * TX, J0 = blockIdx.y * TY;
    const int tid = threadIdx.x;
    T vb[NS], vi[NS], vs[NS], vh[NS], vx[NS], vy[NS], vw[NS];
#pragma unroll
    for (int k = 0; k < NS; ++k) {
        const int t = tid + k * NT;
        vb[k] = vi[k] = vs[k] = vh[k] = vx[k] = vy[k] = vw[k] = T(0);
        if (t < CN) {
            int ci = I0 - 1 + t % CW, cj = J0 - 1 + t / CW;
            ci = ci > nx ? nx : ci;   // beyond the first ghost: feeds no node of the tile
            cj = cj > ny ? ny : cj;
            bool r;
            const int ii = map_cell(ci, nx, P.bcw, P.bce, r);
            const int jj = map_cell(cj, ny, P.bcs, P.bcn, r);
            const size_t m = (size_t)jj * nx + ii;
            vh[k] = H[m]; vb[k] = etab[m]; vi[k] = etain[m]; vs[k] = etas[m];
        }
        if (t < XN) {   // faces outside the grid carry nothing
            const int If = I0 - 1 + t % XW, j = J0 - 1 + t / XW;
            if (If >= 0 && If <= nx && j >= 0 && j < ny) vx[k] = fmx[(size_t)j * nxn + If];
        }
        if (t < YN) {
            const int i = I0 - 1 + t % YW, Jf = J0 - 1 + t / YW;
            if (i >= 0 && i < nx && Jf >= 0 && Jf <= ny) vy[k] = fmy[(size_t)Jf * nx + i];
        }
        if (t < WN) {
            const int I = I0 - 1 + t % WW, J = J0 - 1 + t / WW;
            if (I >= 0 && I <= nx && J >= 0 && J <= ny) vw[k] = win[(size_t)J * nxn + I];
        }
    }
#pragma unroll
    for (int k = 0; k < NS; ++k) {
        const int t = tid + k * NT;
        if (t < CN) {
            hB[t] = tmax(vb[k] + vh[k], T(0));
            hI[t] = tmax(vi[k] + vh[k], T(0));
            hS[t] = tmax(vs[k] + vh[k], T(0));
        }
        if (t < XN) sx[t] = vx[k];
        if (t < YN) sy[t] = vy[k];
        if (t < WN) sw[t] = vw[k];
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < TX * TY / NT; ++r) {
        const int li = tid % TX, lj = tid / TX + r * (NT / TX);
        const int I = I0 + li, J = J0 + lj;
        if (I > nx || J > ny) continue;
        // cells (I-1, J-1), (I, J-1), (I-1, J), (I, J) at ka, ka + 1, ka + CW, ka + CW + 1
        const int ka = lj * CW + li;
        auto depth = [&](const T* h) {
            return T(0.25) * (((h[ka] + h[ka + 1]) + h[ka + CW]) + h[ka + CW + 1]);
        };
        // column sums of the x faces I-1+d over the cell rows J-1, J; row sums of the y
        // faces J-1+d over the cell columns I-1, I
        const int xa = lj * XW + li, ya = lj * YW + li;
        T cs[3], rs[3];
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            cs[d] = sx[xa + d] + sx[xa + XW + d];
            rs[d] = sy[ya + d * YW] + sy[ya + d * YW + 1];
        }
        const T FE = I == nx ? T(0.5) * cs[1] : T(0.25) * (cs[1] + cs[2]);
        const T FW = I == 0 ? T(0.5) * cs[1] : T(0.25) * (cs[0] + cs[1]);
        const T FN = J == ny ? T(0.5) * rs[1] : T(0.25) * (rs[1] + rs[2]);
        const T FS = J == 0 ? T(0.5) * rs[1] : T(0.25) * (rs[0] + rs[1]);
        const int wc_i = (lj + 1) * WW + li + 1;
        const T wc = sw[wc_i];
        const T wE = I == nx ? wc : (FE > T(0) ? wc : sw[wc_i + 1]);
        const T wW = I == 0 ? wc : (FW > T(0) ? sw[wc_i - 1] : wc);
        const T wN = J == ny ? wc : (FN > T(0) ? wc : sw[wc_i + WW]);
        const T wS = J == 0 ? wc : (FS > T(0) ? sw[wc_i - WW] : wc);
        const T area = ((I == 0 || I == nx) ? T(0.5) : T(1)) *
                       ((J == 0 || J == ny) ? T(0.5) : T(1));
        const size_t idx = (size_t)J * nxn + I;
        const T m = area * depth(hI) * wc - dt / P.dx * (FE * wE - FW * wW)
                  - dt / P.dy * (FN * wN - FS * wS);
        const T hw = a * depth(hB) * wb[idx] + b * m / area;
        wo[idx] = hw * desing(depth(hS), T(1), d4);
    }
}

template <typename T, int TX, int TY>
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? 5 : 1)
k_asm2d_t(Prm<T> P, const T* __restrict__ eta, const T* __restrict__ H,
          const T* __restrict__ q1k, const T* __restrict__ q2k, const T* __restrict__ q1s,
          const T* __restrict__ q2s, const T* __restrict__ w_in, const T* __restrict__ w_b,
          T a, T b, T de, int with_coef, T* __restrict__ ws, T* __restrict__ cC,
          T* __restrict__ cW, T* __restrict__ cE, T* __restrict__ cS, T* __restrict__ cN,
          T* __restrict__ rhs, const T* __restrict__ p0, int resid_form, double* partials,
          SolveCtl* ctl, double tol2, int max_iter, int kpass, int ntx, int ntiles,
          T* __restrict__ q1k_out, T* __restrict__ q2k_out, const double* dtd, T deb)
{
    if (dtd) de = deb * (T)*dtd;   // as the host forms it: dt rounded to T, times the stage's b
    double acc[3] = {0.0, 0.0, 0.0};
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
        asm_tile<T, TX, TY>(P, eta, H, q1k, q2k, q1s, q2s, w_in, w_b, a, b, de, with_coef, ws, cC,
                            cW, cE, cS, cN, rhs, p0, resid_form, t % ntx, t / ntx, acc, q1k_out,
                            q2k_out);
        __syncthreads();   // the tile's shared arrays are restaged by the next tile
    }
    if (grid_reduce<3, 4u>(acc, partials, &ctl->counter) && threadIdx.x == 0)
        asm_finish(ctl, acc, tol2, max_iter, kpass, with_coef);
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
            SolveCtl* ctl, int only_fb)
{
    if (only_fb && !ctl->fb) return;   // captured steps: no fallback in this stage
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
// (residual test, or criterion (32) on the iterate's change when eps_dp > 0)
template <typename T>
__global__ void __launch_bounds__(kThreads)
k_bicg_C(Rows<T> R, T* __restrict__ r, const T* __restrict__ rh, const T* __restrict__ ph,
         const T* __restrict__ v, const T* __restrict__ t, T* __restrict__ x, double* partials,
         SolveCtl* ctl)
{
    if (ctl->done) return;
    const T al = (T)ctl->alpha, om = (T)ctl->omega;
    double acc[3] = {0.0, 0.0, 0.0};
    GRID_STRIDE(idx, (long long)(R.nx + 1) * (R.ny + 1))
    {
        const T s = r[idx] - al * v[idx];
        const T dinv = T(1) / R.cC[idx];
        const T dx = (al * ph[idx] + om * s) * dinv;
        x[idx] += dx;
        const T rn = s - om * t[idx];
        r[idx] = rn;
        acc[0] += (double)rh[idx] * (double)rn;
        acc[1] += (double)rn * (double)rn;
        acc[2] = fmax(acc[2], (double)fabs(dx));
    }
    if (grid_reduce<3, 4u>(acc, partials, &ctl->counter) && threadIdx.x == 0) {
        ctl->rho1 = acc[0];
        ctl->rr = acc[1];
        ctl->dpmax = acc[2];
        ctl->iter += 1;
        if (acc[1] <= ctl->tol2 * ctl->bb || (ctl->eps_dp > 0.0 && acc[2] < ctl->eps_dp)) {
            ctl->done = 1;
            ctl->status = 1;
        }
        else if (ctl->iter >= ctl->max_iter) { ctl->done = 1; ctl->status = 2; }
        else if (ctl->omega == 0.0 || acc[0] == 0.0 || !isfinite(acc[1])) {
            ctl->done = 1; ctl->status = 3;
        }
    }
}

template <typename T, int NA, int NB, int BY, int K, bool REGW, int MINB, bool PAD>
__global__ void __launch_bounds__(32 * BY, MINB)
k_cheb_pass2(Rows<T> R, const T* __restrict__ b, const T* __restrict__ xi,
             const T* __restrict__ xpi, T* __restrict__ xo, T* __restrict__ xpo,
             double* partials, SolveCtl* ctl)
{
    if (ctl->done) return;
    extern __shared__ unsigned char cheb2_smem[];
    NormAcc<T> rsum;
    T dmax;
    if constexpr (PAD)
        cheb_tile_pad<T, NA, NB, BY, K>(R, b, xi, xpi, xo, xpo, ctl, blockIdx.x, blockIdx.y,
                                        reinterpret_cast<T*>(cheb2_smem), rsum, dmax);
    else
        cheb_tile<T, NA, NB, BY, K, REGW>(R, b, xi, xpi, xo, xpo, ctl, blockIdx.x, blockIdx.y,
                                          reinterpret_cast<T*>(cheb2_smem), rsum, dmax);
    double acc[2];
    if (dom_reduce_sum_max<T>(rsum, (double)dmax, ctl->rinv2, partials, &ctl->counter, acc,
                              blockIdx.y * gridDim.x + blockIdx.x, gridDim.x * gridDim.y) &&
        threadIdx.x == 0 && threadIdx.y == 0)
        cheb_finish_stall(ctl, acc, K);
}

// Register form of the pass (cheb_region_reg): persistent blocks walk the regions
// blockIdx.x, blockIdx.x + gridDim.x, ... (row-major over nrx columns of regions), each
// prefetching its next region while it sweeps the current one.  A wait for a region's
// copies gives up after `polls` polls: the block then issues no further copies, waits for
// the copies of that region it has issued (cheb_drain), marks the solve failed (status 6,
// or 7 if even the drain ran out) and leaves the region walk.  stall_block >= 0 is a test
// hook: that block announces bytes on its mbarrier for its first region without issuing
// any copy, so that its first wait runs out with nothing in flight.
template <typename T, int C, int R, int NW, int K>
__global__ void __launch_bounds__(32 * NW, 1)
k_cheb_reg(Rows<T> Rw, const T* __restrict__ b, const T* __restrict__ xi,
           const T* __restrict__ xpi, T* __restrict__ xo, T* __restrict__ xpo,
           double* partials, SolveCtl* ctl, int nrx, int nreg, unsigned polls, int stall_block)
{
    if (ctl->done) return;
    constexpr int RW = 32 * C, RH = R * NW, TX = RW - 2 * K, TY = RH - 2 * K;
    using G = RegionGeom<T, RW, RH>;
    extern __shared__ __align__(16) unsigned char cheb_reg_raw[];
    T* planes = reinterpret_cast<T*>(cheb_reg_raw);
    T* exch = planes + kPlanes * G::PLN;
    __shared__ T c1s[K], c2s[K];
    __shared__ const T* bases[kPlanes];
    __shared__ __align__(8) unsigned long long bar;
    const int tid = threadIdx.x, nx = Rw.nx, ny = Rw.ny;
    if (tid < K) {
        c1s[tid] = sizeof(T) == 4 ? (T)ctl->c1f[tid] : (T)ctl->c1[tid];
        c2s[tid] = sizeof(T) == 4 ? (T)ctl->c2f[tid] : (T)ctl->c2[tid];
    }
    const T rsc = sizeof(T) == 4 ? (T)ctl->rscf : (T)ctl->rscd;
    const double rinv2 = ctl->rinv2;
    // region g = gy nrx + gx, advanced by the grid stride (dgy rows and dgx columns, with a
    // carry) instead of dividing by nrx for every region
    int g = blockIdx.x, gx = g % nrx, gy = g / nrx;
    const int dgx = (int)gridDim.x % nrx, dgy = (int)gridDim.x / nrx;
    auto step = [&](int& x, int& y) {
        x += dgx;
        y += dgy;
        if (x >= nrx) { x -= nrx; ++y; }
    };
    auto I0of = [&](int x) { return x * TX - K; };
    auto J0of = [&](int y) { return y * TY - K; };
    // test hook: this block announces 16 bytes that no copy will bring
    const bool stall = (int)blockIdx.x == stall_block;
    if (tid == 0) {
        bases[kPlX] = xi; bases[kPlXp] = xpi; bases[kPlB] = b; bases[kPlC] = Rw.cC;
        bases[kPlW] = Rw.cW; bases[kPlE] = Rw.cE; bases[kPlS] = Rw.cS; bases[kPlN] = Rw.cN;
        mbar_init(&bar, 1);
        if (g < nreg)
            mbar_arrive_expect_tx(&bar, stall ? 16u : region_bulk_bytes<T, RW, RH>(I0of(gx), nx));
    }
    __syncthreads();
    if (g < nreg && !stall)
        cheb_stage_region<T, RW, RH, 32 * NW>(bases, nx, ny, I0of(gx), J0of(gy), planes, &bar);
    NormAcc<T> rsum;
    norm_zero(rsum);
    T dmax = T(0);
    unsigned phase = 0;
    bool ok = true;
    for (; g < nreg; g += gridDim.x) {
        cp_async_wait_all();
        const bool got = mbar_wait_bounded(&bar, phase, polls);
        if (__syncthreads_or(!got)) { ok = false; break; }
        phase ^= 1u;
        const int nxt = g + gridDim.x;
        int nx_ = gx, ny_ = gy;
        step(nx_, ny_);
        auto next = [&](int part) {
            if (nxt >= nreg) return;
            if (part < 0) {   // before the barrier that frees the planes
                fence_proxy_async_smem();
                if (tid == 0)
                    mbar_arrive_expect_tx(&bar, region_bulk_bytes<T, RW, RH>(I0of(nx_), nx));
            } else {
                cheb_stage_region<T, RW, RH, 32 * NW>(bases, nx, ny, I0of(nx_), J0of(ny_),
                                                      planes, &bar);
            }
        };
        if constexpr (sizeof(T) == 4 && C == 2)
            cheb_region_reg2<R, NW, K>(Rw, planes, exch, c1s, c2s, rsc, I0of(gx),
                                       J0of(gy), xo, xpo, rsum, dmax, next);
        else
            cheb_region_reg<T, C, R, NW, K>(Rw, planes, exch, c1s, c2s, rsc, I0of(gx),
                                            J0of(gy), xo, xpo, rsum, dmax, next);
        gx = nx_;
        gy = ny_;
    }
    if (!ok) {
        const bool issued = !(stall && g == (int)blockIdx.x);
        const bool drained = cheb_drain(&bar, phase, issued);
        if (tid == 0) { ctl->status = drained ? 6 : 7; ctl->done = 1; }
    }
    double acc[2];
    if (dom_reduce_sum_max<T>(rsum, (double)dmax, rinv2, partials, &ctl->counter, acc,
                              blockIdx.x, gridDim.x) &&
        threadIdx.x == 0 && ok)
        cheb_finish_stall(ctl, acc, K);
}

// Cyclic form of the pass (cheb_region_rb): regions of 64 x (R NW) nodes, one persistent
// block per SM walking them, the next region's seven planes fetched by bulk copies during
// the steps; waits, time-out and test hook as in k_cheb_reg.  x only: the pass reads xi
// and writes xo (no previous iterate).
template <typename T, int R, int NW, int K>
__global__ void __launch_bounds__(32 * NW, 1)
k_cheb_rb(Rows<T> Rw, const T* __restrict__ b, const T* __restrict__ xi, T* __restrict__ xo,
          double* partials, SolveCtl* ctl, int nrx, int nreg, unsigned polls, int stall_block)
{
    if (ctl->done) return;
    constexpr int RW = 64, RH = R * NW, TX = RW - 2 * K, TY = RH - 2 * K;
    using G = RegionGeom<T, RW, RH>;
    extern __shared__ __align__(16) unsigned char cheb_rb_raw[];
    T* planes = reinterpret_cast<T*>(cheb_rb_raw);
    T* exch = planes + kRbPlanes * G::PLN;
    __shared__ T c2s[K];
    __shared__ const T* bases[kRbPlanes];
    __shared__ __align__(8) unsigned long long bar;
    const int tid = threadIdx.x, nx = Rw.nx, ny = Rw.ny;
    if (tid < K) c2s[tid] = sizeof(T) == 4 ? (T)ctl->c2f[tid] : (T)ctl->c2[tid];
    const T rsc = sizeof(T) == 4 ? (T)ctl->rscf : (T)ctl->rscd;
    const double rinv2 = ctl->rinv2;
    int g = blockIdx.x, gx = g % nrx, gy = g / nrx;
    const int dgx = (int)gridDim.x % nrx, dgy = (int)gridDim.x / nrx;
    auto step = [&](int& x, int& y) {
        x += dgx;
        y += dgy;
        if (x >= nrx) { x -= nrx; ++y; }
    };
    auto I0of = [&](int x) { return x * TX - K; };
    auto J0of = [&](int y) { return y * TY - K; };
    const bool stall = (int)blockIdx.x == stall_block;
    if (tid == 0) {
        bases[kRbX] = xi; bases[kRbB] = b; bases[kRbC] = Rw.cC; bases[kRbW] = Rw.cW;
        bases[kRbE] = Rw.cE; bases[kRbS] = Rw.cS; bases[kRbN] = Rw.cN;
        mbar_init(&bar, 1);
        if (g < nreg)
            mbar_arrive_expect_tx(&bar, stall ? 16u
                                              : region_bulk_bytes<T, RW, RH, kRbPlanes>(I0of(gx), nx));
    }
    __syncthreads();
    if (g < nreg && !stall)
        cheb_stage_region<T, RW, RH, 32 * NW, kRbPlanes>(bases, nx, ny, I0of(gx), J0of(gy),
                                                         planes, &bar);
    NormAcc<T> rsum;
    norm_zero(rsum);
    T dmax = T(0);
    unsigned phase = 0;
    bool ok = true;
    for (; g < nreg; g += gridDim.x) {
        cp_async_wait_all();
        const bool got = mbar_wait_bounded(&bar, phase, polls);
        if (__syncthreads_or(!got)) { ok = false; break; }
        phase ^= 1u;
        const int nxt = g + gridDim.x;
        int nx_ = gx, ny_ = gy;
        step(nx_, ny_);
        auto next = [&](int part) {
            if (nxt >= nreg) return;
            if (part < 0) {   // before a barrier that frees planes
                fence_proxy_async_smem();
                if (part == -1 && tid == 0)
                    mbar_arrive_expect_tx(&bar, region_bulk_bytes<T, RW, RH, kRbPlanes>(I0of(nx_), nx));
            } else {
                cheb_stage_region<T, RW, RH, 32 * NW, kRbPlanes>(
                    bases, nx, ny, I0of(nx_), J0of(ny_), planes, &bar, part == 1 ? 0 : kRbRows,
                    part == 1 ? kRbRows : kRbPlanes);
            }
        };
        cheb_region_rb<T, R, NW, K>(Rw, planes, exch, c2s, rsc, I0of(gx), J0of(gy), xo, rsum,
                                    dmax, next);
        gx = nx_;
        gy = ny_;
    }
    if (!ok) {
        const bool issued = !(stall && g == (int)blockIdx.x);
        const bool drained = cheb_drain(&bar, phase, issued);
        if (tid == 0) { ctl->status = drained ? 6 : 7; ctl->done = 1; }
    }
    double acc[2];
    if (dom_reduce_sum_max<T>(rsum, (double)dmax, rinv2, partials, &ctl->counter, acc,
                              blockIdx.x, gridDim.x) &&
        threadIdx.x == 0 && ok)
        cheb_finish_stall(ctl, acc, K);
}

template <typename T, int TX, int TY>
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? 3 : 1)
k_corr2d_t(Prm<T> P, const T* __restrict__ eta, const T* __restrict__ H,
           const T* __restrict__ q1k, const T* __restrict__ q2k, const T* __restrict__ ws,
           const T* __restrict__ p, const T* __restrict__ dp, T* __restrict__ pout, T de,
           int with_p, T* __restrict__ eo, T* __restrict__ q1o, T* __restrict__ q2o,
           T* __restrict__ wo, int final_stage, double* partials, StepCtl* st, int ntx,
           int ntiles, const double* dtd, T deb, const T* __restrict__ dp_alt,
           const SolveCtl* sctl, int K)
{
    if (dtd) de = deb * (T)*dtd;
    // captured steps: a Chebyshev solve that ended on an odd pass left its iterate in the
    // other buffer of the ping-pong pair (a BiCGStab fallback always writes dp)
    if (dp_alt && !sctl->fb && ((sctl->sweeps / K) & 1)) dp = dp_alt;
    T lam = T(0);
    int bad = 0;
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
        corr_tile<T, TX, TY>(P, eta, H, q1k, q2k, ws, p, dp, pout, de, with_p, eo, q1o, q2o, wo,
                             final_stage, t % ntx, t / ntx, lam, bad);
        __syncthreads();   // the tile's shared arrays are restaged by the next tile
    }
    if (bad) atomicOr(&st->nonfinite, 1);
    if (final_stage) {
        double acc[1] = {(double)lam};
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
        T b, T dt, T* __restrict__ eo, T* __restrict__ qo, StepCtl* st, T* __restrict__ fm)
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
        const T sg = qsqrt(g);
        pvm(g, sg, hdry, hi[0].h, hi[0].e, hi[0].u, T(0), lo[1].h, lo[1].e, lo[1].u, T(0), DmW, DpW);
        pvm(g, sg, hdry, hi[1].h, hi[1].e, hi[1].u, T(0), lo[2].h, lo[2].e, lo[2].u, T(0), DmE, DpE);
        const St<T>& E = hi[1]; const St<T>& W = lo[1];
        if (fm != nullptr) {   // face mass fluxes F_h(U^-) + D^-_h (the w transport's)
            const size_t f = (size_t)row * (P.nx + 1) + i;
            fm[f] = hi[0].h * hi[0].u + DmW[0];
            if (i == P.nx - 1) fm[f + 1] = E.h * E.u + DmE[0];
        }
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

// Relaxation coefficient of Sec. 4.4 for cell i of a line of n cells (FP64, as the zone
// geometry): the zone on the low side is the klo + 1 cells nearest it, the distance is
// measured from the zone's inner cell (m = 1 there, 0 at the boundary cell); the same on
// the high side; overlapping zones multiply.  k = 0: no zone.
__device__ __forceinline__ double relax_coef(int i, int n, double d, double Llo, int klo,
                                             double Lhi, int khi)
{
    double m = 1.0;
    if (klo > 0 && i <= klo) {
        const double r = (double)(klo - i) * d / Llo, v = 1.0 - r * r;
        m *= v > 0.0 ? sqrt(v) : 0.0;
    }
    if (khi > 0 && i >= n - 1 - khi) {
        const double r = (double)(i - (n - 1 - khi)) * d / Lhi, v = 1.0 - r * r;
        m *= v > 0.0 ? sqrt(v) : 0.0;
    }
    return m;
}

// Node I (between cells I-1 and I): the mean of its two cells' coefficients (the cell
// beyond an end takes the end cell's).
__device__ __forceinline__ double relax_node_coef(int I, int n, double d, double Llo, int klo,
                                                  double Lhi, int khi)
{
    const int a = I - 1 < 0 ? 0 : I - 1, b = I > n - 1 ? n - 1 : I;
    return 0.5 * (relax_coef(a, n, d, Llo, klo, Lhi, khi) +
                  relax_coef(b, n, d, Llo, klo, Lhi, khi));
}

// Relaxation zones of Sec. 4.4 after a step: U <- m U + (1 - m) U* at the zone cells
// (depth h = eta + H blended toward max(eta* + H, 0)), w and p at the zone nodes; 2D
// coefficients are the products of the x and y ones.  One thread per cell, then per node.
template <typename T>
__global__ void __launch_bounds__(kThreads)
k_relax(Prm<T> P, RelaxZ Z, int dim, T* __restrict__ eta, T* __restrict__ q1,
        T* __restrict__ q2, T* __restrict__ w, T* __restrict__ p, const T* __restrict__ H,
        const T* __restrict__ et, const T* __restrict__ q1t, const T* __restrict__ q2t,
        const T* __restrict__ wt, const T* __restrict__ pt)
{
    const int nx = P.nx, ny = P.ny;
    const long long nc = (long long)nx * ny;
    const long long nn = dim == 2 ? (long long)(nx + 1) * (ny + 1) : (long long)(nx + 1) * ny;
    GRID_STRIDE(idx, nc + nn)
    {
        if (idx < nc) {
            const int i = (int)(idx % nx), j = (int)(idx / nx);
            double m = relax_coef(i, nx, Z.d[0], Z.L[0], Z.k[0], Z.L[1], Z.k[1]);
            if (dim == 2) m *= relax_coef(j, ny, Z.d[1], Z.L[2], Z.k[2], Z.L[3], Z.k[3]);
            if (m == 1.0) continue;
            const T mt = (T)m, mc = (T)(1.0 - m);
            const T Hc = H[idx];
            const T hs = tmax(et[idx] + Hc, T(0));
            eta[idx] = (mt * (eta[idx] + Hc) + mc * hs) - Hc;
            q1[idx] = mt * q1[idx] + mc * q1t[idx];
            if (dim == 2) q2[idx] = mt * q2[idx] + mc * q2t[idx];
        } else {
            const long long k = idx - nc;
            const int I = (int)(k % (nx + 1)), J = (int)(k / (nx + 1));
            double m = relax_node_coef(I, nx, Z.d[0], Z.L[0], Z.k[0], Z.L[1], Z.k[1]);
            if (dim == 2) m *= relax_node_coef(J, ny, Z.d[1], Z.L[2], Z.k[2], Z.L[3], Z.k[3]);
            if (m == 1.0) continue;
            const T mt = (T)m, mc = (T)(1.0 - m);
            w[k] = mt * w[k] + mc * wt[k];
            p[k] = mt * p[k] + mc * pt[k];
        }
    }
}

// 1D form of k_wtrans2d_t: node k of a channel owns the dual cell between the centres of
// cells k-1 and k (its inner half at a wall or outflow end); the dual faces carry the
// mean of a cell's two face mass fluxes (the boundary face at an end).  Periodic
// channels wrap (node nx is node 0).
template <typename T>
__global__ void __launch_bounds__(kThreads)
k_wtrans1d(Prm<T> P, const T* __restrict__ etab, const T* __restrict__ etain,
           const T* __restrict__ etas, const T* __restrict__ H, const T* __restrict__ wb,
           const T* __restrict__ win, const T* __restrict__ fm, T a, T b, T dt,
           T* __restrict__ wo)
{
    const T d2 = P.delta * P.delta, d4 = d2 * d2;
    const int n = P.nx, nn = n + 1;
    const bool per = P.bcw == 2;
    GRID_STRIDE(idx, (long long)nn * P.ny)
    {
        const int row = (int)(idx / nn), ko = (int)(idx % nn);
        const int k = per && ko == n ? 0 : ko;   // periodic: node n is node 0
        const T* F = fm + (size_t)row * nn;
        const T* w = win + (size_t)row * nn;
        const size_t c0 = (size_t)row * n;
        auto depth = [&](const T* e) {   // mean of the cells k-1 and k (mapped)
            bool r;
            const int il = map_cell(k - 1, n, P.bcw, P.bce, r);
            const int ir = map_cell(k, n, P.bcw, P.bce, r);
            return T(0.5) * (tmax(e[c0 + il] + H[c0 + il], T(0)) +
                             tmax(e[c0 + ir] + H[c0 + ir], T(0)));
        };
        const bool west_end = !per && k == 0, east_end = !per && k == n;
        const T area = (west_end || east_end) ? T(0.5) : T(1);
        const int kw = k == 0 ? n - 1 : k - 1;
        const T FE = east_end ? F[n] : T(0.5) * (F[k] + F[k + 1]);
        const T FW = west_end ? F[0] : T(0.5) * (F[kw] + F[kw + 1]);
        const T wE = east_end ? w[k] : (FE > T(0) ? w[k] : w[k + 1]);
        const T wW = west_end ? w[k] : (FW > T(0) ? w[kw] : w[k]);
        const T m = area * depth(etain) * w[k] - dt / P.dx * (FE * wE - FW * wW);
        const T hw = a * depth(etab) * wb[(size_t)row * nn + k] + b * m / area;
        wo[idx] = hw * desing(depth(etas), T(1), d4);
    }
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
        // walls / outflow fold the outside node onto its mirror; a periodic channel keeps
        // the cyclic coupling (node nx is node 0 again)
        if (k == 0 && P.bcw != 2) { ck += ak; ak = T(0); }
        if (k == P.nx && P.bce != 2) { ak += ck; ck = T(0); }
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
    // the recurrences run in registers; the arrays are only streamed
    T cpv = Cc[o] / Bd[o], dpv = D[o] / Bd[o];
    cp[o] = cpv;
    dp[o] = dpv;
    for (int i = 1; i < n; ++i) {
        const T ai = A[o + i];
        const T m = Bd[o + i] - ai * cpv;
        cpv = Cc[o + i] / m;
        dpv = (D[o + i] - ai * dpv) / m;
        cp[o + i] = cpv;
        dp[o + i] = dpv;
    }
    T xv = dpv;
    x[o + n - 1] = xv;
    for (int i = n - 2; i >= 0; --i) {
        xv = dp[o + i] - cp[o + i] * xv;
        x[o + i] = xv;
    }
}

// Cyclic tridiagonal solve (periodic channels, Sec. 4.4's modified Thomas algorithm), one
// channel per thread: Sherman-Morrison over two Thomas sweeps that share their elimination
// (right-hand sides d and u = (gamma, 0, ..., 0, alpha)).  Channel rows start every ld
// entries and hold n unknowns; cp and z are scratch; x[n] = x[0] afterwards (the node past
// the last one is the first again).
template <typename T>
__global__ void k_thomas_cyclic(int n, int ld, int rows, const T* __restrict__ A,
                                const T* __restrict__ Bd, const T* __restrict__ Cc,
                                const T* __restrict__ D, T* __restrict__ cp,
                                T* __restrict__ z, T* __restrict__ x)
{
    const int row = blockIdx.x * blockDim.x + threadIdx.x;
    if (row >= rows) return;
    const size_t o = (size_t)row * ld;
    const T alpha = Cc[o + n - 1], beta = A[o], gam = -Bd[o];
    auto bb = [&](int i) {   // diagonal with the rank-one part taken out
        T v = Bd[o + i];
        if (i == 0) v -= gam;
        if (i == n - 1) v -= alpha * beta / gam;
        return v;
    };
    // the recurrences run in registers; the arrays are only streamed
    T m = bb(0);
    T cpv = Cc[o] / m, xv = D[o] / m, zv = gam / m;
    cp[o] = cpv; x[o] = xv; z[o] = zv;
    for (int i = 1; i < n; ++i) {
        const T ai = A[o + i];
        m = bb(i) - ai * cpv;
        cpv = Cc[o + i] / m;
        xv = (D[o + i] - ai * xv) / m;
        zv = ((i == n - 1 ? alpha : T(0)) - ai * zv) / m;
        cp[o + i] = cpv; x[o + i] = xv; z[o + i] = zv;
    }
    for (int i = n - 2; i >= 0; --i) {
        const T c = cp[o + i];
        xv = x[o + i] - c * xv;
        zv = z[o + i] - c * zv;
        x[o + i] = xv; z[o + i] = zv;
    }
    const T fact = (x[o] + beta * x[o + n - 1] / gam) / (T(1) + z[o] + beta * z[o + n - 1] / gam);
    for (int i = 0; i < n; ++i) x[o + i] -= fact * z[o + i];
    x[o + n] = x[o];
}

// y = M x for the channel systems (rows of ld entries); cyclic: n = ld - 1 unknowns with
// wrap-around coupling, and entry n repeats entry 0.
template <typename T>
__global__ void __launch_bounds__(kThreads)
k_tri_apply(int ld, long long total, int cyclic, const T* __restrict__ A,
            const T* __restrict__ Bd, const T* __restrict__ Cc, const T* __restrict__ x,
            T* __restrict__ y)
{
    GRID_STRIDE(idx, total)
    {
        int k = (int)(idx % ld);
        const long long o = idx - k;
        if (cyclic && k == ld - 1) k = 0;   // the repeated first node
        const int n = cyclic ? ld - 1 : ld;
        T v = Bd[o + k] * x[o + k];
        if (k > 0) v += A[o + k] * x[o + k - 1];
        else if (cyclic) v += A[o + k] * x[o + n - 1];
        if (k < n - 1) v += Cc[o + k] * x[o + k + 1];
        else if (cyclic) v += Cc[o + k] * x[o];
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
            if (P.dry_zero && h <= P.hdry) qn = T(0);   // dry cells: no discharge
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
    double acc[1] = {0.0};
    GRID_STRIDE(idx, (long long)P.nx * P.ny)
        acc[0] = fmax(acc[0], lambda_cell(P, dim, eta, q1, q2, H, idx));
    if (grid_reduce<1, 1u>(acc, partials, &st->counter) && threadIdx.x == 0) st->lam = acc[0];
}

// ================================================================ FP64 defect correction

__global__ void __launch_bounds__(kThreads)
k_refine_resid(Rows<double> R, const double* __restrict__ b, const double* __restrict__ x,
               double* __restrict__ r64, double* partials, SolveCtl* ctl64, SolveCtl* ctl32,
               double tol2_in, int max_iter_in, int kpass)
{
    const int nxn = R.nx + 1;
    const long long n = (long long)(R.nx + 1) * (R.ny + 1);
    double acc[1] = {0.0};
    GRID_STRIDE(idx, n)
    {
        const int I = (int)(idx % nxn), J = (int)(idx / nxn);
        const double r = b[idx] - row_apply(R, I, J, x[idx], [&](size_t m) { return x[m]; });
        r64[idx] = r;
        const double rd = r / R.cC[idx];
        acc[0] = fma(rd, rd, acc[0]);
    }
    if (grid_reduce<1, 0u>(acc, partials, &ctl64->counter) && threadIdx.x == 0) {
        ctl64->rr = acc[0];
        const double rms = sqrt(acc[0] / (double)n);
        int e = rms > 0.0 ? ilogb(rms) : 0;
        e = e < -120 ? -120 : (e > 120 ? 120 : e);
        const double s = ldexp(1.0, -e);
        ctl64->rfs = s;
        const double a3[3] = {0.0, acc[0] * s * s, ctl64->gersh};
        asm_finish(ctl32, a3, tol2_in, max_iter_in, kpass, 1);
        ctl32->eps_dp = 0.0;
    }
}

__global__ void __launch_bounds__(kThreads)
k_refine_scale(const double* __restrict__ r64, float* __restrict__ r32, long long n,
               const SolveCtl* ctl64)
{
    const double s = ctl64->rfs;
    GRID_STRIDE(idx, n) r32[idx] = (float)(r64[idx] * s);
}

__global__ void __launch_bounds__(kThreads)
k_refine_add(double* __restrict__ x, const float* __restrict__ d32, long long n,
             const SolveCtl* ctl64)
{
    const double is = 1.0 / ctl64->rfs;   // a power of two: exact
    GRID_STRIDE(idx, n) x[idx] += (double)d32[idx] * is;
}

// ================================================================ captured steps

__global__ void k_loop_cond(cudaGraphConditionalHandle h, const SolveCtl* ctl, unsigned* cnt,
                            unsigned cap, int count)
{
    if (threadIdx.x == 0) {
        const unsigned it = count ? ++*cnt : *cnt;
        cudaGraphSetConditional(h, (!ctl->done && it < cap) ? 1u : 0u);
    }
}

__global__ void k_fb_begin(SolveCtl* ctl)
{
    if (threadIdx.x == 0) ctl->fb = (ctl->status == 4 || ctl->status == 5) ? 1 : 0;
}

template <typename T>
__global__ void __launch_bounds__(kThreads)
k_settle_fb(const SolveCtl* ctl, const T* __restrict__ x2, T* __restrict__ dp, long long n, int K)
{
    if (!ctl->fb || ((ctl->sweeps / K) & 1) == 0) return;
    GRID_STRIDE(idx, n) dp[idx] = x2[idx];
}

__global__ void k_solve_stats(const SolveCtl* ctl, const unsigned* cnt, SolveStat* out)
{
    if (threadIdx.x == 0) {
        out->rr = ctl->rr; out->bb = ctl->bb; out->bdb = ctl->bdb;
        out->sweeps = ctl->sweeps; out->iter = ctl->iter; out->status = ctl->status;
        out->fb = ctl->fb; out->passes = 2 * (int)cnt[0]; out->bicg = 2 * (int)cnt[1];
    }
}

// Flags st->nonfinite when any of the n values of x is NaN or infinite (input checks).
template <typename T>
__global__ void __launch_bounds__(kThreads)
k_nonfinite(const T* __restrict__ x, long long n, StepCtl* st)
{
    int bad = 0;
    GRID_STRIDE(idx, n) bad |= !isfinite(x[idx]);
    if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(&st->nonfinite, 1);
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

// Resident blocks of `kernel` on the current device: SMs x blocks per SM (at least one per
// SM).  The tiled kernels that end in a grid reduction walk their tiles with this many
// blocks, so that the reduction has one partial per resident block.
template <typename K>
int resident_grid(K kernel, int threads, size_t smem)
{
    int dev = 0, nsm = 0, occ = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || nsm < 1)
        nsm = 1;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kernel, threads, smem) != cudaSuccess ||
        occ < 1)
        occ = 1;
    return nsm * occ;
}

template <typename T>
void launch_hyp2d(const Prm<T>& P, const Launch& L, const T* eta, const T* q1, const T* q2,
                  const T* etab, const T* q1b, const T* q2b, const T* H, T a, T b, T dt,
                  T* eo, T* q1o, T* q2o, StepCtl* st, T* fmx, T* fmy, const double* dtd)
{
    constexpr int TX = 32, TY = sizeof(T) == 4 ? 16 : 8;
    dim3 grid((P.nx + TX - 1) / TX, (P.ny + TY - 1) / TY);
    k_hyp2d_t<T, TX, TY><<<grid, kThreads, 0, L.s>>>(P, eta, q1, q2, etab, q1b, q2b, H, a, b, dt,
                                                    eo, q1o, q2o, st, fmx, fmy, dtd);
}

template <typename T>
void launch_wtrans2d(const Prm<T>& P, const Launch& L, const T* etab, const T* etain,
                     const T* etas, const T* H, const T* wb, const T* win, const T* fmx,
                     const T* fmy, T a, T b, T dt, T* wo, const double* dtd)
{
    constexpr int TX = 32, TY = 16, NT = 256;
    dim3 grid((P.nx + 1 + TX - 1) / TX, (P.ny + 1 + TY - 1) / TY);
    k_wtrans2d_t<T, TX, TY, NT><<<grid, NT, 0, L.s>>>(P, etab, etain, etas, H, wb, win, fmx,
                                                       fmy, a, b, dt, wo, dtd);
}

template <typename T>
void launch_asm2d(const Prm<T>& P, const Launch& L, const Bufs<T>& B, const T* w_in,
                  const T* w_base, T a, T b, T de, int with_coef, int resid_form, double tol2,
                  int max_iter, int kpass, double* partials, SolveCtl* ctl, int fuse_break,
                  const double* dtd, T deb)
{
    constexpr int TX = 32, TY = sizeof(T) == 4 ? 16 : 8;   // FP64: static shared memory < 48 KB
    static const int res = resident_grid(k_asm2d_t<T, TX, TY>, kThreads, 0);
    const int ntx = (P.nx + 1 + TX - 1) / TX, ntiles = ntx * ((P.ny + 1 + TY - 1) / TY);
    // fused breaking: q** is computed from q* and written to B.q1k / B.q2k (not read)
    const bool fuse = fuse_break && P.breaking;
    k_asm2d_t<T, TX, TY><<<ntiles < res ? ntiles : res, kThreads, 0, L.s>>>(
        P, B.etas, B.H, fuse ? nullptr : B.q1k, fuse ? nullptr : B.q2k, B.q1s, B.q2s, w_in, w_base,
        a, b, de, with_coef, B.ws, B.cC, B.cW, B.cE, B.cS, B.cN, B.rhs, B.p, resid_form, partials,
        ctl, tol2, max_iter, kpass, ntx, ntiles, fuse ? B.q1k : nullptr, fuse ? B.q2k : nullptr,
        dtd, deb);
}

// Sweeps per Chebyshev pass: 8 in FP32, 4 in FP64 (the forms below).
template <typename T>
int cheb_sweeps_per_pass() { return sizeof(T) == 4 ? 8 : 4; }

template <typename T>
size_t asm_tiles(const Prm<T>& P)
{
    constexpr int TY = sizeof(T) == 4 ? 16 : 8;
    return (size_t)((P.nx + 1 + 31) / 32) * ((P.ny + 1 + TY - 1) / TY);
}

template <typename T>
size_t cheb_tiles(const Prm<T>& P)
{
    // the smallest tile of the forms (64 x 32 region: 56 x 24) gives the most tiles
    constexpr int TX = 56, TY = 24;
    return (size_t)((P.nx + 1 + TX - 1) / TX) * ((P.ny + 1 + TY - 1) / TY);
}

// One form of the pass: region (32 NA) x (BY NB) nodes, 32 x BY threads, weights in
// registers (REGW) or shared memory, at least MINB blocks per SM.
template <typename T, int NA, int NB, int BY, bool REGW, int MINB, bool PAD = false,
          int K = 4>
int launch_cheb_cfg(const Prm<T>& P, cudaStream_t s, const Bufs<T>& B, const T* xi,
                    const T* xpi, T* xo, T* xpo, double* partials)
{
    constexpr int TX = 32 * NA - 2 * K, TY = BY * NB - 2 * K;
    constexpr size_t smem = PAD ? 2 * (size_t)(32 * NA + 2) * (BY * NB + 2) * sizeof(T)
                                : (REGW ? 2 : 7) * (size_t)(32 * NA) * (BY * NB) * sizeof(T);
    static bool attr_set = false;
    if (!attr_set) {
        if (cudaFuncSetAttribute(k_cheb_pass2<T, NA, NB, BY, K, REGW, MINB, PAD>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
            cudaSuccess)
            return -1;
        attr_set = true;
    }
    dim3 grid((P.nx + 1 + TX - 1) / TX, (P.ny + 1 + TY - 1) / TY);
    k_cheb_pass2<T, NA, NB, BY, K, REGW, MINB, PAD><<<grid, dim3(32, BY), smem, s>>>(
        rows_of(P, B), B.rhs, xi, xpi, xo, xpo, partials, B.sctl);
    return 0;
}


// Register form: region (32 C) x (R NW) nodes, 32 NW threads, one resident block per SM
// (the staged planes take most of the shared memory), K sweeps per pass.
template <typename T, int C, int R, int NW, int K>
int launch_cheb_reg(const Prm<T>& P, cudaStream_t s, const Bufs<T>& B, const T* xi,
                    const T* xpi, T* xo, T* xpo, double* partials, unsigned polls,
                    int stall_block)
{
    constexpr int TX = 32 * C - 2 * K, TY = R * NW - 2 * K;
    constexpr size_t smem = cheb_reg_smem<T, C, R, NW>();
    static int nblk = 0;
    if (nblk == 0) {
        if (cudaFuncSetAttribute(k_cheb_reg<T, C, R, NW, K>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
            cudaSuccess)
            return -1;
        int dev = 0, nsm = 0, occ = 0;
        if (cudaGetDevice(&dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_cheb_reg<T, C, R, NW, K>,
                                                          32 * NW, smem) != cudaSuccess ||
            occ < 1)
            return -1;
        nblk = nsm * occ;
    }
    const int nrx = (P.nx + 1 + TX - 1) / TX, nry = (P.ny + 1 + TY - 1) / TY;
    const int nreg = nrx * nry;
    k_cheb_reg<T, C, R, NW, K><<<nreg < nblk ? nreg : nblk, 32 * NW, smem, s>>>(
        rows_of(P, B), B.rhs, xi, xpi, xo, xpo, partials, B.sctl, nrx, nreg, polls,
        stall_block);
    return 0;
}

// Cyclic form: region 64 x (R NW) nodes, 32 NW threads, one resident block per SM.
template <typename T, int R, int NW, int K>
int launch_cheb_rb(const Prm<T>& P, cudaStream_t s, const Bufs<T>& B, const T* xi, T* xo,
                   double* partials, unsigned polls, int stall_block)
{
    constexpr int TX = 64 - 2 * K, TY = R * NW - 2 * K;
    constexpr size_t smem = cheb_rb_smem<T, R, NW>();
    static int nblk = 0;
    if (nblk == 0) {
        if (cudaFuncSetAttribute(k_cheb_rb<T, R, NW, K>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
            cudaSuccess)
            return -1;
        int dev = 0, nsm = 0, occ = 0;
        if (cudaGetDevice(&dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_cheb_rb<T, R, NW, K>,
                                                          32 * NW, smem) != cudaSuccess ||
            occ < 1)
            return -1;
        nblk = nsm * occ;
    }
    const int nrx = (P.nx + 1 + TX - 1) / TX, nry = (P.ny + 1 + TY - 1) / TY;
    const int nreg = nrx * nry;
    k_cheb_rb<T, R, NW, K><<<nreg < nblk ? nreg : nblk, 32 * NW, smem, s>>>(
        rows_of(P, B), B.rhs, xi, xo, partials, B.sctl, nrx, nreg, polls, stall_block);
    return 0;
}

// The pass forms the handle chooses from by timing its first passes; all forms of a
// precision sweep the same number of times per pass (K) and give the same iterates.
// FP32 (K = 8, weights in registers, padded buffers): 0: 64x64 region, 1024 threads;
// 1: 128x64, 1024 threads; 2: 64x64, 512 threads, 2 blocks / SM; 3: 64x64, 512 threads,
// 1 block; 4: 128x64, 512 threads, 1 block; register forms (sweeps in registers,
// persistent blocks with prefetched regions): 5: 64x64, 512 threads; 6: 64x64, 1024
// threads; 7: 96x64, 512 threads.
// FP64 (K = 4): 0: 64x32, shared-memory weights; 1: 64x32, registers; 2: 64x32, registers,
// padded; 3: register form, 64x32, 512 threads.
// The cyclic forms (k_cheb_rb, one colour per step) follow: FP32 8: 64x96 region, 512
// threads; 9: 64x64, 512 threads; 10: 64x64, 1024 threads; FP64 4: 64x32, 512 threads.  They
// give the same iterates as each other (not those of the Jacobi forms), so they are timed
// against each other only.
template <typename T> int cheb_pass_forms() { return sizeof(T) == 4 ? 8 : 4; }
template <typename T> int cheb_cyclic_forms() { return sizeof(T) == 4 ? 3 : 1; }

template <typename T>
int launch_cheb_pass(const Prm<T>& P, cudaStream_t s, const Bufs<T>& B, const T* xi,
                     const T* xpi, T* xo, T* xpo, double* partials, int variant,
                     unsigned polls, int stall_block)
{
    if constexpr (sizeof(T) == 4) {
        switch (variant) {
        case 1: return launch_cheb_cfg<T, 4, 2, 32, true, 1, true, 8>(P, s, B, xi, xpi, xo, xpo, partials);
        case 2: return launch_cheb_cfg<T, 2, 4, 16, true, 2, true, 8>(P, s, B, xi, xpi, xo, xpo, partials);
        case 3: return launch_cheb_cfg<T, 2, 4, 16, true, 1, true, 8>(P, s, B, xi, xpi, xo, xpo, partials);
        case 4: return launch_cheb_cfg<T, 4, 4, 16, true, 1, true, 8>(P, s, B, xi, xpi, xo, xpo, partials);
        case 5: return launch_cheb_reg<T, 2, 4, 16, 8>(P, s, B, xi, xpi, xo, xpo, partials, polls, stall_block);
        case 6: return launch_cheb_reg<T, 2, 2, 32, 8>(P, s, B, xi, xpi, xo, xpo, partials, polls, stall_block);
        case 7: return launch_cheb_reg<T, 3, 4, 16, 8>(P, s, B, xi, xpi, xo, xpo, partials, polls, stall_block);
        case 8: return launch_cheb_rb<T, 6, 16, 8>(P, s, B, xi, xo, partials, polls, stall_block);
        case 9: return launch_cheb_rb<T, 4, 16, 8>(P, s, B, xi, xo, partials, polls, stall_block);
        case 10: return launch_cheb_rb<T, 2, 32, 8>(P, s, B, xi, xo, partials, polls, stall_block);
        default: return launch_cheb_cfg<T, 2, 2, 32, true, 1, true, 8>(P, s, B, xi, xpi, xo, xpo, partials);
        }
    } else {
        if (variant == 4) return launch_cheb_rb<T, 2, 16, 4>(P, s, B, xi, xo, partials, polls, stall_block);
        if (variant == 1) return launch_cheb_cfg<T, 2, 2, 16, true, 1>(P, s, B, xi, xpi, xo, xpo, partials);
        if (variant == 2) return launch_cheb_cfg<T, 2, 2, 16, true, 1, true>(P, s, B, xi, xpi, xo, xpo, partials);
        if (variant == 3) return launch_cheb_reg<T, 2, 2, 16, 4>(P, s, B, xi, xpi, xo, xpo, partials, polls, stall_block);
        return launch_cheb_cfg<T, 2, 2, 16, false, 2>(P, s, B, xi, xpi, xo, xpo, partials);
    }
}

template <typename T>
void launch_matvec2d(const Prm<T>& P, const Launch& L, const Bufs<T>& B, const T* x, T* y)
{
    k_matvec2d<T><<<L.nblk, kThreads, 0, L.s>>>(rows_of(P, B), x, y);
}

template <typename T>
void launch_bicg_init(const Prm<T>& P, const Launch& L, const Bufs<T>& B, double* partials,
                      int only_fb)
{
    k_bicg_init<T><<<L.nblk, kThreads, 0, L.s>>>(rows_of(P, B), B.rhs, B.dp, B.r, B.rh, B.ph[0],
                                                 B.v[0], partials, B.sctl, only_fb);
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
                   double* partials, StepCtl* st, const double* dtd, T deb, const T* dp_alt)
{
    constexpr int TX = 32, TY = 16;   // 2 nodes a thread (32x8: 0.251 ms, 32x16: 0.229 ms at 4096^2 FP32)
    static const int res = resident_grid(k_corr2d_t<T, TX, TY>, 256, 0);
    const int ntx = (P.nx + 1 + TX - 1) / TX, ntiles = ntx * ((P.ny + 1 + TY - 1) / TY);
    k_corr2d_t<T, TX, TY><<<ntiles < res ? ntiles : res, 256, 0, L.s>>>(
        P, B.etas, B.H, q1k, q2k, B.ws, B.p, B.dp, B.palt, de, with_p, eo, q1o, q2o, wo,
        final_stage, partials, st, ntx, ntiles, dtd, deb, dp_alt, B.sctl,
        cheb_sweeps_per_pass<T>());
}

template <typename T>
void launch_hyp1d(const Prm<T>& P, const Launch& L, const T* eta, const T* q, const T* etab,
                  const T* qb, const T* H, T a, T b, T dt, T* eo, T* qo, StepCtl* st, T* fm)
{
    k_hyp1d<T><<<L.nblk, kThreads, 0, L.s>>>(P, eta, q, etab, qb, H, a, b, dt, eo, qo, st, fm);
}

template <typename T>
void launch_relax(const Prm<T>& P, const Launch& L, const RelaxZ& Z, int dim, T* eta, T* q1,
                  T* q2, T* w, T* p, const T* H, const T* et, const T* q1t, const T* q2t,
                  const T* wt, const T* pt)
{
    k_relax<T><<<L.nblk, kThreads, 0, L.s>>>(P, Z, dim, eta, q1, q2, w, p, H, et, q1t, q2t, wt,
                                             pt);
}

template <typename T>
void launch_wtrans1d(const Prm<T>& P, const Launch& L, const T* etab, const T* etain,
                     const T* etas, const T* H, const T* wb, const T* win, const T* fm, T a,
                     T b, T dt, T* wo)
{
    k_wtrans1d<T><<<L.nblk, kThreads, 0, L.s>>>(P, etab, etain, etas, H, wb, win, fm, a, b, dt,
                                                wo);
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
    if (P.bcw == 2) {   // periodic channels: nx unknowns with cyclic coupling
        k_thomas_cyclic<T><<<(P.ny + 127) / 128, 128, 0, s>>>(P.nx, P.nx + 1, P.ny, B.cW, B.cC,
                                                              B.cE, B.rhs, B.r, B.rh, x);
        return 0;
    }
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
    k_tri_apply<T><<<L.nblk, kThreads, 0, L.s>>>(P.nx + 1, (long long)(P.nx + 1) * P.ny,
                                                 P.bcw == 2 ? 1 : 0, B.cW, B.cC, B.cE, x, y);
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

void launch_refine_resid(const Prm<double>& P, const Launch& L, const Bufs<double>& B,
                         const double* x, double* r64, double* partials, SolveCtl* ctl64,
                         SolveCtl* ctl32, double tol2_in, int max_iter_in, int kpass)
{
    k_refine_resid<<<L.nblk, kThreads, 0, L.s>>>(rows_of(P, B), B.rhs, x, r64, partials, ctl64,
                                                 ctl32, tol2_in, max_iter_in, kpass);
}

void launch_refine_scale(const Launch& L, const double* r64, float* r32, size_t n,
                         const SolveCtl* ctl64)
{
    k_refine_scale<<<L.nblk, kThreads, 0, L.s>>>(r64, r32, (long long)n, ctl64);
}

void launch_refine_add(const Launch& L, double* x, const float* d32, size_t n,
                       const SolveCtl* ctl64)
{
    k_refine_add<<<L.nblk, kThreads, 0, L.s>>>(x, d32, (long long)n, ctl64);
}

void launch_loop_cond(cudaStream_t s, cudaGraphConditionalHandle h, const SolveCtl* ctl,
                      unsigned* cnt, unsigned cap, int count)
{
    k_loop_cond<<<1, 32, 0, s>>>(h, ctl, cnt, cap, count);
}

void launch_fb_begin(cudaStream_t s, SolveCtl* ctl) { k_fb_begin<<<1, 32, 0, s>>>(ctl); }

template <typename T>
void launch_settle_fb(const Launch& L, const SolveCtl* ctl, const T* x2, T* dp, size_t n, int K)
{
    k_settle_fb<T><<<L.nblk, kThreads, 0, L.s>>>(ctl, x2, dp, (long long)n, K);
}

void launch_solve_stats(cudaStream_t s, const SolveCtl* ctl, const unsigned* cnt, SolveStat* out)
{
    k_solve_stats<<<1, 32, 0, s>>>(ctl, cnt, out);
}

template <typename T>
__global__ void k_gather(const T* __restrict__ x, const int* __restrict__ idx, int n,
                         T* __restrict__ out)
{
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x)
        out[k] = x[idx[k]];
}

template <typename T>
void launch_gather(cudaStream_t s, const T* x, const int* idx, int n, T* out)
{
    k_gather<T><<<(n + 255) / 256 < 148 ? (n + 255) / 256 : 148, 256, 0, s>>>(x, idx, n, out);
}

template <typename T>
void launch_nonfinite(const Launch& L, const T* x, size_t n, StepCtl* st)
{
    k_nonfinite<T><<<L.nblk, kThreads, 0, L.s>>>(x, (long long)n, st);
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
                                  StepCtl*, T*, T*, const double*);                            \
    template void launch_wtrans2d<T>(const Prm<T>&, const Launch&, const T*, const T*,         \
                                     const T*, const T*, const T*, const T*, const T*,         \
                                     const T*, T, T, T, T*, const double*);                    \
    template void launch_relax<T>(const Prm<T>&, const Launch&, const RelaxZ&, int, T*, T*,    \
                                  T*, T*, T*, const T*, const T*, const T*, const T*,          \
                                  const T*, const T*);                                         \
    template void launch_wtrans1d<T>(const Prm<T>&, const Launch&, const T*, const T*,         \
                                     const T*, const T*, const T*, const T*, const T*, T, T,   \
                                     T, T*);                                                   \
    template void launch_asm2d<T>(const Prm<T>&, const Launch&, const Bufs<T>&, const T*,      \
                                  const T*, T, T, T, int, int, double, int, int, double*,      \
                                  SolveCtl*, int, const double*, T);                           \
    template int cheb_sweeps_per_pass<T>();                                                    \
    template size_t cheb_tiles<T>(const Prm<T>&);                                              \
    template size_t asm_tiles<T>(const Prm<T>&);                                               \
    template int cheb_pass_forms<T>();                                                          \
    template int cheb_cyclic_forms<T>();                                                        \
    template int launch_cheb_pass<T>(const Prm<T>&, cudaStream_t, const Bufs<T>&, const T*,   \
                                     const T*, T*, T*, double*, int, unsigned, int);            \
    template void launch_matvec2d<T>(const Prm<T>&, const Launch&, const Bufs<T>&, const T*,   \
                                     T*);                                                      \
    template void launch_bicg_init<T>(const Prm<T>&, const Launch&, const Bufs<T>&, double*,   \
                                      int);                                                    \
    template void launch_settle_fb<T>(const Launch&, const SolveCtl*, const T*, T*, size_t,    \
                                      int);                                                    \
    template void launch_bicg_phase<T>(const Prm<T>&, const Launch&, const Bufs<T>&, int, int, \
                                       double*);                                               \
    template void launch_corr2d<T>(const Prm<T>&, const Launch&, const Bufs<T>&, const T*,     \
                                   const T*, T, int, T*, T*, T*, T*, int, double*, StepCtl*,   \
                                   const double*, T, const T*);                                \
    template void launch_hyp1d<T>(const Prm<T>&, const Launch&, const T*, const T*, const T*,  \
                                  const T*, const T*, T, T, T, T*, T*, StepCtl*, T*);          \
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
    template void launch_nonfinite<T>(const Launch&, const T*, size_t, StepCtl*);               \
    template void launch_gather<T>(cudaStream_t, const T*, const int*, int, T*);               \
    template void launch_convert_from_double<T>(const Launch&, const double*, T*, size_t);

NH_INSTANTIATE(float)
NH_INSTANTIATE(double)

}  // namespace nh
