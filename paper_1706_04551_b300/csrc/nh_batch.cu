// nh_batch.cu -- ensembles of independent 2D domains of uneven sizes, advanced together.
//
// Every domain runs the same step as a single handle (the tile and element bodies of
// nh_device.cuh, Chebyshev-scheduled Jacobi for the pressure), but each kernel class is
// ONE launch for all domains: its blocks walk a work list of (domain, tile) items, sorted
// largest domain first, either one block per item or a persistent grid of the blocks that
// fit on the GPU at once.  Per domain the device keeps its own time step (Eq. 23 from its
// own state, or a fixed step), its own solver control block and convergence, and its own
// reductions (a last-block-done finish per domain).  A domain whose solve has converged
// drops out of the remaining Chebyshev passes of that stage; the pass loop ends when no
// domain is left.  With the graph option one whole step (two stages) is a CUDA graph whose
// solver loops are device-side conditional WHILE nodes, so a run of n steps is n graph
// launches and no host round trip.  Tile shapes and grid forms are chosen by a small
// autotuner that times the candidates on the ensemble's own state before the first step.
#include "../../include/nh.h"
#include "nh_device.cuh"

#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <functional>
#include <memory>
#include <numeric>
#include <string>
#include <utility>
#include <vector>

namespace nh {
namespace {

using namespace dev;

constexpr int kChunk = 2048;   // cells / nodes per element work item (8 per thread)

template <typename T>
struct Dom {
    Prm<T> P;
    long long coff, noff;   // first cell / node of the domain in the arenas
    long long poff;         // first partial (doubles) of the domain
    int ncc, nnc;           // element work items: cell chunks, node chunks
};

// Per-domain bookkeeping kept on the device.
struct DomState {
    double t, dt, lam, mass;
    long long steps, sweeps, bicg_iters;   // sweeps: Chebyshev sweeps + BiCGStab iterations
    double last_resid[2];
    int last_sweeps[2];
    int last_status[2];   // 1 converged, 2 cap, 3 breakdown, 4 not diagonally dominant, 5 stalled
    int nonconv;          // solves that ended without converging (cap or breakdown)
    int fallbacks;        // solves finished by BiCGStab (Chebyshev stalled: status 5, or
                          // the system was not diagonally dominant: status 4)
    int clamped, nonfinite;
};

template <typename T>
struct Arena {
    const Dom<T>* dom;
    SolveCtl* sctl;
    StepCtl* stctl;
    DomState* ds;
    double* partials;
    unsigned* loop;        // [0] domains in Chebyshev passes, [1] passes launched this stage,
                           // [2] domains in the BiCGStab fallback, [3] its iterations
    double fixed_dt, cfl;
    unsigned polls;        // bounded waits of the register-form pass (nh_params.wait_polls)
};

__host__ __device__ inline int cdiv(int a, int b) { return (a + b - 1) / b; }

// ---------------------------------------------------------------- kernels

template <typename T>
__global__ void __launch_bounds__(kThreads)
kb_lambda(Arena<T> A, const int2* __restrict__ wl, int nw, const T* __restrict__ eta,
          const T* __restrict__ q1, const T* __restrict__ q2, const T* __restrict__ H)
{
    for (int w = blockIdx.x; w < nw; w += gridDim.x) {
        const int2 it = wl[w];
        const Dom<T>& D = A.dom[it.x];
        const Prm<T> P = D.P;
        const long long c = D.coff, n = (long long)P.nx * P.ny;
        double acc[1] = {0.0};
        for (long long k = (long long)it.y * kChunk + threadIdx.x;
             k < n && k < (long long)(it.y + 1) * kChunk; k += blockDim.x)
            acc[0] = fmax(acc[0], lambda_cell(P, 2, eta + c, q1 + c, q2 + c, H + c, k));
        if (dom_reduce<1, 1u>(acc, A.partials + D.poff, &A.stctl[it.x].counter, it.y, D.ncc) &&
            threadIdx.x == 0) {
            DomState& s = A.ds[it.x];
            s.lam = acc[0];
            s.dt = A.fixed_dt > 0.0 ? A.fixed_dt : (acc[0] > 0.0 ? A.cfl / acc[0] : 0.0);
        }
        __syncthreads();
    }
}

template <typename T>
__global__ void __launch_bounds__(kThreads)
kb_mass(Arena<T> A, const int2* __restrict__ wl, int nw, const T* __restrict__ eta,
        const T* __restrict__ H)
{
    for (int w = blockIdx.x; w < nw; w += gridDim.x) {
        const int2 it = wl[w];
        const Dom<T>& D = A.dom[it.x];
        const long long c = D.coff, n = (long long)D.P.nx * D.P.ny;
        double acc[1] = {0.0};
        for (long long k = (long long)it.y * kChunk + threadIdx.x;
             k < n && k < (long long)(it.y + 1) * kChunk; k += blockDim.x)
            acc[0] += (double)tmax(eta[c + k] + H[c + k], T(0));
        if (dom_reduce<1, 0u>(acc, A.partials + D.poff, &A.stctl[it.x].counter, it.y, D.ncc) &&
            threadIdx.x == 0)
            A.ds[it.x].mass = acc[0] * (double)D.P.dx * (double)D.P.dy;
        __syncthreads();
    }
}

template <typename T, int TX, int TY>
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? 4 : 2)
kb_hyp(Arena<T> A, const int2* __restrict__ wl, int nw, const T* eta, const T* q1,
       const T* q2, const T* etab, const T* q1b, const T* q2b, const T* H, T a, T b, T* eo,
       T* q1o, T* q2o)
{
    for (int w = blockIdx.x; w < nw; w += gridDim.x) {
        const int2 it = wl[w];
        const Dom<T>& D = A.dom[it.x];
        const Prm<T> P = D.P;
        const long long c = D.coff;
        const T dt = (T)A.ds[it.x].dt;
        const int tx = cdiv(P.nx, TX);
        const int nclamp = hyp_tile<T, TX, TY>(P, eta + c, q1 + c, q2 + c, etab + c, q1b + c,
                                               q2b + c, H + c, a, b, dt, eo + c, q1o + c,
                                               q2o + c, it.y % tx, it.y / tx);
        if (nclamp) atomicAdd(&A.ds[it.x].clamped, nclamp);
        __syncthreads();
    }
}

struct AsmArgs {
    double tol2;
    int max_iter, kpass, with_coef, stage;
    int fuse;   // breaking terms inside the assembly (q* -> q** into q1k / q2k)
};

template <typename T, int TX, int TY>
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? 6 : 3)
kb_asm(Arena<T> A, const int2* __restrict__ wl, int nw, const T* eta, const T* H,
       T* q1k, T* q2k, const T* q1s, const T* q2s, const T* w_in, const T* w_b,
       T a, T b, T* ws, T* cC, T* cW, T* cE, T* cS, T* cN, T* rhs, const T* p0, AsmArgs G)
{
    // a contiguous share of the list (one item when the grid has a block per item); the
    // norms and Gershgorin ratio of the block's consecutive items of one domain accumulate
    // per thread and are published once for the group (dom_publish)
    const int lo = (int)((long long)nw * blockIdx.x / gridDim.x);
    const int hi = (int)((long long)nw * (blockIdx.x + 1) / gridDim.x);
    int gd = -1, gy = 0, gn = 0, gnt = 0;
    long long gpoff = 0;
    double acc[3] = {0.0, 0.0, 0.0};
    auto flush = [&]() {
        if (gn == 0) return;
        SolveCtl* ctl = &A.sctl[gd];
        if (dom_publish<3, 4u>(acc, A.partials + gpoff, &ctl->counter, gy, gn, gnt) &&
            threadIdx.x == 0) {
            asm_finish(ctl, acc, G.tol2, G.max_iter, G.kpass, G.with_coef);
            ctl->best = 1.0e300;
            ctl->stale = 0;
            ctl->fb = 0;
            A.ds[gd].last_sweeps[G.stage] = 0;
            if (!G.with_coef) {
                ctl->done = 1;
            } else if (!ctl->done) {
                atomicAdd(&A.loop[0], 1u);
            } else {
                // not diagonally dominant (status 4): the Chebyshev interval does not hold,
                // solve with BiCGStab from dp = 0
                ctl->fb = 1;
                atomicAdd(&A.loop[2], 1u);
            }
        }
        gn = 0;
        acc[0] = acc[1] = acc[2] = 0.0;
    };
    for (int w = lo; w < hi; ++w) {
        const int2 it = wl[w];
        const Dom<T>& D = A.dom[it.x];
        const Prm<T> P = D.P;
        const long long c = D.coff, n = D.noff;
        const T de = b * (T)A.ds[it.x].dt;
        const int tx = cdiv(P.nx + 1, TX);
        if (it.x != gd) {
            flush();
            gd = it.x;
            gy = it.y;
            gnt = tx * cdiv(P.ny + 1, TY);
            gpoff = D.poff;
        } else if (threadIdx.x == 0) {   // pooled into the group's slot: this item's is zero
            double* sl = A.partials + gpoff + 3 * (long long)it.y;
            sl[0] = sl[1] = sl[2] = 0.0;
        }
        // fused breaking: q** is computed in the tile and written to q1k / q2k (not read)
        const bool fuse = G.fuse && P.breaking;
        asm_tile<T, TX, TY>(P, eta + c, H + c, fuse ? nullptr : q1k + c, fuse ? nullptr : q2k + c,
                            q1s + c, q2s + c, w_in + n, w_b + n, a, b, de, G.with_coef, ws + n,
                            cC + n, cW + n, cE + n, cS + n, cN + n, rhs + n, p0 + n,
                            /*resid_form=*/G.with_coef, it.y % tx, it.y / tx, acc,
                            fuse ? q1k + c : nullptr, fuse ? q2k + c : nullptr);
        ++gn;
        __syncthreads();   // the tile's shared arrays are restaged by the next item
    }
    flush();
}

// Last block of a domain's items in a pass: convergence test and next weights, the stall
// test (cheb_finish_stall: status 5, BiCGStab takes over from the current dp), and the loop
// counters and statistics of a finished domain.
template <typename T>
__device__ __forceinline__ void kb_cheb_finish(const Arena<T>& A, int d, SolveCtl* ctl,
                                               const double (&acc)[2], int K, int stage)
{
    cheb_finish_stall(ctl, acc, K);
    if (ctl->done) {
        atomicSub(&A.loop[0], 1u);
        DomState& s = A.ds[d];
        s.sweeps += ctl->sweeps;
        s.last_sweeps[stage] = ctl->sweeps;
        if (ctl->status == 5) {
            // stalled (rounding floor of the precision, or a spectrum the Gershgorin
            // interval does not describe)
            ctl->fb = 1;
            atomicAdd(&A.loop[2], 1u);
        } else {
            s.last_status[stage] = ctl->status;
            s.last_resid[stage] = ctl->bdb > 0.0 ? sqrt(ctl->rr / ctl->bdb) : 0.0;
            if (ctl->status != 1) s.nonconv += 1;
        }
    }
}

template <typename T, int NA, int NB, int BY, int K, bool REGW, int MINB, bool PAD>
__global__ void __launch_bounds__(32 * BY, MINB)
kb_cheb(Arena<T> A, const int2* __restrict__ wl, int nw, const T* cC, const T* cW,
        const T* cE, const T* cS, const T* cN, const T* rhs, const T* xi, const T* xpi, T* xo,
        T* xpo, int stage, const int* plan, int want)
{
    if (plan) {   // a planned pass: run only the branch the plan chose (kb_cheb_plan)
        if (plan[0] != want) return;
        if (want == 1) nw = plan[1];
    }
    extern __shared__ unsigned char kb_cheb_smem[];
    constexpr int TX = 32 * NA - 2 * K, TY = BY * NB - 2 * K;
    for (int w = blockIdx.x; w < nw; w += gridDim.x) {
        const int2 it = wl[w];
        SolveCtl* ctl = &A.sctl[it.x];
        if (ctl->done) continue;   // uniform: set only after all of this domain's items
        const Dom<T>& D = A.dom[it.x];
        const long long n = D.noff;
        Rows<T> R;
        R.cC = cC + n; R.cW = cW + n; R.cE = cE + n; R.cS = cS + n; R.cN = cN + n;
        R.nx = D.P.nx; R.ny = D.P.ny;
        const int tx = cdiv(R.nx + 1, TX), nt = tx * cdiv(R.ny + 1, TY);
        NormAcc<T> rsum;
        T dmax;
        if constexpr (PAD)
            cheb_tile_pad<T, NA, NB, BY, K>(R, rhs + n, xi + n, xpi + n, xo + n, xpo + n, ctl,
                                            it.y % tx, it.y / tx,
                                            reinterpret_cast<T*>(kb_cheb_smem), rsum, dmax);
        else
            cheb_tile<T, NA, NB, BY, K, REGW>(R, rhs + n, xi + n, xpi + n, xo + n, xpo + n, ctl,
                                              it.y % tx, it.y / tx,
                                              reinterpret_cast<T*>(kb_cheb_smem), rsum, dmax);
        double acc[2];
        if (dom_reduce_sum_max<T>(rsum, (double)dmax, ctl->rinv2, A.partials + D.poff,
                                  &ctl->counter, acc, it.y, nt) &&
            threadIdx.x == 0 && threadIdx.y == 0)
            kb_cheb_finish(A, it.x, ctl, acc, K, stage);
        __syncthreads();
    }
}

// Register form of the batched pass: each block takes a contiguous, balanced share
// [lo, hi) of the work list (a chunk of a few items, or a whole resident block's share), in
// which a domain's items are contiguous, so a share covers parts of a few domains.  The block walks its share, skipping whole domains that
// have converged, and prefetches its next item's region (bulk copies on an mbarrier,
// element copies at the domain's west and east edges) while it sweeps the current one.  A
// domain's geometry and solver weights are read when the walk enters it (the next region
// of the same domain follows by arithmetic), and the residual sums of the block's
// consecutive items of one domain accumulate in registers and are published once for the
// group (dom_publish_sum_max: the group's first slot holds the sum, its other slots zero).
// A wait that runs out of `polls` polls ends the block's walk: the block issues no further
// copies, waits (bounded) for those of the item it was waiting on (cheb_drain) and marks
// the item's domain failed (status 6, or 7 if the drain ran out too; counted as a
// non-converged solve).
template <typename T, int C, int R, int NW, int K>
__global__ void __launch_bounds__(32 * NW, 1)
kb_cheb_reg(Arena<T> A, const int2* __restrict__ wl, int nw, const T* cC, const T* cW,
            const T* cE, const T* cS, const T* cN, const T* rhs, const T* xi, const T* xpi,
            T* xo, T* xpo, int stage, const int* plan, int want)
{
    if (plan) {   // a planned pass: run only the branch the plan chose (kb_cheb_plan)
        if (plan[0] != want) return;
        if (want == 1) nw = plan[1];
    }
    const unsigned polls = A.polls;
    constexpr int RW = 32 * C, RH = R * NW, TX = RW - 2 * K, TY = RH - 2 * K;
    using G = RegionGeom<T, RW, RH>;
    extern __shared__ __align__(16) unsigned char kb_reg_raw[];
    T* planes = reinterpret_cast<T*>(kb_reg_raw);
    T* exch = planes + kPlanes * G::PLN;
    __shared__ T c1s[K], c2s[K];
    __shared__ const T* bases[kPlanes];
    __shared__ __align__(8) unsigned long long bar;
    const int tid = threadIdx.x;
    const int lo = (int)((long long)nw * blockIdx.x / gridDim.x);
    const int hi = (int)((long long)nw * (blockIdx.x + 1) / gridDim.x);
    // an item of the walk (uniform across the block): work-list index, domain, region and
    // the domain's node offset and size
    struct Item { int w, d, y, cx, cy, nx, ny; long long n; };   // (cx, cy): region column, row
    auto ntx_of = [&](const Item& it) { return cdiv(it.nx + 1, TX); };
    auto nt_of = [&](const Item& it) { return ntx_of(it) * cdiv(it.ny + 1, TY); };
    // the first item at or after `from` of this share whose domain still solves; `cur` is
    // the item being processed (a domain still solving), so its successor inside the same
    // domain needs no load.  False when the share is exhausted.
    auto advance = [&](const Item& cur, int from, Item& it) -> bool {
        if (from >= hi) return false;
        if (cur.w == from - 1 && cur.y + 1 < nt_of(cur)) {
            it = cur;
            it.w = from;
            it.y = cur.y + 1;
            if (++it.cx == ntx_of(it)) { it.cx = 0; ++it.cy; }
            return true;
        }
        for (int w = from; w < hi;) {
            const int2 e = wl[w];
            const Dom<T>& D = A.dom[e.x];
            it.w = w; it.d = e.x; it.y = e.y; it.nx = D.P.nx; it.ny = D.P.ny; it.n = D.noff;
            if (!A.sctl[e.x].done) {
                const int ntx = ntx_of(it);
                it.cx = e.y % ntx;
                it.cy = e.y / ntx;
                return true;
            }
            w += nt_of(it) - it.y;   // past this domain's items
        }
        return false;
    };
    auto origin = [&](const Item& it, int& I0, int& J0) {
        I0 = it.cx * TX - K;
        J0 = it.cy * TY - K;
    };
    auto announce = [&](const Item& it) {   // thread 0: the item's sources and expected bytes
        const long long n = it.n;
        bases[kPlX] = xi + n; bases[kPlXp] = xpi + n; bases[kPlB] = rhs + n; bases[kPlC] = cC + n;
        bases[kPlW] = cW + n; bases[kPlE] = cE + n; bases[kPlS] = cS + n; bases[kPlN] = cN + n;
        int I0, J0;
        origin(it, I0, J0);
        mbar_arrive_expect_tx(&bar, region_bulk_bytes<T, RW, RH>(I0, it.nx));
    };
    auto stage_item = [&](const Item& it) {
        int I0, J0;
        origin(it, I0, J0);
        cheb_stage_region<T, RW, RH, 32 * NW>(bases, it.nx, it.ny, I0, J0, planes, &bar);
    };
    Item cur{-2, 0, 0, 0, 0, 0, 0, 0}, nxt{-2, 0, 0, 0, 0, 0, 0, 0};
    bool have = advance(cur, lo, nxt);
    if (tid == 0) {
        mbar_init(&bar, 1);
        if (have) announce(nxt);
    }
    __syncthreads();
    if (have) stage_item(nxt);
    unsigned phase = 0;
    // the group: this block's consecutive items of domain gd (first item gy, gn items)
    int gd = -1, gy = 0, gn = 0, gnt = 0;
    long long gpoff = 0;
    NormAcc<T> rsum;
    norm_zero(rsum);
    T dmax = T(0), rsc = T(0);
    double rinv2 = 0.0;
    auto flush = [&]() {
        if (gn == 0) return;
        double bs = 0.0, bm = 0.0;
        block_sum_max_scaled<T>(rsum, (double)dmax, bs, bm);   // into thread 0
        double acc[2];
        if (dom_publish_sum_max(bs * rinv2, bm, A.partials + gpoff, &A.sctl[gd].counter, gy, gn,
                                gnt, acc) &&
            tid == 0)
            kb_cheb_finish(A, gd, &A.sctl[gd], acc, K, stage);
        gn = 0;
        norm_zero(rsum);
        dmax = T(0);
    };
    while (have) {
        cur = nxt;
        cp_async_wait_all();
        const bool got = mbar_wait_bounded(&bar, phase, polls);
        if (__syncthreads_or(!got)) {
            const bool drained = cheb_drain(&bar, phase, true);
            if (tid == 0) {
                A.sctl[cur.d].status = drained ? 6 : 7;
                A.ds[cur.d].last_status[stage] = drained ? 6 : 7;
                atomicAdd(&A.ds[cur.d].nonconv, 1);
            }
            break;
        }
        phase ^= 1u;
        if (cur.d != gd) {   // the walk enters a domain: publish the last one's group
            flush();
            gd = cur.d;
            gy = cur.y;
            gnt = nt_of(cur);
            gpoff = A.dom[gd].poff;
            const SolveCtl* ctl = &A.sctl[gd];
            if (tid < K) {   // read by the sweeps after the region's first barrier
                c1s[tid] = sizeof(T) == 4 ? (T)ctl->c1f[tid] : (T)ctl->c1[tid];
                c2s[tid] = sizeof(T) == 4 ? (T)ctl->c2f[tid] : (T)ctl->c2[tid];
            }
            rsc = sizeof(T) == 4 ? (T)ctl->rscf : (T)ctl->rscd;
            rinv2 = ctl->rinv2;
        } else if (tid == 0) {   // pooled into the group's slot: this item's slot is zero
            A.partials[gpoff + 2 * (long long)cur.y] = 0.0;
            A.partials[gpoff + 2 * (long long)cur.y + 1] = 0.0;
        }
        have = advance(cur, cur.w + 1, nxt);
        auto next = [&](int part) {
            if (!have) return;
            if (part < 0) {   // before the barrier that frees the planes
                fence_proxy_async_smem();
                if (tid == 0) announce(nxt);
            } else {
                stage_item(nxt);
            }
        };
        Rows<T> Rw;
        const long long n = cur.n;
        Rw.cC = cC + n; Rw.cW = cW + n; Rw.cE = cE + n; Rw.cS = cS + n; Rw.cN = cN + n;
        Rw.nx = cur.nx; Rw.ny = cur.ny;
        int I0, J0;
        origin(cur, I0, J0);
        if constexpr (sizeof(T) == 4 && C == 2)
            cheb_region_reg2<R, NW, K>(Rw, planes, exch, c1s, c2s, rsc, I0, J0, xo + n, xpo + n,
                                       rsum, dmax, next);
        else
            cheb_region_reg<T, C, R, NW, K>(Rw, planes, exch, c1s, c2s, rsc, I0, J0, xo + n,
                                            xpo + n, rsum, dmax, next);
        ++gn;
    }
    flush();
}

// After the Chebyshev passes of a stage: a domain that ran an odd number of passes holds
// its iterate in the second buffer; copy it to dp (the correction and the fallback read dp).
template <typename T>
__global__ void __launch_bounds__(kThreads)
kb_settle(Arena<T> A, const int2* __restrict__ wl, int nw, const T* __restrict__ x2,
          T* __restrict__ dp, int K)
{
    for (int w = blockIdx.x; w < nw; w += gridDim.x) {
        const int2 it = wl[w];
        if (((A.sctl[it.x].sweeps / K) & 1) == 0) continue;
        const Dom<T>& D = A.dom[it.x];
        const long long n = D.noff, nn = (long long)(D.P.nx + 1) * (D.P.ny + 1);
        for (long long k = (long long)it.y * kChunk + threadIdx.x;
             k < nn && k < (long long)(it.y + 1) * kChunk; k += blockDim.x)
            dp[n + k] = x2[n + k];
    }
}

// Device side of the solver loops of a captured step: keep iterating while a domain is
// still solving (loop[k]) and the iteration cap is not reached (counter loop[k + 1]).
// count = 0 only evaluates the condition (before a loop's first body).
__global__ void kb_loop_cond(cudaGraphConditionalHandle h, unsigned* loop, int k, unsigned cap,
                             int count)
{
    if (threadIdx.x == 0) {
        const unsigned it = count ? ++loop[k + 1] : loop[k + 1];
        cudaGraphSetConditional(h, (loop[k] > 0u && it < cap) ? 1u : 0u);
    }
}

// Plan of one Chebyshev pass of a stage: the regions (TX x TY interior nodes each) of the
// domains still solving, counted in work-list order by one block.  More than `cap` of them:
// the pass walks the full work list (mode 0: converged domains' items are skipped there);
// 1 .. cap: their (domain, region) pairs are compacted into wl_act and a grid of resident
// blocks walks them (mode 1), so that the passes that only a few slowly converging domains
// still need do not launch a block per item of every domain; none: mode 2.  plan[0] =
// mode, plan[1] = length of wl_act.  In a captured step the plan also sets the conditions
// of the two branches' IF nodes (graph != 0).
template <typename T>
__global__ void __launch_bounds__(1024)
kb_cheb_plan(Arena<T> A, int n, const int* __restrict__ order, int TX, int TY, int cap,
             int2* __restrict__ wl_act, int* __restrict__ plan, int graph,
             cudaGraphConditionalHandle hbulk, cudaGraphConditionalHandle htail)
{
    __shared__ int wsum[32];
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5, nwarp = blockDim.x >> 5;
    auto items_of = [&](int i) {
        if (i >= n) return 0;
        const int d = order[i];
        if (A.sctl[d].done) return 0;
        const Prm<T>& P = A.dom[d].P;
        return cdiv(P.nx + 1, TX) * cdiv(P.ny + 1, TY);
    };
    // block-wide exclusive prefix of v (returned) and the block's total (tot)
    auto scan = [&](int v, int& tot) {
        int x = v;
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) wsum[wid] = x;
        __syncthreads();
        if (wid == 0) {
            int t = lane < nwarp ? wsum[lane] : 0;
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, t, o);
                if (lane >= o) t += y;
            }
            if (lane < nwarp) wsum[lane] = t;
        }
        __syncthreads();
        const int pre = (wid > 0 ? wsum[wid - 1] : 0) + x - v;
        tot = wsum[nwarp - 1];
        __syncthreads();   // wsum is rewritten by the next call
        return pre;
    };
    int total = 0;
    for (int c0 = 0; c0 < n; c0 += blockDim.x) {
        int t;
        scan(items_of(c0 + tid), t);
        total += t;
    }
    const int mode = total > cap ? 0 : (total > 0 ? 1 : 2);
    if (mode == 1) {
        int base = 0;
        for (int c0 = 0; c0 < n; c0 += blockDim.x) {
            const int v = items_of(c0 + tid);
            int t;
            const int pre = scan(v, t);
            for (int y = 0; y < v; ++y) wl_act[base + pre + y] = make_int2(order[c0 + tid], y);
            base += t;
        }
    }
    if (tid == 0) {
        plan[0] = mode;
        plan[1] = mode == 1 ? total : 0;
        if (graph) {
            cudaGraphSetConditional(hbulk, mode == 0 ? 1u : 0u);
            cudaGraphSetConditional(htail, mode == 1 ? 1u : 0u);
        }
    }
}

// ---- BiCGStab fallback (the single-domain k_bicg_* arithmetic, per domain), over node
// chunks; only domains with fb set take part.

template <typename T>
struct BiVec {
    T *cC, *cW, *cE, *cS, *cN, *b, *x, *r, *rh, *ph[2], *v[2], *t;
};

template <typename T>
__device__ __forceinline__ Rows<T> rows_at(const BiVec<T>& V, const Prm<T>& P, long long n)
{
    Rows<T> R;
    R.cC = V.cC + n; R.cW = V.cW + n; R.cE = V.cE + n; R.cS = V.cS + n; R.cN = V.cN + n;
    R.nx = P.nx; R.ny = P.ny;
    return R;
}

// Compact the (domain, chunk) list of the domains whose solve continues with BiCGStab
// (one thread per domain; the order of the domains in the list is immaterial: every
// reduction slot is the chunk's own index).
template <typename T>
__global__ void kb_build_fb(Arena<T> A, int n, int2* __restrict__ wl, int* __restrict__ count)
{
    const int d = blockIdx.x * blockDim.x + threadIdx.x;
    if (d >= n || !A.sctl[d].fb) return;
    const int k = A.dom[d].nnc;
    const int base = atomicAdd(count, k);
    for (int i = 0; i < k; ++i) wl[base + i] = make_int2(d, i);
}

// record the end of a domain's fallback solve
__device__ __forceinline__ void bicg_end(SolveCtl* ctl, DomState& s, unsigned* loop, int stage,
                                         int status)
{
    ctl->done = 1;
    ctl->status = status;
    ctl->fb = 0;
    atomicSub(&loop[2], 1u);
    s.fallbacks += 1;
    s.sweeps += ctl->iter;
    s.bicg_iters += ctl->iter;
    s.last_sweeps[stage] += ctl->iter;
    s.last_status[stage] = status;
    s.last_resid[stage] = ctl->bb > 0.0 ? sqrt(ctl->rr / ctl->bb) : 0.0;
    if (status != 1) s.nonconv += 1;
}

#define BATCH_NODE_LOOP(k, nn, chunk)                                                    \
    for (long long k = (long long)(chunk) * kChunk + threadIdx.x;                         \
         k < (nn) && k < (long long)((chunk) + 1) * kChunk; k += blockDim.x)

template <typename T>
__global__ void __launch_bounds__(kThreads)
kb_bicg_init(Arena<T> A, const int2* __restrict__ wl, const int* __restrict__ nwp, BiVec<T> V, int stage)
{
    const int nw = *nwp;   // compacted list of the domains in the fallback
    for (int w = blockIdx.x; w < nw; w += gridDim.x) {
        const int2 it = wl[w];
        SolveCtl* ctl = &A.sctl[it.x];
        if (!ctl->fb) continue;
        const Dom<T>& D = A.dom[it.x];
        const long long n = D.noff, nn = (long long)(D.P.nx + 1) * (D.P.ny + 1);
        const Rows<T> R = rows_at(V, D.P, n);
        const int nxn = D.P.nx + 1;
        const bool zero_rhs = ctl->bb == 0.0;
        T* x = V.x + n;
        const T* b = V.b + n;
        double acc[1] = {0.0};
        BATCH_NODE_LOOP(k, nn, it.y)
        {
            T rv;
            if (zero_rhs) {
                x[k] = T(0);
                rv = T(0);
            } else {
                const int I = (int)(k % nxn), J = (int)(k / nxn);
                rv = b[k] - row_apply(R, I, J, x[k], [&](size_t m) { return x[m]; });
            }
            V.r[n + k] = rv; V.rh[n + k] = rv; V.ph[0][n + k] = T(0); V.v[0][n + k] = T(0);
            acc[0] += (double)rv * (double)rv;
        }
        if (dom_reduce<1, 0u>(acc, A.partials + D.poff, &ctl->counter, it.y, D.nnc) &&
            threadIdx.x == 0) {
            ctl->rho1 = acc[0];
            ctl->rr = acc[0];
            ctl->rho = 1.0; ctl->alpha = 1.0; ctl->omega = 1.0;
            ctl->iter = 0;
            ctl->done = 0;
            ctl->status = 0;
            if (zero_rhs || acc[0] <= ctl->tol2 * ctl->bb) bicg_end(ctl, A.ds[it.x], A.loop, stage, 1);
        }
        __syncthreads();
    }
}

// phase A: p^ = r + beta (p^ - omega v); v = M D^-1 p^; alpha = rho1 / (rhat . v)
template <typename T>
__global__ void __launch_bounds__(kThreads)
kb_bicg_A(Arena<T> A, const int2* __restrict__ wl, const int* __restrict__ nwp, BiVec<T> V, int parity, int stage)
{
    const int nw = *nwp;   // compacted list of the domains in the fallback
    for (int w = blockIdx.x; w < nw; w += gridDim.x) {
        const int2 it = wl[w];
        SolveCtl* ctl = &A.sctl[it.x];
        if (!ctl->fb || ctl->done) continue;
        const Dom<T>& D = A.dom[it.x];
        const long long n = D.noff, nn = (long long)(D.P.nx + 1) * (D.P.ny + 1);
        const Rows<T> R = rows_at(V, D.P, n);
        const int nxn = D.P.nx + 1;
        const double beta_d = (ctl->rho1 / ctl->rho) * (ctl->alpha / ctl->omega);
        const T beta = (T)beta_d, om = (T)ctl->omega;
        const T* r = V.r + n;
        const T* ph_old = V.ph[parity] + n;
        const T* v_old = V.v[parity] + n;
        T* ph_new = V.ph[parity ^ 1] + n;
        T* v_new = V.v[parity ^ 1] + n;
        double acc[1] = {0.0};
        BATCH_NODE_LOOP(k, nn, it.y)
        {
            const int I = (int)(k % nxn), J = (int)(k / nxn);
            auto pnew = [&](size_t m) { return r[m] + beta * (ph_old[m] - om * v_old[m]); };
            const T pc = pnew((size_t)k);
            const T vc = row_apply(R, I, J, pc / R.cC[k], [&](size_t m) { return pnew(m) / R.cC[m]; });
            ph_new[k] = pc;
            v_new[k] = vc;
            acc[0] += (double)V.rh[n + k] * (double)vc;
        }
        if (dom_reduce<1, 0u>(acc, A.partials + D.poff, &ctl->counter, it.y, D.nnc) &&
            threadIdx.x == 0) {
            ctl->rv = acc[0];
            ctl->rho = ctl->rho1;
            if (acc[0] == 0.0 || !isfinite(acc[0])) bicg_end(ctl, A.ds[it.x], A.loop, stage, 3);
            else ctl->alpha = ctl->rho1 / acc[0];
        }
        __syncthreads();
    }
}

// phase B: s = r - alpha v; t = M D^-1 s; omega = (t . s) / (t . t)
template <typename T>
__global__ void __launch_bounds__(kThreads)
kb_bicg_B(Arena<T> A, const int2* __restrict__ wl, const int* __restrict__ nwp, BiVec<T> V, int parity)
{
    const int nw = *nwp;   // compacted list of the domains in the fallback
    for (int w = blockIdx.x; w < nw; w += gridDim.x) {
        const int2 it = wl[w];
        SolveCtl* ctl = &A.sctl[it.x];
        if (!ctl->fb || ctl->done) continue;
        const Dom<T>& D = A.dom[it.x];
        const long long n = D.noff, nn = (long long)(D.P.nx + 1) * (D.P.ny + 1);
        const Rows<T> R = rows_at(V, D.P, n);
        const int nxn = D.P.nx + 1;
        const T al = (T)ctl->alpha;
        const T* r = V.r + n;
        const T* v = V.v[parity ^ 1] + n;
        double acc[2] = {0.0, 0.0};
        BATCH_NODE_LOOP(k, nn, it.y)
        {
            const int I = (int)(k % nxn), J = (int)(k / nxn);
            auto sat = [&](size_t m) { return r[m] - al * v[m]; };
            const T sc = sat((size_t)k);
            const T tc = row_apply(R, I, J, sc / R.cC[k], [&](size_t m) { return sat(m) / R.cC[m]; });
            V.t[n + k] = tc;
            acc[0] += (double)tc * (double)sc;
            acc[1] += (double)tc * (double)tc;
        }
        if (dom_reduce<2, 0u>(acc, A.partials + D.poff, &ctl->counter, it.y, D.nnc) &&
            threadIdx.x == 0) {
            ctl->ts = acc[0];
            ctl->tt = acc[1];
            ctl->omega = acc[1] > 0.0 ? acc[0] / acc[1] : 0.0;
        }
        __syncthreads();
    }
}

// phase C: x += alpha D^-1 p^ + omega D^-1 s; r = s - omega t; rho1 = rhat . r; test
template <typename T>
__global__ void __launch_bounds__(kThreads)
kb_bicg_C(Arena<T> A, const int2* __restrict__ wl, const int* __restrict__ nwp, BiVec<T> V, int parity, int stage)
{
    const int nw = *nwp;   // compacted list of the domains in the fallback
    for (int w = blockIdx.x; w < nw; w += gridDim.x) {
        const int2 it = wl[w];
        SolveCtl* ctl = &A.sctl[it.x];
        if (!ctl->fb || ctl->done) continue;
        const Dom<T>& D = A.dom[it.x];
        const long long n = D.noff, nn = (long long)(D.P.nx + 1) * (D.P.ny + 1);
        const T al = (T)ctl->alpha, om = (T)ctl->omega;
        const T* ph = V.ph[parity ^ 1] + n;
        const T* v = V.v[parity ^ 1] + n;
        double acc[3] = {0.0, 0.0, 0.0};
        BATCH_NODE_LOOP(k, nn, it.y)
        {
            const T s = V.r[n + k] - al * v[k];
            const T dinv = T(1) / V.cC[n + k];
            const T dx = (al * ph[k] + om * s) * dinv;
            V.x[n + k] += dx;
            const T rn = s - om * V.t[n + k];
            V.r[n + k] = rn;
            acc[0] += (double)V.rh[n + k] * (double)rn;
            acc[1] += (double)rn * (double)rn;
            acc[2] = fmax(acc[2], (double)fabs(dx));
        }
        if (dom_reduce<3, 4u>(acc, A.partials + D.poff, &ctl->counter, it.y, D.nnc) &&
            threadIdx.x == 0) {
            ctl->rho1 = acc[0];
            ctl->rr = acc[1];
            ctl->dpmax = acc[2];
            ctl->iter += 1;
            // residual test, or criterion (32) on the iterate's change when eps_dp > 0
            if (acc[1] <= ctl->tol2 * ctl->bb || (ctl->eps_dp > 0.0 && acc[2] < ctl->eps_dp))
                bicg_end(ctl, A.ds[it.x], A.loop, stage, 1);
            else if (ctl->iter >= ctl->max_iter) bicg_end(ctl, A.ds[it.x], A.loop, stage, 2);
            else if (ctl->omega == 0.0 || acc[0] == 0.0 || !isfinite(acc[1]))
                bicg_end(ctl, A.ds[it.x], A.loop, stage, 3);
        }
        __syncthreads();
    }
}

// The whole fallback solve of a small domain (at most max_nodes nodes) in one block: the
// initial residual of kb_bicg_init and the iterations of kb_bicg_A / B / C with the same
// node arithmetic, each phase separated by a block barrier instead of a launch and its dot
// products summed by the block (FP64).  One block per domain (blockIdx.x = domain); a
// domain it ends leaves the fallback (bicg_end clears fb), so the chunked kernels and their
// loop see the other domains only.  In a step it runs on a side stream, concurrently with
// the Chebyshev passes of the other domains, on one SM per domain.
template <typename T>
__global__ void __launch_bounds__(1024, 1)
kb_bicg_small(Arena<T> A, BiVec<T> V, int stage, long long max_nodes)
{
    const int d = blockIdx.x;
    SolveCtl* ctl = &A.sctl[d];
    // only the domains the assembly sent to the fallback (status 4: the Chebyshev interval
    // does not hold); no Chebyshev pass touches them, so this kernel may run beside the
    // passes of the other domains
    if (!ctl->fb || ctl->status != 4) return;
    const Dom<T>& D = A.dom[d];
    const long long n = D.noff, nn = (long long)(D.P.nx + 1) * (D.P.ny + 1);
    if (nn > max_nodes) return;
    const Rows<T> R = rows_at(V, D.P, n);
    const int nxn = D.P.nx + 1;
    const int tid = threadIdx.x, nt = blockDim.x;
    // each thread takes its nodes U at a time: the U nodes' values are computed (their loads
    // in flight together) before any of them is stored (FP64: 2, within 64 registers)
    constexpr int U = sizeof(T) == 4 ? 4 : 2;
    const long long step = (long long)U * nt;
    __shared__ double res[3];
    __shared__ int stop;
    // the block's totals into res (the third a max; every thread after the next barrier)
    auto total1 = [&](double a0) {
        double v[1] = {a0};
        block_reduce<1, 0u>(v);
        if (tid == 0) res[0] = v[0];
    };
    auto total2 = [&](double a0, double a1) {
        double v[2] = {a0, a1};
        block_reduce<2, 0u>(v);
        if (tid == 0) { res[0] = v[0]; res[1] = v[1]; }
    };
    auto total3 = [&](double a0, double a1, double a2) {
        double v[3] = {a0, a1, a2};
        block_reduce<3, 4u>(v);
        if (tid == 0) { res[0] = v[0]; res[1] = v[1]; res[2] = v[2]; }
    };
    T* x = V.x + n;
    const T* b = V.b + n;
    T* r = V.r + n;
    T* rh = V.rh + n;
    T* t = V.t + n;
    {
        const bool zero_rhs = ctl->bb == 0.0;
        double a0 = 0.0;
        for (long long k0 = tid; k0 < nn; k0 += step) {
            T rv[U];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const long long k = k0 + (long long)u * nt;
                rv[u] = T(0);
                if (k < nn && !zero_rhs) {
                    const int I = (int)(k % nxn), J = (int)(k / nxn);
                    rv[u] = b[k] - row_apply(R, I, J, x[k], [&](size_t m) { return x[m]; });
                }
            }
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const long long k = k0 + (long long)u * nt;
                if (k >= nn) continue;
                if (zero_rhs) x[k] = T(0);
                r[k] = rv[u]; rh[k] = rv[u]; V.ph[0][n + k] = T(0); V.v[0][n + k] = T(0);
                a0 += (double)rv[u] * (double)rv[u];
            }
        }
        total1(a0);
        __syncthreads();
        if (tid == 0) {
            ctl->rho1 = res[0];
            ctl->rr = res[0];
            ctl->rho = 1.0; ctl->alpha = 1.0; ctl->omega = 1.0;
            ctl->iter = 0;
            // (done stays 1: the Chebyshev passes running beside this solve skip the domain)
            ctl->status = 0;
            stop = 0;
            if (zero_rhs || res[0] <= ctl->tol2 * ctl->bb) {
                bicg_end(ctl, A.ds[d], A.loop, stage, 1);
                stop = 1;
            }
        }
        __syncthreads();
    }
    for (int parity = 0; !stop; parity ^= 1) {
        const T* ph_old = (parity ? V.ph[1] : V.ph[0]) + n;
        const T* v_old = (parity ? V.v[1] : V.v[0]) + n;
        T* ph = (parity ? V.ph[0] : V.ph[1]) + n;
        T* v = (parity ? V.v[0] : V.v[1]) + n;
        // phase A: p^ = r + beta (p^ - omega v); v = M D^-1 p^; alpha = rho1 / (rhat . v)
        {
            const T beta = (T)((ctl->rho1 / ctl->rho) * (ctl->alpha / ctl->omega));
            const T om = (T)ctl->omega;
            auto pnew = [&](size_t m) { return r[m] + beta * (ph_old[m] - om * v_old[m]); };
            double a0 = 0.0;
            for (long long k0 = tid; k0 < nn; k0 += step) {
                T pc[U], vc[U], rr[U];
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    const long long k = k0 + (long long)u * nt;
                    pc[u] = vc[u] = rr[u] = T(0);
                    if (k < nn) {
                        const int I = (int)(k % nxn), J = (int)(k / nxn);
                        pc[u] = pnew((size_t)k);
                        vc[u] = row_apply(R, I, J, pc[u] / R.cC[k],
                                          [&](size_t m) { return pnew(m) / R.cC[m]; });
                        rr[u] = rh[k];
                    }
                }
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    const long long k = k0 + (long long)u * nt;
                    if (k >= nn) continue;
                    ph[k] = pc[u];
                    v[k] = vc[u];
                    a0 += (double)rr[u] * (double)vc[u];
                }
            }
            total1(a0);
            __syncthreads();
            if (tid == 0) {
                ctl->rv = res[0];
                ctl->rho = ctl->rho1;
                if (res[0] == 0.0 || !isfinite(res[0])) {
                    bicg_end(ctl, A.ds[d], A.loop, stage, 3);
                    stop = 1;
                } else {
                    ctl->alpha = ctl->rho1 / res[0];
                }
            }
            __syncthreads();
            if (stop) break;
        }
        // phase B: s = r - alpha v; t = M D^-1 s; omega = (t . s) / (t . t)
        {
            const T al = (T)ctl->alpha;
            auto sat = [&](size_t m) { return r[m] - al * v[m]; };
            double a0 = 0.0, a1 = 0.0;
            for (long long k0 = tid; k0 < nn; k0 += step) {
                T sc[U], tc[U];
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    const long long k = k0 + (long long)u * nt;
                    sc[u] = tc[u] = T(0);
                    if (k < nn) {
                        const int I = (int)(k % nxn), J = (int)(k / nxn);
                        sc[u] = sat((size_t)k);
                        tc[u] = row_apply(R, I, J, sc[u] / R.cC[k],
                                          [&](size_t m) { return sat(m) / R.cC[m]; });
                    }
                }
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    const long long k = k0 + (long long)u * nt;
                    if (k >= nn) continue;
                    t[k] = tc[u];
                    a0 += (double)tc[u] * (double)sc[u];
                    a1 += (double)tc[u] * (double)tc[u];
                }
            }
            total2(a0, a1);
            __syncthreads();
            if (tid == 0) {
                ctl->ts = res[0];
                ctl->tt = res[1];
                ctl->omega = res[1] > 0.0 ? res[0] / res[1] : 0.0;
            }
            __syncthreads();
        }
        // phase C: x += alpha D^-1 p^ + omega D^-1 s; r = s - omega t; rho1 = rhat . r; test
        {
            const T al = (T)ctl->alpha, om = (T)ctl->omega;
            double a0 = 0.0, a1 = 0.0, a2 = 0.0;
            for (long long k0 = tid; k0 < nn; k0 += step) {
                T xn[U], rn[U], dx[U], rr[U];
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    const long long k = k0 + (long long)u * nt;
                    xn[u] = rn[u] = dx[u] = rr[u] = T(0);
                    if (k < nn) {
                        const T s = r[k] - al * v[k];
                        const T dinv = T(1) / R.cC[k];
                        dx[u] = (al * ph[k] + om * s) * dinv;
                        xn[u] = x[k] + dx[u];
                        rn[u] = s - om * t[k];
                        rr[u] = rh[k];
                    }
                }
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    const long long k = k0 + (long long)u * nt;
                    if (k >= nn) continue;
                    x[k] = xn[u];
                    r[k] = rn[u];
                    a0 += (double)rr[u] * (double)rn[u];
                    a1 += (double)rn[u] * (double)rn[u];
                    a2 = fmax(a2, (double)fabs(dx[u]));
                }
            }
            total3(a0, a1, a2);
            __syncthreads();
            if (tid == 0) {
                ctl->rho1 = res[0];
                ctl->rr = res[1];
                ctl->dpmax = res[2];
                ctl->iter += 1;
                if (res[1] <= ctl->tol2 * ctl->bb || (ctl->eps_dp > 0.0 && res[2] < ctl->eps_dp)) {
                    bicg_end(ctl, A.ds[d], A.loop, stage, 1);
                    stop = 1;
                } else if (ctl->iter >= ctl->max_iter) {
                    bicg_end(ctl, A.ds[d], A.loop, stage, 2);
                    stop = 1;
                } else if (ctl->omega == 0.0 || res[0] == 0.0 || !isfinite(res[1])) {
                    bicg_end(ctl, A.ds[d], A.loop, stage, 3);
                    stop = 1;
                }
            }
            __syncthreads();
        }
    }
}

// Correction of q and w (and the Eq. (23) rate in the final stage) over a work list of
// (domain, tile) items of TX x TY nodes: corr_tile, the single-domain tile body.  Blocks
// walk contiguous shares [lo, hi) of the list (one item
// each when the grid has one block per item); the rates of a block's consecutive items of
// one domain are pooled and published once (the group's first slot holds them, its other
// slots zero), and the domain's last publication advances its clock and sets its next
// step (every item of the domain has read the step by then).
template <typename T, int TX, int TY>
__global__ void __launch_bounds__(kThreads, sizeof(T) == 4 ? 3 : 2)
kb_corr_t(Arena<T> A, const int2* __restrict__ wl, int nw, const T* eta, const T* H,
          const T* q1k, const T* q2k, const T* ws, const T* p, const T* dp, T* pout, T bfac,
          int with_p, T* eo, T* q1o, T* q2o, T* wo, int final_stage)
{
    const int lo = (int)((long long)nw * blockIdx.x / gridDim.x);
    const int hi = (int)((long long)nw * (blockIdx.x + 1) / gridDim.x);
    int gd = -1, gy = 0, gn = 0, gnt = 0;
    long long gpoff = 0;
    T lam = T(0);   // the group's rate (this thread's part)
    auto flush = [&]() {
        if (gn == 0) return;
        double v[1] = {(double)lam};
        block_reduce<1, 1u>(v);   // into thread 0
        double acc[2];
        if (dom_publish_sum_max(0.0, v[0], A.partials + gpoff, &A.stctl[gd].counter, gy, gn,
                                gnt, acc) &&
            threadIdx.x == 0) {
            DomState& s = A.ds[gd];
            s.t += s.dt;
            s.steps += 1;
            s.lam = acc[1];
            s.dt = A.fixed_dt > 0.0 ? A.fixed_dt : (acc[1] > 0.0 ? A.cfl / acc[1] : 0.0);
        }
        gn = 0;
        lam = T(0);
    };
    for (int w = lo; w < hi; ++w) {
        const int2 it = wl[w];
        const Dom<T>& D = A.dom[it.x];
        const Prm<T> P = D.P;
        const long long c = D.coff, n = D.noff;
        const int ntx = cdiv(P.nx + 1, TX);
        if (final_stage) {
            if (it.x != gd) {
                flush();
                gd = it.x;
                gy = it.y;
                gnt = ntx * cdiv(P.ny + 1, TY);
                gpoff = D.poff;
            } else if (threadIdx.x == 0) {
                A.partials[gpoff + 2 * (long long)it.y] = 0.0;
                A.partials[gpoff + 2 * (long long)it.y + 1] = 0.0;
            }
        }
        DomState& s = A.ds[it.x];
        const T de = bfac * (T)s.dt;
        int bad = 0;
        corr_tile<T, TX, TY>(P, eta + c, H + c, q1k + c, q2k + c, ws + n, p + n, dp + n,
                             pout + n, de, with_p, eo + c, q1o + c, q2o + c, wo + n,
                             final_stage, it.y % ntx, it.y / ntx, lam, bad);
        if (bad) atomicOr(&s.nonfinite, 1);
        if (final_stage) ++gn;
        __syncthreads();   // the tile's shared arrays are restaged by the next item
    }
    if (final_stage) flush();
}

// correction tiles of the batched form (nodes)
constexpr int kCorrTX = 32, kCorrTY = 16;

// ---------------------------------------------------------------- candidates

// Kernel shapes the autotuner chooses from (per precision).
struct Shape {
    int tx, ty, threads;
};

template <typename T> struct Cands;

template <typename T>
using HypFn = void (*)(int grid, cudaStream_t, const Arena<T>&, const int2*, int, const T*,
                       const T*, const T*, const T*, const T*, const T*, const T*, T, T, T*, T*,
                       T*);
template <typename T>
using AsmFn = void (*)(int grid, cudaStream_t, const Arena<T>&, const int2*, int, const T*,
                       const T*, T*, T*, const T*, const T*, const T*, const T*, T, T,
                       T*, T*, T*, T*, T*, T*, T*, const T*, AsmArgs);
template <typename T>
using ChebFn = void (*)(int grid, cudaStream_t, const Arena<T>&, const int2*, int, const T*,
                        const T*, const T*, const T*, const T*, const T*, const T*, const T*,
                        T*, T*, int, const int*, int);

template <typename T, int TX, int TY>
void run_hyp(int grid, cudaStream_t s, const Arena<T>& A, const int2* wl, int nw, const T* e,
             const T* a1, const T* a2, const T* eb, const T* ab, const T* bb, const T* H, T a,
             T b, T* eo, T* ao, T* bo)
{
    kb_hyp<T, TX, TY><<<grid, 256, 0, s>>>(A, wl, nw, e, a1, a2, eb, ab, bb, H, a, b, eo, ao, bo);
}

template <typename T, int TX, int TY>
void run_asm(int grid, cudaStream_t s, const Arena<T>& A, const int2* wl, int nw, const T* e,
             const T* H, T* q1k, T* q2k, const T* q1s, const T* q2s, const T* win,
             const T* wb, T a, T b, T* ws, T* cC, T* cW, T* cE, T* cS, T* cN, T* rhs,
             const T* p0, AsmArgs G)
{
    kb_asm<T, TX, TY><<<grid, 256, 0, s>>>(A, wl, nw, e, H, q1k, q2k, q1s, q2s, win, wb, a, b,
                                           ws, cC, cW, cE, cS, cN, rhs, p0, G);
}

// sweeps per pass of the batched Chebyshev passes (all candidates of a precision)
template <typename T> struct ChebK { static constexpr int value = sizeof(T) == 4 ? 8 : 4; };

template <typename T, int NA, int NB, int BY, bool REGW, bool PAD>
constexpr size_t cheb_smem()
{
    return PAD ? 2 * (size_t)(32 * NA + 2) * (BY * NB + 2) * sizeof(T)
               : (REGW ? 2 : 7) * (size_t)(32 * NA) * (BY * NB) * sizeof(T);
}

template <typename T, int NA, int NB, int BY, bool REGW, int MINB, bool PAD>
void run_cheb(int grid, cudaStream_t s, const Arena<T>& A, const int2* wl, int nw, const T* cC,
              const T* cW, const T* cE, const T* cS, const T* cN, const T* rhs, const T* xi,
              const T* xpi, T* xo, T* xpo, int stage, const int* plan, int want)
{
    kb_cheb<T, NA, NB, BY, ChebK<T>::value, REGW, MINB, PAD>
        <<<grid, dim3(32, BY), cheb_smem<T, NA, NB, BY, REGW, PAD>(), s>>>(
            A, wl, nw, cC, cW, cE, cS, cN, rhs, xi, xpi, xo, xpo, stage, plan, want);
}

#define KB_CHEB(T, NA, NB, BY, REGW, MINB, PAD) kb_cheb<T, NA, NB, BY, ChebK<T>::value, REGW, MINB, PAD>

// register form: region (32 C) x (R NW), 32 NW threads
template <typename T, int C, int R, int NW>
void run_cheb_reg(int grid, cudaStream_t s, const Arena<T>& A, const int2* wl, int nw,
                  const T* cC, const T* cW, const T* cE, const T* cS, const T* cN, const T* rhs,
                  const T* xi, const T* xpi, T* xo, T* xpo, int stage, const int* plan,
                  int want)
{
    kb_cheb_reg<T, C, R, NW, ChebK<T>::value>
        <<<grid, 32 * NW, cheb_reg_smem<T, C, R, NW>(), s>>>(A, wl, nw, cC, cW, cE, cS, cN, rhs,
                                                             xi, xpi, xo, xpo, stage, plan, want);
}

#define KB_CHEB_REG(T, C, R, NW) kb_cheb_reg<T, C, R, NW, ChebK<T>::value>

template <typename T>
struct Cand {
    Shape shape;
    const void* kernel;   // for occupancy queries
    size_t smem;
};

template <>
struct Cands<float> {
    static constexpr int nh = 3, na = 3, nc = 6;
    static Shape hyp_shape(int k) { const Shape s[nh] = {{32, 16, 256}, {32, 8, 256}, {64, 8, 256}}; return s[k]; }
    static HypFn<float> hyp(int k)
    {
        const HypFn<float> f[nh] = {run_hyp<float, 32, 16>, run_hyp<float, 32, 8>, run_hyp<float, 64, 8>};
        return f[k];
    }
    static const void* hyp_kernel(int k)
    {
        const void* f[nh] = {(const void*)kb_hyp<float, 32, 16>, (const void*)kb_hyp<float, 32, 8>,
                             (const void*)kb_hyp<float, 64, 8>};
        return f[k];
    }
    static Shape asm_shape(int k) { const Shape s[na] = {{32, 16, 256}, {32, 8, 256}, {64, 8, 256}}; return s[k]; }
    static AsmFn<float> assembly(int k)
    {
        const AsmFn<float> f[na] = {run_asm<float, 32, 16>, run_asm<float, 32, 8>, run_asm<float, 64, 8>};
        return f[k];
    }
    static const void* asm_kernel(int k)
    {
        const void* f[na] = {(const void*)kb_asm<float, 32, 16>, (const void*)kb_asm<float, 32, 8>,
                             (const void*)kb_asm<float, 64, 8>};
        return f[k];
    }
    // Chebyshev: region (tile + 8-node halo on every side) and threads, 8 sweeps per pass.
    // 0-3: weights in registers, padded buffers: regions 64x64 (1024 threads), 64x64 (512
    // threads, 1 block / SM), 128x64 (1024 threads), 128x64 (512 threads); 4-5: register
    // form (sweeps in registers, prefetched regions): 96x64 (512 threads), 64x64 (512
    // threads, packed FP32 pairs)
    static Shape cheb_shape(int k)
    {
        const Shape s[nc] = {{64, 64, 1024}, {64, 64, 512}, {128, 64, 1024},
                             {128, 64, 512}, {96, 64, 512},  {64, 64, 512}};
        return s[k];
    }
    static ChebFn<float> cheb(int k)
    {
        const ChebFn<float> f[nc] = {run_cheb<float, 2, 2, 32, true, 1, true>,
                                     run_cheb<float, 2, 4, 16, true, 1, true>,
                                     run_cheb<float, 4, 2, 32, true, 1, true>,
                                     run_cheb<float, 4, 4, 16, true, 1, true>,
                                     run_cheb_reg<float, 3, 4, 16>,
                                     run_cheb_reg<float, 2, 4, 16>};
        return f[k];
    }
    static const void* cheb_kernel(int k)
    {
        const void* f[nc] = {(const void*)KB_CHEB(float, 2, 2, 32, true, 1, true),
                             (const void*)KB_CHEB(float, 2, 4, 16, true, 1, true),
                             (const void*)KB_CHEB(float, 4, 2, 32, true, 1, true),
                             (const void*)KB_CHEB(float, 4, 4, 16, true, 1, true),
                             (const void*)KB_CHEB_REG(float, 3, 4, 16),
                             (const void*)KB_CHEB_REG(float, 2, 4, 16)};
        return f[k];
    }
    static bool cheb_is_reg(int k) { return k >= 4; }
    static size_t cheb_smem_of(int k)
    {
        const size_t s[nc] = {cheb_smem<float, 2, 2, 32, true, true>(),
                              cheb_smem<float, 2, 4, 16, true, true>(),
                              cheb_smem<float, 4, 2, 32, true, true>(),
                              cheb_smem<float, 4, 4, 16, true, true>(),
                              cheb_reg_smem<float, 3, 4, 16>(),
                              cheb_reg_smem<float, 2, 4, 16>()};
        return s[k];
    }
};

template <>
struct Cands<double> {
    static constexpr int nh = 2, na = 2, nc = 3;
    static Shape hyp_shape(int k) { const Shape s[nh] = {{32, 8, 256}, {16, 16, 256}}; return s[k]; }
    static HypFn<double> hyp(int k)
    {
        const HypFn<double> f[nh] = {run_hyp<double, 32, 8>, run_hyp<double, 16, 16>};
        return f[k];
    }
    static const void* hyp_kernel(int k)
    {
        const void* f[nh] = {(const void*)kb_hyp<double, 32, 8>, (const void*)kb_hyp<double, 16, 16>};
        return f[k];
    }
    // (static shared memory stays under 48 KB)
    static Shape asm_shape(int k) { const Shape s[na] = {{32, 8, 256}, {16, 16, 256}}; return s[k]; }
    static AsmFn<double> assembly(int k)
    {
        const AsmFn<double> f[na] = {run_asm<double, 32, 8>, run_asm<double, 16, 16>};
        return f[k];
    }
    static const void* asm_kernel(int k)
    {
        const void* f[na] = {(const void*)kb_asm<double, 32, 8>, (const void*)kb_asm<double, 16, 16>};
        return f[k];
    }
    // 4 sweeps per pass: 64x32 regions, shared-memory weights (512 or 256 threads), and the
    // register form (512 threads)
    static Shape cheb_shape(int k) { const Shape s[nc] = {{64, 32, 512}, {64, 32, 256}, {64, 32, 512}}; return s[k]; }
    static ChebFn<double> cheb(int k)
    {
        const ChebFn<double> f[nc] = {run_cheb<double, 2, 2, 16, false, 2, false>,
                                      run_cheb<double, 2, 4, 8, false, 2, false>,
                                      run_cheb_reg<double, 2, 2, 16>};
        return f[k];
    }
    static const void* cheb_kernel(int k)
    {
        const void* f[nc] = {(const void*)KB_CHEB(double, 2, 2, 16, false, 2, false),
                             (const void*)KB_CHEB(double, 2, 4, 8, false, 2, false),
                             (const void*)KB_CHEB_REG(double, 2, 2, 16)};
        return f[k];
    }
    static bool cheb_is_reg(int k) { return k == 2; }
    static size_t cheb_smem_of(int k)
    {
        const size_t s[nc] = {cheb_smem<double, 2, 2, 16, false, false>(),
                              cheb_smem<double, 2, 4, 8, false, false>(),
                              cheb_reg_smem<double, 2, 2, 16>()};
        return s[k];
    }
};


}  // namespace
}  // namespace nh

using namespace nh;

// ---------------------------------------------------------------- host runtime

struct BatchBase {
    virtual ~BatchBase() {}
    virtual int set_state(int d, const void* eta, const void* q1, const void* q2, const void* w,
                          const void* p, double t, int where) = 0;
    virtual int get_state(int d, void* eta, void* q1, void* q2, void* w, void* p, double* t,
                          int where) = 0;
    virtual int run(int nsteps) = 0;
    virtual int stats(int d, nh_stats_t* out) = 0;
    virtual int get_tuning(nh_batch_tuning* out) = 0;
    virtual int profile_enable(int on) = 0;
    virtual int profile_read(nh_profile_t* out) = 0;
    virtual int set_tuning(const nh_batch_tuning* in) = 0;
};

struct nh_batch {
    int n = 0;
    std::vector<nh_grid> grids;
    nh_params prm;
    int flags = 0;
    cudaStream_t s = nullptr;
    cudaStream_t own = nullptr;     // created when the caller passes the legacy stream
    cudaStream_t side = nullptr;    // capture of the solver-loop bodies
    cudaStream_t side2 = nullptr;   // capture of the branches inside a loop body
    cudaStream_t side3 = nullptr;   // fallback solves beside the Chebyshev passes
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    std::unique_ptr<BatchBase> impl;
    std::string err;
};

namespace {

int bfail(nh_batch* b, int code, const std::string& msg)
{
    if (b) b->err = msg;
    return code;
}

int bcuda(nh_batch* b, cudaError_t e, const char* where)
{
    return bfail(b, NH_ECUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

// CUDA-event pairs around launches, summed per kernel class (nh_profile_t).
struct BProf {
    bool on = false;
    std::vector<cudaEvent_t> pool;
    std::vector<int> cls;
    size_t used = 0;
    long long launches[NH_K_COUNT] = {};
    double ms[NH_K_COUNT] = {};
    ~BProf()
    {
        for (cudaEvent_t e : pool) cudaEventDestroy(e);
    }
    cudaEvent_t next()
    {
        if (used == pool.size()) {
            cudaEvent_t e;
            cudaEventCreate(&e);
            pool.push_back(e);
        }
        return pool[used++];
    }
    void flush()
    {
        if (used == 0) return;
        cudaEventSynchronize(pool[used - 1]);
        for (size_t k = 0; k < cls.size(); ++k) {
            float t = 0.f;
            cudaEventElapsedTime(&t, pool[2 * k], pool[2 * k + 1]);
            ms[cls[k]] += t;
            launches[cls[k]] += 1;
        }
        used = 0;
        cls.clear();
    }
    void reset()
    {
        flush();
        for (int k = 0; k < NH_K_COUNT; ++k) { launches[k] = 0; ms[k] = 0.0; }
    }
};

template <typename T>
struct BatchImpl : BatchBase {
    using C = Cands<T>;
    nh_batch* hb;
    int n;
    std::vector<Dom<T>> doms;
    std::vector<int> order;            // domains, largest first
    long long ncell = 0, nnode = 0;
    int nsm = 148;
    Bufs<T> B{};
    Dom<T>* d_dom = nullptr;
    DomState* d_ds = nullptr;
    SolveCtl* d_sctl = nullptr;
    StepCtl* d_stctl = nullptr;
    unsigned* d_loop = nullptr;
    unsigned* h_loop = nullptr;        // pinned
    // planned Chebyshev passes (kb_cheb_plan): domains in work-list order, the compacted
    // items of the few domains still solving, and the plan (mode, length)
    int* d_order = nullptr;
    int2* wl_act = nullptr;
    int* d_plan = nullptr;
    int cap_tail = 0;
    DomState* h_ds = nullptr;          // pinned
    std::vector<void*> allocs;
    // work lists: element items (cell chunks, node chunks) and one per tile candidate
    int2 *wl_cell = nullptr, *wl_node = nullptr, *wl_fb = nullptr, *wl_corr = nullptr;
    int nw_cell = 0, nw_node = 0, nw_corr = 0;
    std::vector<int2*> wl_hyp, wl_asm, wl_cheb;
    std::vector<int> nw_hyp, nw_asm, nw_cheb;
    nh_batch_tuning tun{};
    bool need_lambda = true;
    bool tuned_once = false;
    cudaGraphExec_t exec = nullptr;
    bool graph_failed = false;
    BProf prof;

    // launch f (one kernel on stream st) between two recorded events when profiling
    template <typename F>
    void K_(int c, cudaStream_t st, F&& f)
    {
        if (!prof.on) { f(); return; }
        if (prof.used + 2 > 16384) prof.flush();
        cudaEventRecord(prof.next(), st);
        f();
        cudaEventRecord(prof.next(), st);
        prof.cls.push_back(c);
    }

    ~BatchImpl() override
    {
        if (exec) cudaGraphExecDestroy(exec);
        for (void* p : allocs) cudaFree(p);
        if (h_loop) cudaFreeHost(h_loop);
        if (h_ds) cudaFreeHost(h_ds);
    }

    template <typename U>
    int alloc(U** p, size_t k)
    {
        void* q = nullptr;
        cudaError_t e = cudaMalloc(&q, k * sizeof(U) + 256);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return bfail(hb, NH_ENOMEM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
        }
        allocs.push_back(q);
        *p = static_cast<U*>(q);
        return NH_OK;
    }

    Arena<T> arena() const
    {
        Arena<T> A;
        A.dom = d_dom; A.sctl = d_sctl; A.stctl = d_stctl; A.ds = d_ds;
        A.partials = B.partials; A.loop = d_loop;
        A.fixed_dt = hb->prm.fixed_dt; A.cfl = hb->prm.cfl;
        A.polls = hb->prm.wait_polls > 0 ? (unsigned)hb->prm.wait_polls : kDefaultWaitPolls;
        return A;
    }

    // (domain, item) lists, largest domain first; items(d) = number of items of domain d
    template <typename F>
    int make_list(F items, int2** out, int* count)
    {
        std::vector<int2> v;
        for (int d : order) {
            const int k = items(d);
            for (int i = 0; i < k; ++i) v.push_back(make_int2(d, i));
        }
        int rc = alloc(out, v.size() + 1);
        if (rc != NH_OK) return rc;
        cudaMemcpyAsync(*out, v.data(), v.size() * sizeof(int2), cudaMemcpyHostToDevice, hb->s);
        *count = (int)v.size();
        return NH_OK;
    }

    int init(const double* const* Hs)
    {
        const nh_params& q = hb->prm;
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
        if (nsm <= 0) nsm = 148;
        doms.resize(n);
        long long poff = 0;
        for (int d = 0; d < n; ++d) {
            const nh_grid& g = hb->grids[d];
            Dom<T>& D = doms[d];
            Prm<T>& P = D.P;
            P.nx = g.nx; P.ny = g.ny;
            P.bcw = g.bc[0]; P.bce = g.bc[1]; P.bcs = g.bc[2]; P.bcn = g.bc[3];
            P.dx = (T)g.dx; P.dy = (T)g.dy;
            P.g = (T)q.g; P.delta = (T)q.delta; P.hdry = (T)q.hdry; P.manning = (T)q.manning_n;
            P.B1 = (T)q.B1; P.breaking = q.breaking; P.dry_zero = q.dry_zero ? 1 : 0;
            const long long nc = (long long)g.nx * g.ny, nn = (long long)(g.nx + 1) * (g.ny + 1);
            D.coff = ncell; D.noff = nnode;
            // keep every domain's arrays 256-byte aligned
            const long long al = 256 / (long long)sizeof(T);
            ncell += (nc + al - 1) / al * al;
            nnode += (nn + al - 1) / al * al;
            D.ncc = (int)((nc + kChunk - 1) / kChunk);
            D.nnc = (int)((nn + kChunk - 1) / kChunk);
            long long np = std::max<long long>(D.ncc, 3LL * D.nnc);   // (BiCGStab: 3 per chunk)
            for (int k = 0; k < C::na; ++k) {
                const Shape s = C::asm_shape(k);
                np = std::max<long long>(np, 3LL * cdiv(g.nx + 1, s.tx) * cdiv(g.ny + 1, s.ty));
            }
            for (int k = 0; k < C::nc; ++k) {
                const Shape s = C::cheb_shape(k);
                np = std::max<long long>(np, 2LL * cdiv(g.nx + 1, s.tx - 2 * ChebK<T>::value) *
                                                  cdiv(g.ny + 1, s.ty - 2 * ChebK<T>::value));
            }
            np = std::max<long long>(np, 2LL * cdiv(g.nx + 1, kCorrTX) * cdiv(g.ny + 1, kCorrTY));
            D.poff = poff;
            poff += (np + 31) / 32 * 32;
        }
        order.resize(n);
        std::iota(order.begin(), order.end(), 0);
        std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
            return (long long)hb->grids[a].nx * hb->grids[a].ny >
                   (long long)hb->grids[b].nx * hb->grids[b].ny;
        });
        int rc = NH_OK;
#define A_(ptr, k) if ((rc = alloc(&(ptr), (k))) != NH_OK) return rc
        A_(B.H, ncell);
        A_(B.eta, ncell); A_(B.q1, ncell); A_(B.q2, ncell);
        A_(B.eta1, ncell); A_(B.q11, ncell); A_(B.q21, ncell);
        A_(B.etas, ncell); A_(B.q1s, ncell); A_(B.q2s, ncell);
        if (q.breaking) { A_(B.q1k, ncell); A_(B.q2k, ncell); }
        else { B.q1k = B.q1s; B.q2k = B.q2s; }
        A_(B.w, nnode); A_(B.p, nnode); A_(B.w1, nnode); A_(B.ws, nnode);
        A_(B.dp, nnode); A_(B.palt, nnode); A_(B.r, nnode);
        A_(B.cC, nnode); A_(B.cW, nnode); A_(B.cE, nnode); A_(B.cS, nnode); A_(B.cN, nnode);
        A_(B.rhs, nnode);
        if (q.nonhydrostatic) {
            A_(B.rh, nnode); A_(B.ph[0], nnode); A_(B.ph[1], nnode);
            A_(B.v[0], nnode); A_(B.v[1], nnode); A_(B.t, nnode);
        }
        A_(B.partials, poff + 64);
        A_(d_dom, n);
        A_(d_ds, n);
        A_(d_sctl, n);
        A_(d_stctl, n);
        A_(d_loop, 8);   // [0..3] solver loops, [4] length of the fallback list
        cap_tail = 16 * nsm;
        A_(d_order, n);
        A_(wl_act, (size_t)cap_tail + 1);
        A_(d_plan, 4);
#undef A_
        cudaError_t e;
        if ((e = cudaMallocHost(&h_loop, 4 * sizeof(unsigned))) != cudaSuccess) return bcuda(hb, e, "cudaMallocHost");
        if ((e = cudaMallocHost(&h_ds, n * sizeof(DomState))) != cudaSuccess) return bcuda(hb, e, "cudaMallocHost");
        cudaStream_t s = hb->s;
        cudaMemcpyAsync(d_dom, doms.data(), n * sizeof(Dom<T>), cudaMemcpyHostToDevice, s);
        cudaMemsetAsync(d_ds, 0, n * sizeof(DomState), s);
        cudaMemsetAsync(d_stctl, 0, n * sizeof(StepCtl), s);
        cudaMemsetAsync(d_loop, 0, 8 * sizeof(unsigned), s);
        cudaMemsetAsync(d_plan, 0, 4 * sizeof(int), s);
        cudaMemcpyAsync(d_order, order.data(), n * sizeof(int), cudaMemcpyHostToDevice, s);
        {
            std::vector<SolveCtl> sc(n);
            std::memset(sc.data(), 0, n * sizeof(SolveCtl));
            for (auto& c : sc) c.eps_dp = q.eps_dp;
            cudaMemcpyAsync(d_sctl, sc.data(), n * sizeof(SolveCtl), cudaMemcpyHostToDevice, s);
            cudaStreamSynchronize(s);
        }
        // all node and cell arrays start at zero (padding included), then H and eta
        T* cell_arrays[] = {B.eta, B.q1, B.q2, B.eta1, B.q11, B.q21, B.etas, B.q1s, B.q2s, B.H};
        for (T* a : cell_arrays) cudaMemsetAsync(a, 0, ncell * sizeof(T), s);
        if (q.breaking) {
            cudaMemsetAsync(B.q1k, 0, ncell * sizeof(T), s);
            cudaMemsetAsync(B.q2k, 0, ncell * sizeof(T), s);
        }
        T* node_arrays[] = {B.w, B.p, B.w1, B.ws, B.dp, B.palt, B.r, B.cC, B.cW, B.cE, B.cS, B.cN, B.rhs,
                            B.rh, B.ph[0], B.ph[1], B.v[0], B.v[1], B.t};
        for (T* a : node_arrays)
            if (a) cudaMemsetAsync(a, 0, nnode * sizeof(T), s);
        for (int d = 0; d < n; ++d) {
            const nh_grid& g = hb->grids[d];
            const size_t nc = (size_t)g.nx * g.ny;
            std::vector<T> Hv(nc), e0(nc);
            for (size_t k = 0; k < nc; ++k) {
                Hv[k] = (T)Hs[d][k];
                e0[k] = (T)(Hs[d][k] > 0.0 ? 0.0 : -Hs[d][k]);
            }
            cudaMemcpyAsync(B.H + doms[d].coff, Hv.data(), nc * sizeof(T), cudaMemcpyHostToDevice, s);
            cudaMemcpyAsync(B.eta + doms[d].coff, e0.data(), nc * sizeof(T), cudaMemcpyHostToDevice, s);
            cudaStreamSynchronize(s);   // host vectors go out of scope
        }
        if ((rc = make_list([&](int d) { return doms[d].ncc; }, &wl_cell, &nw_cell)) != NH_OK) return rc;
        if ((rc = make_list([&](int d) { return doms[d].nnc; }, &wl_node, &nw_node)) != NH_OK) return rc;
        if ((rc = make_list([&](int d) {
                 return cdiv(doms[d].P.nx + 1, kCorrTX) * cdiv(doms[d].P.ny + 1, kCorrTY);
             }, &wl_corr, &nw_corr)) != NH_OK)
            return rc;
        if ((rc = alloc(&wl_fb, (size_t)nw_node + 1)) != NH_OK) return rc;
        wl_hyp.resize(C::nh); nw_hyp.resize(C::nh);
        for (int k = 0; k < C::nh; ++k) {
            const Shape sh = C::hyp_shape(k);
            rc = make_list([&](int d) { return cdiv(doms[d].P.nx, sh.tx) * cdiv(doms[d].P.ny, sh.ty); },
                           &wl_hyp[k], &nw_hyp[k]);
            if (rc != NH_OK) return rc;
        }
        wl_asm.resize(C::na); nw_asm.resize(C::na);
        for (int k = 0; k < C::na; ++k) {
            const Shape sh = C::asm_shape(k);
            rc = make_list([&](int d) { return cdiv(doms[d].P.nx + 1, sh.tx) * cdiv(doms[d].P.ny + 1, sh.ty); },
                           &wl_asm[k], &nw_asm[k]);
            if (rc != NH_OK) return rc;
        }
        wl_cheb.resize(C::nc); nw_cheb.resize(C::nc);
        for (int k = 0; k < C::nc; ++k) {
            const Shape sh = C::cheb_shape(k);
            rc = make_list([&](int d) {
                return cdiv(doms[d].P.nx + 1, sh.tx - 2 * ChebK<T>::value) * cdiv(doms[d].P.ny + 1, sh.ty - 2 * ChebK<T>::value);
            }, &wl_cheb[k], &nw_cheb[k]);
            if (rc != NH_OK) return rc;
            if ((e = cudaFuncSetAttribute(C::cheb_kernel(k), cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          (int)C::cheb_smem_of(k))) != cudaSuccess)
                return bcuda(hb, e, "cudaFuncSetAttribute");
        }
        if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return bcuda(hb, e, "nh_create_batch");
        if ((e = cudaGetLastError()) != cudaSuccess) return bcuda(hb, e, "nh_create_batch");
        // defaults until tuned: the single-domain shapes, one block per item
        tun = nh_batch_tuning{};
        tun.hyp = 0; tun.assembly = 0; tun.cheb = 0;
        tun.persistent = 0;
        tun.graph = (hb->flags & NH_BATCH_GRAPH) ? 1 : 0;
        tun.tuned = 0;
        return NH_OK;
    }

    // grid of a launch: one block per item, or the resident capacity (persistent)
    std::vector<std::pair<const void*, int>> occ;   // resident blocks per SM, per kernel
    int grid_of(const void* kernel, int threads, size_t smem, int items, bool persistent)
    {
        if (items <= 0) return 1;
        if (!persistent) return items;
        int per = -1;
        for (auto& o : occ)
            if (o.first == kernel) per = o.second;
        if (per < 0) {
            if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kernel, threads, smem) != cudaSuccess || per < 1) {
                cudaGetLastError();
                per = 1;
            }
            occ.emplace_back(kernel, per);
        }
        const int g = per * nsm;
        return g < items ? g : items;
    }
    bool pers(int cls) const { return (tun.persistent >> cls) & 1; }

    int launch_lambda()
    {
        kb_lambda<T><<<grid_of((const void*)kb_lambda<T>, kThreads, 0, nw_cell, true), kThreads, 0, hb->s>>>(
            arena(), wl_cell, nw_cell, B.eta, B.q1, B.q2, B.H);
        return cudaGetLastError() == cudaSuccess ? NH_OK : NH_ECUDA;
    }

    void hyp(int s, int cand, bool persistent)
    {
        const T a = s == 0 ? T(0) : T(0.5), b = s == 0 ? T(1) : T(0.5);
        const T* ein = s == 0 ? B.eta : B.eta1;
        const T* ain = s == 0 ? B.q1 : B.q11;
        const T* bin = s == 0 ? B.q2 : B.q21;
        const Shape sh = C::hyp_shape(cand);
        C::hyp(cand)(grid_of(C::hyp_kernel(cand), sh.threads, 0, nw_hyp[cand], persistent), hb->s,
                     arena(), wl_hyp[cand], nw_hyp[cand], ein, ain, bin, B.eta, B.q1, B.q2, B.H,
                     a, b, B.etas, B.q1s, B.q2s);
    }

    void assembly(int s, int cand, bool persistent)
    {
        const nh_params& q = hb->prm;
        const T a = s == 0 ? T(0) : T(0.5), b = s == 0 ? T(1) : T(0.5);
        const T* win = s == 0 ? B.w : B.w1;
        AsmArgs G;
        G.tol2 = q.tol * q.tol;
        G.max_iter = q.max_iter;
        G.kpass = ChebK<T>::value;
        G.with_coef = q.nonhydrostatic ? 1 : 0;
        G.stage = s;
        G.fuse = 1;
        const Shape sh = C::asm_shape(cand);
        C::assembly(cand)(grid_of(C::asm_kernel(cand), sh.threads, 0, nw_asm[cand], persistent),
                          hb->s, arena(), wl_asm[cand], nw_asm[cand], B.etas, B.H, B.q1k, B.q2k,
                          B.q1s, B.q2s, win, B.w, a, b, B.ws, B.cC, B.cW, B.cE, B.cS, B.cN, B.rhs,
                          B.p, G);
    }

    // pass `odd`: reads (dp, r) and writes (v[0], v[1]) when 0, the other way when 1;
    // over the items wl[0 .. nw) on `grid` blocks, or the branch `want` of a plan
    void cheb_launch(int s, int cand, int grid, cudaStream_t st, int odd, const int2* wl, int nw,
                     const int* plan, int want)
    {
        T* xa = odd ? B.v[0] : B.dp;
        T* pa = odd ? B.v[1] : B.r;
        T* xb = odd ? B.dp : B.v[0];
        T* pb = odd ? B.r : B.v[1];
        C::cheb(cand)(grid, st, arena(), wl, nw, B.cC, B.cW, B.cE, B.cS, B.cN, B.rhs, xa, pa, xb,
                      pb, s, plan, want);
    }
    // grid of a pass of candidate cand over the full list: one block per item; or (the
    // tuning's persistent form) for the register forms chunks of kRegChunk consecutive items
    // a block, for the others the resident blocks.  Chunks keep the hardware's in-order
    // block scheduling, under which the regions being swept at a time are neighbours whose
    // shared rows stay in L2, and let each block prefetch its next region and publish one
    // residual sum per chunk (a resident grid of register-form blocks walking whole shares
    // loses that locality).
    static constexpr int kRegChunk = 8;
    int cheb_grid(int cand, bool persistent)
    {
        const int nw = nw_cheb[cand];
        if (persistent && C::cheb_is_reg(cand)) return nw > 0 ? (nw + kRegChunk - 1) / kRegChunk : 1;
        const Shape sh = C::cheb_shape(cand);
        return grid_of(C::cheb_kernel(cand), sh.threads, C::cheb_smem_of(cand), nw, persistent);
    }
    // an unplanned pass over the full work list (the autotuner's timings)
    void cheb_pass(int s, int cand, bool persistent, cudaStream_t st, int odd)
    {
        cheb_launch(s, cand, cheb_grid(cand, persistent), st, odd, wl_cheb[cand], nw_cheb[cand],
                    nullptr, 0);
    }
    // the plan of a pass of the tuned candidate (graph: set the branch conditions too)
    void cheb_plan(cudaStream_t st, int graph, cudaGraphConditionalHandle hbulk,
                   cudaGraphConditionalHandle htail)
    {
        const Shape sh = C::cheb_shape(tun.cheb);
        constexpr int K = ChebK<T>::value;
        kb_cheb_plan<T><<<1, 1024, 0, st>>>(arena(), n, d_order, sh.tx - 2 * K, sh.ty - 2 * K,
                                            cap_tail, wl_act, d_plan, graph, hbulk, htail);
    }
    // the two branches of a planned pass: the tuned launch over the full list, or a grid of
    // resident blocks over the compacted items
    void cheb_bulk(int s, cudaStream_t st, int odd)
    {
        const int cand = tun.cheb;
        cheb_launch(s, cand, cheb_grid(cand, pers(2)), st, odd, wl_cheb[cand], nw_cheb[cand],
                    d_plan, 0);
    }
    void cheb_tail(int s, cudaStream_t st, int odd)
    {
        const int cand = tun.cheb;
        const Shape sh = C::cheb_shape(cand);
        cheb_launch(s, cand, grid_of(C::cheb_kernel(cand), sh.threads, C::cheb_smem_of(cand),
                                     cap_tail, true),
                    st, odd, wl_act, cap_tail, d_plan, 1);
    }
    // two eager passes (the buffer pairs alternate, so a pair of passes restores them); each
    // launches its plan and both branches, of which the one the plan did not choose returns
    void cheb_pair(int s, cudaStream_t st)
    {
        for (int odd = 0; odd < 2; ++odd)
            K_(NH_K_CHEB_PASS, st, [&] {
                cheb_plan(st, 0, 0, 0);
                cheb_bulk(s, st, odd);
                cheb_tail(s, st, odd);
            });
    }
    // the same two passes inside a captured loop body (stream bs): plan, then one IF node
    // per branch, whose bodies are captured on side2
    template <typename Chk>
    void cheb_pair_graph(int s, cudaStream_t bs, Chk& chk)
    {
        for (int odd = 0; odd < 2; ++odd) {
            cudaStreamCaptureStatus cs;
            cudaGraph_t g = nullptr;
            chk(cudaStreamGetCaptureInfo(bs, &cs, nullptr, &g, nullptr, nullptr, nullptr));
            cudaGraphConditionalHandle hbulk = 0, htail = 0;
            chk(cudaGraphConditionalHandleCreate(&hbulk, g, 0, cudaGraphCondAssignDefault));
            chk(cudaGraphConditionalHandleCreate(&htail, g, 0, cudaGraphCondAssignDefault));
            cheb_plan(bs, 1, hbulk, htail);
            add_cond(bs, hb->side2, chk, hbulk, cudaGraphCondTypeIf,
                     [&](cudaStream_t ts) { cheb_bulk(s, ts, odd); });
            add_cond(bs, hb->side2, chk, htail, cudaGraphCondTypeIf,
                     [&](cudaStream_t ts) { cheb_tail(s, ts, odd); });
        }
    }
    void settle(cudaStream_t st)
    {
        kb_settle<T><<<grid_of((const void*)kb_settle<T>, kThreads, 0, nw_node, true), kThreads, 0, st>>>(
            arena(), wl_node, nw_node, B.v[0], B.dp, ChebK<T>::value);
    }

    unsigned pass_cap() const { return (unsigned)((hb->prm.max_iter / ChebK<T>::value + 16) / 2); }   // pairs
    unsigned bicg_cap() const { return (unsigned)(hb->prm.max_iter / 2 + 2); }

    BiVec<T> bivec() const
    {
        BiVec<T> V;
        V.cC = B.cC; V.cW = B.cW; V.cE = B.cE; V.cS = B.cS; V.cN = B.cN;
        V.b = B.rhs; V.x = B.dp; V.r = B.r; V.rh = B.rh;
        V.ph[0] = B.ph[0]; V.ph[1] = B.ph[1]; V.v[0] = B.v[0]; V.v[1] = B.v[1]; V.t = B.t;
        return V;
    }

    const int* nfb() const { return reinterpret_cast<const int*>(d_loop + 4); }

    // the fallback solves that the assembly decided (status 4) of the domains of at most
    // nh_params.fallback_block_nodes nodes, one block each
    void bicg_small(int s, cudaStream_t st)
    {
        const long long lim = hb->prm.fallback_block_nodes;
        if (lim <= 0) return;
        K_(NH_K_BICG_BLOCK, st, [&] {
            kb_bicg_small<T><<<n, 1024, 0, st>>>(arena(), bivec(), s, lim);
        });
    }

    // compacted list of the fallback domains' chunks, then the BiCGStab initial residual
    void bicg_init(int s, cudaStream_t st)
    {
        kb_build_fb<T><<<(n + 127) / 128, 128, 0, st>>>(arena(), n, wl_fb,
                                                       reinterpret_cast<int*>(d_loop + 4));
        K_(NH_K_SOLVE_INIT, st, [&] {
            kb_bicg_init<T><<<grid_of((const void*)kb_bicg_init<T>, kThreads, 0, nw_node, true), kThreads, 0, st>>>(
                arena(), wl_fb, nfb(), bivec(), s);
        });
    }

    // two BiCGStab iterations (the p^ / v buffers alternate, so a pair restores them)
    void bicg_pair(int s, cudaStream_t st)
    {
        const BiVec<T> V = bivec();
        for (int parity = 0; parity < 2; ++parity) {
            K_(NH_K_BICG_A, st, [&] {
                kb_bicg_A<T><<<grid_of((const void*)kb_bicg_A<T>, kThreads, 0, nw_node, true), kThreads, 0, st>>>(
                    arena(), wl_fb, nfb(), V, parity, s);
            });
            K_(NH_K_BICG_B, st, [&] {
                kb_bicg_B<T><<<grid_of((const void*)kb_bicg_B<T>, kThreads, 0, nw_node, true), kThreads, 0, st>>>(
                    arena(), wl_fb, nfb(), V, parity);
            });
            K_(NH_K_BICG_C, st, [&] {
                kb_bicg_C<T><<<grid_of((const void*)kb_bicg_C<T>, kThreads, 0, nw_node, true), kThreads, 0, st>>>(
                    arena(), wl_fb, nfb(), V, parity, s);
            });
        }
    }

    // the stage up to the solve (hyperbolic step, breaking, assembly)
    void pre_solve(int s)
    {
        const nh_params& q = hb->prm;
        K_(NH_K_HYPERBOLIC, hb->s, [&] { hyp(s, tun.hyp, pers(0)); });
        // the breaking terms (q* -> q**) run inside the assembly
        cudaMemsetAsync(d_loop, 0, 8 * sizeof(unsigned), hb->s);
        if (q.nonhydrostatic) cudaMemsetAsync(B.dp, 0, nnode * sizeof(T), hb->s);
        K_(NH_K_ASSEMBLY, hb->s, [&] { assembly(s, tun.assembly, pers(1)); });
    }

    void post_solve(int s)
    {
        const nh_params& q = hb->prm;
        T* eo = s == 0 ? B.eta1 : B.eta;
        T* ao = s == 0 ? B.q11 : B.q1;
        T* bo = s == 0 ? B.q21 : B.q2;
        T* wo = s == 0 ? B.w1 : B.w;
        const T b = s == 0 ? T(1) : T(0.5);
        K_(NH_K_CORRECTION, hb->s, [&] {
            kb_corr_t<T, kCorrTX, kCorrTY><<<grid_of((const void*)kb_corr_t<T, kCorrTX, kCorrTY>, kThreads, 0, nw_corr, pers(3)), kThreads, 0, hb->s>>>(
                arena(), wl_corr, nw_corr, B.etas, B.H, B.q1k, B.q2k, B.ws, B.p, B.dp, B.palt, b,
                q.nonhydrostatic ? 1 : 0, eo, ao, bo, wo, s == 1 ? 1 : 0);
        });
        std::swap(B.p, B.palt);
    }

    // eager solve: passes in batches, the host reads the number of domains still solving;
    // then the BiCGStab fallback for the domains that need it
    int solve_eager(int s)
    {
        unsigned passes = 0;   // pairs of passes
        int batch = 2;
        cudaError_t e;
        bicg_small(s, hb->s);   // (beside the passes in a captured step)
        for (;;) {
            for (int k = 0; k < batch; ++k) cheb_pair(s, hb->s);
            passes += batch;
            cudaMemcpyAsync(h_loop, d_loop, 4 * sizeof(unsigned), cudaMemcpyDeviceToHost, hb->s);
            if ((e = cudaStreamSynchronize(hb->s)) != cudaSuccess) return bcuda(hb, e, "batched pressure solve");
            if (h_loop[0] == 0u || passes >= pass_cap()) break;
            batch = 1;
        }
        settle(hb->s);
        if (h_loop[2] == 0u) return NH_OK;
        bicg_init(s, hb->s);
        for (unsigned pairs = 0; pairs < bicg_cap();) {
            for (int k = 0; k < 2; ++k, ++pairs) bicg_pair(s, hb->s);
            cudaMemcpyAsync(h_loop, d_loop, 4 * sizeof(unsigned), cudaMemcpyDeviceToHost, hb->s);
            if ((e = cudaStreamSynchronize(hb->s)) != cudaSuccess) return bcuda(hb, e, "batched BiCGStab");
            if (h_loop[2] == 0u) break;
        }
        return NH_OK;
    }

    int step_eager()
    {
        for (int s = 0; s < 2; ++s) {
            pre_solve(s);
            if (hb->prm.nonhydrostatic) {
                int rc = solve_eager(s);
                if (rc != NH_OK) return rc;
            }
            post_solve(s);
        }
        cudaError_t e = cudaGetLastError();
        return e == cudaSuccess ? NH_OK : bcuda(hb, e, "batched step");
    }

    // Append to the capture on stream s a conditional node of `type` on handle h, whose body
    // is captured from body(bs) on stream bs.
    template <typename Chk, typename Body>
    void add_cond(cudaStream_t s, cudaStream_t bs, Chk& chk, cudaGraphConditionalHandle h,
                  cudaGraphConditionalNodeType type, Body&& body)
    {
        cudaStreamCaptureStatus cs;
        cudaGraph_t g = nullptr;
        const cudaGraphNode_t* deps = nullptr;
        size_t nd = 0;
        chk(cudaStreamGetCaptureInfo(s, &cs, nullptr, &g, &deps, nullptr, &nd));
        // (the params union has no default constructor: zeroed storage)
        alignas(cudaGraphNodeParams) unsigned char npb[sizeof(cudaGraphNodeParams)] = {};
        cudaGraphNodeParams& np = *reinterpret_cast<cudaGraphNodeParams*>(npb);
        np.type = cudaGraphNodeTypeConditional;
        np.conditional.handle = h;
        np.conditional.type = type;
        np.conditional.size = 1;
        cudaGraphNode_t node = nullptr;
        chk(cudaGraphAddNode(&node, g, deps, nullptr, nd, &np));
        if (!node) return;
        cudaGraph_t bodyg = np.conditional.phGraph_out[0];
        chk(cudaStreamUpdateCaptureDependencies(s, &node, nullptr, 1, cudaStreamSetCaptureDependencies));
        chk(cudaStreamBeginCaptureToGraph(bs, bodyg, nullptr, nullptr, 0,
                                          cudaStreamCaptureModeThreadLocal));
        body(bs);
        chk(cudaGetLastError());
        cudaGraph_t bout = nullptr;
        chk(cudaStreamEndCapture(bs, &bout));
    }

    // Append to the capture on stream s a conditional WHILE node whose body is captured from
    // body(side stream, handle); pre(handle), when given, is captured before the node and
    // sets the first condition (the handle's default value is dflt).
    template <typename Chk, typename Body, typename Pre>
    void add_while(cudaStream_t s, Chk& chk, unsigned dflt, Body&& body, Pre&& pre)
    {
        cudaStreamCaptureStatus cs;
        cudaGraph_t g = nullptr;
        chk(cudaStreamGetCaptureInfo(s, &cs, nullptr, &g, nullptr, nullptr, nullptr));
        cudaGraphConditionalHandle h = 0;
        chk(cudaGraphConditionalHandleCreate(&h, g, dflt, cudaGraphCondAssignDefault));
        call_pre(pre, h);
        add_cond(s, hb->side, chk, h, cudaGraphCondTypeWhile,
                 [&](cudaStream_t bs) { body(bs, h); });
    }
    template <typename Pre>
    static void call_pre(Pre& pre, cudaGraphConditionalHandle h) { pre(h); }
    static void call_pre(std::nullptr_t, cudaGraphConditionalHandle) {}

    // one step as a graph; the solver loops are conditional WHILE nodes
    int build_graph()
    {
        cudaStream_t s = hb->s;
        cudaError_t e = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) return bcuda(hb, e, "cudaStreamBeginCapture");
        cudaError_t first = cudaSuccess;
        auto chk = [&](cudaError_t x) { if (first == cudaSuccess && x != cudaSuccess) first = x; };
        for (int st = 0; st < 2; ++st) {
            pre_solve(st);
            if (hb->prm.nonhydrostatic) {
                // the small domains whose rows fail the Gershgorin test: their BiCGStab solves
                // on side3, beside the Chebyshev passes of the others
                chk(cudaEventRecord(hb->ev_fork, s));
                chk(cudaStreamWaitEvent(hb->side3, hb->ev_fork, 0));
                bicg_small(st, hb->side3);
                chk(cudaEventRecord(hb->ev_join, hb->side3));
                // Chebyshev passes: WHILE (domains solving) { pass; test }
                add_while(s, chk, 1, [&](cudaStream_t bs, cudaGraphConditionalHandle h) {
                    cheb_pair_graph(st, bs, chk);
                    kb_loop_cond<<<1, 32, 0, bs>>>(h, d_loop, 0, pass_cap(), 1);
                }, nullptr);
                chk(cudaStreamWaitEvent(s, hb->ev_join, 0));
                settle(s);
                // fallback for the others (stalled Chebyshev solves, larger domains): init;
                // WHILE (domains in BiCGStab) { two iterations; test }
                bicg_init(st, s);
                add_while(s, chk, 0, [&](cudaStream_t bs, cudaGraphConditionalHandle h) {
                    bicg_pair(st, bs);
                    kb_loop_cond<<<1, 32, 0, bs>>>(h, d_loop, 2, bicg_cap(), 1);
                }, [&](cudaGraphConditionalHandle h) {
                    kb_loop_cond<<<1, 32, 0, s>>>(h, d_loop, 2, bicg_cap(), 0);
                });
            }
            post_solve(st);
        }
        chk(cudaGetLastError());
        cudaGraph_t graph = nullptr;
        e = cudaStreamEndCapture(s, &graph);
        if (first == cudaSuccess) first = e;
        if (first == cudaSuccess) first = cudaGraphInstantiate(&exec, graph, 0);
        if (graph) cudaGraphDestroy(graph);
        if (first != cudaSuccess) {
            cudaGetLastError();
            exec = nullptr;
            return bcuda(hb, first, "step graph");
        }
        return NH_OK;
    }

    float time_ms(const std::function<void()>& f, int reps)
    {
        cudaEvent_t a, b;
        cudaEventCreate(&a);
        cudaEventCreate(&b);
        f();   // warm-up
        cudaEventRecord(a, hb->s);
        for (int k = 0; k < reps; ++k) f();
        cudaEventRecord(b, hb->s);
        cudaEventSynchronize(b);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, a, b);
        cudaEventDestroy(a);
        cudaEventDestroy(b);
        return ms / reps;
    }

    // Time every candidate (and grid form) of the hyperbolic, assembly and Chebyshev
    // kernels on the current state, stage-1 arguments; keep the fastest.  The state itself
    // is not changed (only scratch arrays), and the per-domain counters are restored.
    int autotune()
    {
        cudaStream_t s = hb->s;
        cudaMemcpyAsync(h_ds, d_ds, n * sizeof(DomState), cudaMemcpyDeviceToHost, s);
        cudaStreamSynchronize(s);
        const int reps = 3;
        float best = 1e30f;
        for (int k = 0; k < C::nh; ++k)
            for (int p = 0; p < 2; ++p) {
                const float t = time_ms([&] { hyp(0, k, p == 1); }, reps);
                if (t < best) { best = t; tun.hyp = k; tun.persistent = (tun.persistent & ~1) | p; }
            }
        tun.ms[0] = best;
        hyp(0, tun.hyp, pers(0));
        best = 1e30f;
        for (int k = 0; k < C::na; ++k)
            for (int p = 0; p < 2; ++p) {
                const float t = time_ms([&] { assembly(0, k, p == 1); }, reps);
                if (t < best) { best = t; tun.assembly = k; tun.persistent = (tun.persistent & ~2) | (p << 1); }
            }
        tun.ms[1] = best;
        if (hb->prm.nonhydrostatic) {
            best = 1e30f;
            for (int k = 0; k < C::nc; ++k)
                for (int p = 0; p < 2; ++p) {
                    cudaMemsetAsync(B.dp, 0, nnode * sizeof(T), s);
                    assembly(0, tun.assembly, pers(1));
                    int odd = 0;
                    const float t = time_ms([&] { cheb_pass(0, k, p == 1, s, odd); odd ^= 1; }, 2 * reps);
                    if (t < best) { best = t; tun.cheb = k; tun.persistent = (tun.persistent & ~4) | (p << 2); }
                }
            tun.ms[2] = best;
        }
        {
            // the correction: compare its two grid forms on a stage-1 correction writing into
            // the stage-1 outputs (overwritten by the real step)
            float tb[2];
            for (int p = 0; p < 2; ++p) {
                const int gsz = grid_of((const void*)kb_corr_t<T, kCorrTX, kCorrTY>, kThreads, 0, nw_corr, p == 1);
                tb[p] = time_ms([&] {
                    kb_corr_t<T, kCorrTX, kCorrTY><<<gsz, kThreads, 0, s>>>(
                        arena(), wl_corr, nw_corr, B.etas, B.H, B.q1k, B.q2k, B.ws, B.p, B.dp,
                        B.palt, T(1), 0, B.eta1, B.q11, B.q21, B.w1, 0);
                }, reps);
            }
            tun.persistent = (tun.persistent & ~8) | ((tb[1] < tb[0] ? 1 : 0) << 3);
        }
        cudaMemsetAsync(d_loop, 0, 8 * sizeof(unsigned), s);
        cudaMemcpyAsync(d_ds, h_ds, n * sizeof(DomState), cudaMemcpyHostToDevice, s);
        cudaError_t e = cudaStreamSynchronize(s);
        if (e == cudaSuccess) e = cudaGetLastError();
        if (e != cudaSuccess) return bcuda(hb, e, "autotune");
        tun.tuned = 1;
        return NH_OK;
    }

    int set_state(int d, const void* eta, const void* q1, const void* q2, const void* w,
                  const void* p, double t, int where) override
    {
        if (d < 0 || d >= n) return bfail(hb, NH_EINVAL, "domain index out of range");
        if (!eta || !q1) return bfail(hb, NH_EINVAL, "eta and q1 are required");
        const cudaMemcpyKind k = where == NH_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
        const Dom<T>& D = doms[d];
        const size_t nc = (size_t)D.P.nx * D.P.ny, nn = (size_t)(D.P.nx + 1) * (D.P.ny + 1);
        cudaStream_t s = hb->s;
        cudaMemcpyAsync(B.eta + D.coff, eta, nc * sizeof(T), k, s);
        cudaMemcpyAsync(B.q1 + D.coff, q1, nc * sizeof(T), k, s);
        if (q2) cudaMemcpyAsync(B.q2 + D.coff, q2, nc * sizeof(T), k, s);
        else cudaMemsetAsync(B.q2 + D.coff, 0, nc * sizeof(T), s);
        if (w) cudaMemcpyAsync(B.w + D.noff, w, nn * sizeof(T), k, s);
        else cudaMemsetAsync(B.w + D.noff, 0, nn * sizeof(T), s);
        if (p) cudaMemcpyAsync(B.p + D.noff, p, nn * sizeof(T), k, s);
        else cudaMemsetAsync(B.p + D.noff, 0, nn * sizeof(T), s);
        DomState z;
        std::memset(&z, 0, sizeof(z));
        z.t = t;
        cudaMemcpyAsync(d_ds + d, &z, sizeof(DomState), cudaMemcpyHostToDevice, s);
        cudaError_t e = cudaStreamSynchronize(s);
        if (e == cudaSuccess) e = cudaGetLastError();
        if (e != cudaSuccess) return bcuda(hb, e, "nh_batch_set_state");
        need_lambda = true;
        return NH_OK;
    }

    int get_state(int d, void* eta, void* q1, void* q2, void* w, void* p, double* t,
                  int where) override
    {
        if (d < 0 || d >= n) return bfail(hb, NH_EINVAL, "domain index out of range");
        const cudaMemcpyKind k = where == NH_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
        const Dom<T>& D = doms[d];
        const size_t nc = (size_t)D.P.nx * D.P.ny, nn = (size_t)(D.P.nx + 1) * (D.P.ny + 1);
        cudaStream_t s = hb->s;
        if (eta) cudaMemcpyAsync(eta, B.eta + D.coff, nc * sizeof(T), k, s);
        if (q1) cudaMemcpyAsync(q1, B.q1 + D.coff, nc * sizeof(T), k, s);
        if (q2) cudaMemcpyAsync(q2, B.q2 + D.coff, nc * sizeof(T), k, s);
        if (w) cudaMemcpyAsync(w, B.w + D.noff, nn * sizeof(T), k, s);
        if (p) cudaMemcpyAsync(p, B.p + D.noff, nn * sizeof(T), k, s);
        cudaMemcpyAsync(h_ds + d, d_ds + d, sizeof(DomState), cudaMemcpyDeviceToHost, s);
        cudaError_t e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return bcuda(hb, e, "nh_batch_get_state");
        if (t) *t = h_ds[d].t;
        return NH_OK;
    }

    int run(int nsteps) override
    {
        if (nsteps < 0) return bfail(hb, NH_EINVAL, "nsteps must be >= 0");
        int rc;
        if (need_lambda) {
            if ((rc = launch_lambda()) != NH_OK) return bcuda(hb, cudaGetLastError(), "lambda");
            need_lambda = false;
        }
        if ((hb->flags & NH_BATCH_AUTOTUNE) && !tuned_once) {
            if ((rc = autotune()) != NH_OK) return rc;
            tuned_once = true;
            if (exec) { cudaGraphExecDestroy(exec); exec = nullptr; }
        }
        if (tun.graph && !exec && !graph_failed && !prof.on) {
            if (build_graph() != NH_OK) {
                graph_failed = true;   // keep the message; run eagerly
                tun.graph = 0;
            }
        }
        cudaMemcpyAsync(h_ds, d_ds, n * sizeof(DomState), cudaMemcpyDeviceToHost, hb->s);
        cudaError_t e = cudaStreamSynchronize(hb->s);
        if (e != cudaSuccess) return bcuda(hb, e, "nh_batch_run");
        std::vector<int> nonconv0(n);
        for (int d = 0; d < n; ++d) nonconv0[d] = h_ds[d].nonconv;
        for (int k = 0; k < nsteps; ++k) {
            if (exec && !prof.on) {
                if ((e = cudaGraphLaunch(exec, hb->s)) != cudaSuccess) return bcuda(hb, e, "cudaGraphLaunch");
            } else if ((rc = step_eager()) != NH_OK) {
                return rc;
            }
        }
        cudaMemcpyAsync(h_ds, d_ds, n * sizeof(DomState), cudaMemcpyDeviceToHost, hb->s);
        e = cudaStreamSynchronize(hb->s);
        if (e == cudaSuccess) e = cudaGetLastError();
        if (e != cudaSuccess) return bcuda(hb, e, "nh_batch_run");
        for (int d = 0; d < n; ++d)
            if (h_ds[d].nonfinite)
                return bfail(hb, NH_ENONFINITE, "non-finite value in domain " + std::to_string(d));
        for (int d = 0; d < n; ++d)
            if (h_ds[d].nonconv != nonconv0[d] &&
                (h_ds[d].last_status[0] >= 6 || h_ds[d].last_status[1] >= 6))
                return bfail(hb, NH_ETIMEOUT, "pressure solve of domain " + std::to_string(d) +
                                                  ": a Chebyshev pass gave up waiting for its "
                                                  "staged copies");
        for (int d = 0; d < n; ++d)
            if (h_ds[d].nonconv != nonconv0[d])
                return bfail(hb, NH_ENOCONV, "pressure solve of domain " + std::to_string(d) +
                                                 " stopped with status " +
                                                 std::to_string(h_ds[d].last_status[0] != 1
                                                                    ? h_ds[d].last_status[0]
                                                                    : h_ds[d].last_status[1]));
        return NH_OK;
    }

    int stats(int d, nh_stats_t* out) override
    {
        if (d < 0 || d >= n) return bfail(hb, NH_EINVAL, "domain index out of range");
        kb_mass<T><<<grid_of((const void*)kb_mass<T>, kThreads, 0, nw_cell, true), kThreads, 0, hb->s>>>(
            arena(), wl_cell, nw_cell, B.eta, B.H);
        cudaMemcpyAsync(h_ds, d_ds, n * sizeof(DomState), cudaMemcpyDeviceToHost, hb->s);
        cudaError_t e = cudaStreamSynchronize(hb->s);
        if (e == cudaSuccess) e = cudaGetLastError();
        if (e != cudaSuccess) return bcuda(hb, e, "nh_batch_stats");
        const DomState& s = h_ds[d];
        std::memset(out, 0, sizeof(*out));
        out->t = s.t;
        out->dt = s.dt;
        out->dt_next = s.dt;
        out->steps = s.steps;
        out->solver_iters = s.sweeps;
        out->last_iters[0] = s.last_sweeps[0];
        out->last_iters[1] = s.last_sweeps[1];
        out->last_resid[0] = s.last_resid[0];
        out->last_resid[1] = s.last_resid[1];
        out->mass = s.mass;
        out->nonfinite = s.nonfinite;
        out->fallbacks = s.fallbacks;
        out->fallback_iters = s.bicg_iters;
        out->cheb_form = -1;
        return NH_OK;
    }

    int profile_enable(int on) override
    {
        prof.reset();
        prof.on = on != 0;
        return NH_OK;
    }

    int profile_read(nh_profile_t* out) override
    {
        prof.flush();
        for (int k = 0; k < NH_K_COUNT; ++k) { out->launches[k] = prof.launches[k]; out->ms[k] = prof.ms[k]; }
        return NH_OK;
    }

    int get_tuning(nh_batch_tuning* out) override
    {
        *out = tun;
        return NH_OK;
    }

    int set_tuning(const nh_batch_tuning* in) override
    {
        if (in->hyp < 0 || in->hyp >= C::nh || in->assembly < 0 || in->assembly >= C::na ||
            in->cheb < 0 || in->cheb >= C::nc || in->persistent < 0 || in->persistent > 15)
            return bfail(hb, NH_EINVAL, "tuning: candidate index out of range");
        tun.hyp = in->hyp;
        tun.assembly = in->assembly;
        tun.cheb = in->cheb;
        tun.persistent = in->persistent;
        tun.graph = in->graph ? 1 : 0;
        tun.tuned = 0;
        tuned_once = true;   // a hand-picked choice is not re-tuned
        graph_failed = false;
        if (exec) { cudaGraphExecDestroy(exec); exec = nullptr; }
        return NH_OK;
    }
};

int check_batch(int n, const nh_grid* grids, const double* const* H, const nh_params* p,
                std::string& why)
{
    if (n < 1 || !grids || !H || !p) { why = "need n >= 1, grids, H and params"; return 0; }
    if (p->precision != NH_FP64 && p->precision != NH_FP32) { why = "precision must be FP64 or FP32"; return 0; }
    if (!(p->g > 0.0) || !(p->cfl > 0.0) || !(p->delta > 0.0) || p->hdry < 0.0 ||
        p->manning_n < 0.0 || !(p->tol > 0.0) || p->max_iter < 1 || p->eps_dp < 0.0) {
        why = "invalid physical or solver parameter";
        return 0;
    }
    if (p->nonhydrostatic && p->solver != NH_SOLVER_CHEBYSHEV) {
        why = "the batched form solves with NH_SOLVER_CHEBYSHEV only";
        return 0;
    }
    if (p->w_equation != NH_W_YAMAZAKI) {
        why = "the batched form runs the h w_t = p form only";
        return 0;
    }
    for (int k = 0; k < 4; ++k)
        if (p->relax_width[k] != 0.0) {
            why = "the batched form has no relaxation zones";
            return 0;
        }
    double total = 0.0;
    for (int d = 0; d < n; ++d) {
        const nh_grid& g = grids[d];
        if (!H[d]) { why = "H of domain " + std::to_string(d) + " is null"; return 0; }
        if (g.dim != 2 || g.nx < 2 || g.ny < 2 || !(g.dx > 0.0) || !(g.dy > 0.0)) {
            why = "domain " + std::to_string(d) + ": need dim 2, nx, ny >= 2, dx, dy > 0";
            return 0;
        }
        for (int k = 0; k < 4; ++k)
            if (g.bc[k] != NH_BC_WALL && g.bc[k] != NH_BC_OUTFLOW) { why = "bc must be WALL or OUTFLOW"; return 0; }
        total += (double)(g.nx + 1) * (g.ny + 1);
    }
    if (total > 1.5e9) { why = "ensemble too large"; return 0; }
    return 1;
}

}  // namespace

extern "C" {

int nh_create_batch(int n, const nh_grid* grids, const double* const* H, const nh_params* params,
                    void* stream, int flags, nh_batch** out)
{
    if (!out) return NH_EINVAL;
    *out = nullptr;
    std::string why;
    if (!check_batch(n, grids, H, params, why)) return NH_EINVAL;
    nh_batch* b = new nh_batch();
    b->n = n;
    b->grids.assign(grids, grids + n);
    b->prm = *params;
    b->flags = flags;
    b->s = (cudaStream_t)stream;
    cudaError_t e = cudaSuccess;
    if (!b->s) {
        e = cudaStreamCreateWithFlags(&b->own, cudaStreamNonBlocking);
        b->s = b->own;
    }
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->side, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->side2, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->side3, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->ev_fork, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->ev_join, cudaEventDisableTiming);
    if (e != cudaSuccess) {
        cudaGetLastError();
        delete b;
        return NH_ECUDA;
    }
    int rc;
    if (params->precision == NH_FP32) {
        auto* im = new BatchImpl<float>();
        im->hb = b; im->n = n;
        b->impl.reset(im);
        rc = im->init(H);
    } else {
        auto* im = new BatchImpl<double>();
        im->hb = b; im->n = n;
        b->impl.reset(im);
        rc = im->init(H);
    }
    if (rc != NH_OK) {
        nh_batch_destroy(b);
        return rc;
    }
    *out = b;
    return NH_OK;
}

int nh_batch_set_state(nh_batch* b, int d, const void* eta, const void* q1, const void* q2,
                       const void* w, const void* p, double t, int where)
{
    if (!b) return NH_EINVAL;
    return b->impl->set_state(d, eta, q1, q2, w, p, t, where);
}

int nh_batch_get_state(nh_batch* b, int d, void* eta, void* q1, void* q2, void* w, void* p,
                       double* t, int where)
{
    if (!b) return NH_EINVAL;
    return b->impl->get_state(d, eta, q1, q2, w, p, t, where);
}

int nh_batch_run(nh_batch* b, int nsteps)
{
    if (!b) return NH_EINVAL;
    return b->impl->run(nsteps);
}

int nh_batch_stats(nh_batch* b, int d, nh_stats_t* out)
{
    if (!b || !out) return NH_EINVAL;
    return b->impl->stats(d, out);
}

int nh_batch_get_tuning(nh_batch* b, nh_batch_tuning* out)
{
    if (!b || !out) return NH_EINVAL;
    return b->impl->get_tuning(out);
}

int nh_batch_set_tuning(nh_batch* b, const nh_batch_tuning* in)
{
    if (!b || !in) return NH_EINVAL;
    return b->impl->set_tuning(in);
}

int nh_batch_candidate(int precision, int kind, int idx, int* tile_x, int* tile_y, int* threads)
{
    Shape s;
    if (precision == NH_FP32) {
        using C = Cands<float>;
        const int lim = kind == 0 ? C::nh : kind == 1 ? C::na : kind == 2 ? C::nc : 0;
        if (idx < 0 || idx >= lim) return NH_EINVAL;
        s = kind == 0 ? C::hyp_shape(idx) : kind == 1 ? C::asm_shape(idx) : C::cheb_shape(idx);
    } else if (precision == NH_FP64) {
        using C = Cands<double>;
        const int lim = kind == 0 ? C::nh : kind == 1 ? C::na : kind == 2 ? C::nc : 0;
        if (idx < 0 || idx >= lim) return NH_EINVAL;
        s = kind == 0 ? C::hyp_shape(idx) : kind == 1 ? C::asm_shape(idx) : C::cheb_shape(idx);
    } else {
        return NH_EINVAL;
    }
    if (tile_x) *tile_x = s.tx;
    if (tile_y) *tile_y = s.ty;
    if (threads) *threads = s.threads;
    return NH_OK;
}

int nh_batch_profile_enable(nh_batch* b, int on)
{
    if (!b) return NH_EINVAL;
    return b->impl->profile_enable(on);
}

int nh_batch_profile_read(nh_batch* b, nh_profile_t* out)
{
    if (!b || !out) return NH_EINVAL;
    return b->impl->profile_read(out);
}

const char* nh_batch_last_error(const nh_batch* b)
{
    return b ? b->err.c_str() : "null batch";
}

void nh_batch_destroy(nh_batch* b)
{
    if (!b) return;
    if (b->s) cudaStreamSynchronize(b->s);
    b->impl.reset();
    if (b->side) cudaStreamDestroy(b->side);
    if (b->side2) cudaStreamDestroy(b->side2);
    if (b->side3) cudaStreamDestroy(b->side3);
    if (b->ev_fork) cudaEventDestroy(b->ev_fork);
    if (b->ev_join) cudaEventDestroy(b->ev_join);
    if (b->own) cudaStreamDestroy(b->own);
    delete b;
}

}  // extern "C"
