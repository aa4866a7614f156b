// nh_internal.h -- declarations shared by the kernels (nh_kernels.cu) and the host
// runtime (nh_api.cu) of libnh.  Not part of the public C-ABI (include/nh.h).
#pragma once

#include <cuda_runtime.h>
#include <cstddef>

namespace nh {

// Grid and physical parameters as the kernels see them (T = float or double).
template <typename T>
struct Prm {
    int nx, ny;                 // cells
    int bcw, bce, bcs, bcn;     // 0 wall (mirror), 1 outflow (copy)
    T dx, dy;
    T g, delta, hdry, manning, B1;
    int breaking;
    int dry_zero;               // 1: q = 0 in dry cells at the end of each stage
};

// Device-side control block of one pressure solve (BiCGStab, FP64 scalars).
struct SolveCtl {
    double rho1;      // rhat . r of the current residual
    double rho;       // rho1 of the previous iteration
    double alpha, omega;
    double bb;        // ||b||^2
    double rr;        // ||r||^2
    double rv, ts, tt;
    int iter;         // iterations done in this solve
    int done;         // 1: stop (converged, cap reached or breakdown)
    int status;       // 0 running, 1 converged, 2 iteration cap, 3 breakdown, 4 Gershgorin
                      // bound >= 1, 5 stalled (batched form), 6 a register-form pass timed
                      // out waiting for its copies
    int max_iter;
    double tol2;      // tol^2
    unsigned counter; // last-block-done ticket
    unsigned pad;
    // Chebyshev-scheduled Jacobi
    double bdb;       // ||D^-1 b||^2
    double gersh;     // max Gershgorin radius of D^-1 M
    double sigma1, delta, rho_prev;
    double c1[8], c2[8];  // weights of the next pass's sweeps
    double dpmax;     // max |x_{k+1} - x_k| of the last sweep
    double eps_dp;    // > 0: stop when dpmax < eps_dp (criterion (32)); else residual test
    int sweeps;       // sweeps done in this solve
    int pad2;
    float c1f[8], c2f[8]; // FP32 copies of c1, c2 for FP32 sweeps
    // batched form: stall test of the Chebyshev passes and the BiCGStab fallback
    double best;      // smallest ||D^-1 r||^2 of the passes so far
    int stale;        // passes since best improved by the stall factor
    int fb;           // 1 while the domain's BiCGStab fallback runs
    // residual norm of the passes: each thread sums the squares of its nodes' scaled
    // residuals r * rsc (rsc = 2^-e with 2^e <= ||D^-1 b|| < 2^(e+1), an exact scaling that
    // keeps every square in range) into an FP64 accumulator; a block adds its threads'
    // sums in double-single (warps) and FP64 (across warps) arithmetic and multiplies by
    // rinv2 = 2^(2e) before its FP64 partial joins the grid sum
    double rscd;      // rsc (FP64 passes)
    double rinv2;     // 1 / rsc^2
    float rscf;       // rsc (FP32 passes)
    int pad3;
    double rfs;       // defect correction with FP32 inner solves: the power of two that
                      // scales the FP64 residual into the inner right-hand side
};

// Statistics of one stage's pressure solve in a captured step, read by the host after it.
struct SolveStat {
    double rr, bb, bdb;   // final squared residual and the two right-hand-side norms
    int sweeps;           // Chebyshev sweeps
    int iter;             // iteration count of the control block at the end
    int status;           // 1 converged, 2 cap, 3 breakdown, 6 / 7 wait ran out
    int fb;               // 1: BiCGStab continued the solve
    int passes;           // Chebyshev passes launched (pairs x 2)
    int bicg;             // BiCGStab iterations launched (pairs x 2)
};

// Device-side per-step scalars.
struct StepCtl {
    double lam;        // max over cells of the Eq. (23) rate, last final stage
    double mass;       // sum of h (cells), when requested
    int nonfinite;     // set when a non-finite value was written
    int clamped;       // depth clamps in the last step
    unsigned counter;  // last-block-done ticket
    unsigned pad;
};

// Device buffers of a 2D (or batched 1D) problem.
template <typename T>
struct Bufs {
    T *H;
    T *eta, *q1, *q2;            // state U^n
    T *eta1, *q11, *q21;         // stage-1 result
    T *etas, *q1s, *q2s;         // U* after the hyperbolic step (+ combination)
    T *q1k, *q2k;                // U* after the breaking terms (aliases q1s/q2s if off)
    T *w, *p, *w1, *ws;          // node fields
    T *dp, *palt;                // 2D: pressure correction of a solve; next pressure buffer
    T *cC, *cW, *cE, *cS, *cN;   // 2D five-point coefficients (1D: a = cW, b = cC, c = cE)
    T *rhs;
    T *r, *rh, *ph[2], *v[2], *t;  // BiCGStab vectors; the Chebyshev passes alternate
                                   // (dp, r) and (v[0], v[1]) as (x, x_{k-1})
    double *partials;             // per-block partial sums (>= 4 * nblk)
    SolveCtl *sctl;
    StepCtl *stctl;
    // w equation (hw)_t + div(hw u) = p only (else null): face mass fluxes of the stage's
    // hyperbolic step (x faces [ny][nx+1], y faces [ny+1][nx]; 1D: [rows][nx+1] in fmx)
    // and the transported w*
    T *fmx, *fmy, *wt;
    // relaxation zones only (else null): target eta*, q1*, q2* (cells), w*, p* (nodes)
    T *rz_eta, *rz_q1, *rz_q2, *rz_w, *rz_p;
};

struct Launch {
    int nblk;          // persistent-style grid size (multiple of the SM count)
    int nthr;          // threads per block
    cudaStream_t s;
};

// ---- 2D ----
// (the 2D correction writes p0 + dp into B.palt; the caller then swaps B.p and B.palt)
// fmx / fmy (or null): the mass flux of every x / y face, F_h(U^-) + D^-_h from its
// west / south cell ([ny][nx+1] and [ny+1][nx])
template <typename T>
void launch_hyp2d(const Prm<T>& P, const Launch& L, const T* eta, const T* q1, const T* q2,
                  const T* etab, const T* q1b, const T* q2b, const T* H, T a, T b, T dt,
                  T* eo, T* q1o, T* q2o, StepCtl* st, T* fmx = nullptr, T* fmy = nullptr,
                  const double* dtd = nullptr);
// dtd (captured steps): when not null, the kernels take dt (and de = b dt) from this device
// scalar instead of their argument
// w* of the w equation (hw)_t + div(hw u) = p at every node: hw moved on the node (dual)
// cells with the face mass fluxes fmx / fmy of the stage's hyperbolic step (input state
// etain, win), combined with the base state (etab, wb) as (hw)* = a h_b w_b + b (hw)**,
// divided by the node depth of the combined state etas.
template <typename T>
void launch_wtrans2d(const Prm<T>& P, const Launch& L, const T* etab, const T* etain,
                     const T* etas, const T* H, const T* wb, const T* win, const T* fmx,
                     const T* fmy, T a, T b, T dt, T* wo, const double* dtd = nullptr);
template <typename T>
void launch_asm2d(const Prm<T>& P, const Launch& L, const Bufs<T>& B, const T* w_in,
                  const T* w_base, T a, T b, T de, int with_coef, int resid_form, double tol2,
                  int max_iter, int kpass, double* partials, SolveCtl* ctl, int fuse_break = 0,
                  const double* dtd = nullptr, T deb = T(0));
// fuse_break (with breaking on): the breaking terms are computed inside the assembly from
// B.q1s / B.q2s, and q** is written to B.q1k / B.q2k (no separate breaking launch)
// Chebyshev-scheduled Jacobi: sweeps per launch, number of tiles (blocks), one launch.
template <typename T>
int cheb_sweeps_per_pass();
template <typename T>
size_t cheb_tiles(const Prm<T>& P);
template <typename T>
size_t asm_tiles(const Prm<T>& P);   // blocks of the 2D assembly (3 partials each)
// One pass: (x, x_{k-1}) from (xi, xpi) to (xo, xpo) in kernel form `variant` (0 ..
// cheb_pass_forms() - 1, listed at the definition; the cyclic forms after them read xi and
// write xo only).  The register forms wait at most
// `polls` polls for each region's staged copies; stall_block >= 0 makes that block's first
// wait run out with no copy issued (a test hook; -1 in normal use).
template <typename T>
int launch_cheb_pass(const Prm<T>& P, cudaStream_t s, const Bufs<T>& B, const T* xi,
                     const T* xpi, T* xo, T* xpo, double* partials, int variant,
                     unsigned polls, int stall_block);
constexpr unsigned kDefaultWaitPolls = 1u << 22;   // nh_params.wait_polls <= 0
template <typename T>
int cheb_pass_forms();   // number of Jacobi pass forms (variants 0 .. n-1)
template <typename T>
int cheb_cyclic_forms();   // number of cyclic forms (variants n .. n + this - 1)
template <typename T>
void launch_matvec2d(const Prm<T>& P, const Launch& L, const Bufs<T>& B, const T* x, T* y);
template <typename T>
void launch_bicg_init(const Prm<T>& P, const Launch& L, const Bufs<T>& B, double* partials,
                      int only_fb = 0);   // only_fb: nothing unless B.sctl->fb is set
// one BiCGStab phase: 0 = A (p^, v), 1 = B (t), 2 = C (x, r); parity selects p^ / v buffers
template <typename T>
void launch_bicg_phase(const Prm<T>& P, const Launch& L, const Bufs<T>& B, int parity, int phase,
                       double* partials);
template <typename T>
void launch_corr2d(const Prm<T>& P, const Launch& L, const Bufs<T>& B, const T* q1k,
                   const T* q2k, T de, int with_p, T* eo, T* q1o, T* q2o, T* wo, int final_stage,
                   double* partials, StepCtl* st, const double* dtd = nullptr, T deb = T(0),
                   const T* dp_alt = nullptr);
// dp_alt (captured steps): the other buffer of the pass pair; the correction takes the
// iterate from it when the Chebyshev solve ended on an odd pass without a fallback

// ---- FP64 solves by defect correction with FP32 inner solves (FP64 handles) ----
// r = b - M x in FP64 into r64, its Jacobi-scaled square norm into ctl64->rr, the scale
// rfs = 2^-e (2^e ~ the rms of D^-1 r) into ctl64, and the inner solve's control block
// ctl32 prepared as an assembly would (norms of the scaled residual, the interval of
// ctl64->gersh, tolerance tol2_in, kpass sweeps per pass)
void launch_refine_resid(const Prm<double>& P, const Launch& L, const Bufs<double>& B,
                         const double* x, double* r64, double* partials, SolveCtl* ctl64,
                         SolveCtl* ctl32, double tol2_in, int max_iter_in, int kpass);
// r32 = (float)(r64 rfs)
void launch_refine_scale(const Launch& L, const double* r64, float* r32, size_t n,
                         const SolveCtl* ctl64);
// x += (double)d32 / rfs
void launch_refine_add(const Launch& L, double* x, const float* d32, size_t n,
                       const SolveCtl* ctl64);

// ---- captured steps: device-side control of the solver loops ----
// condition of a WHILE node: continue while the solve is not done and *cnt < cap (count =
// 1: count this evaluation, after a body; 0: before the first body)
void launch_loop_cond(cudaStream_t s, cudaGraphConditionalHandle h, const SolveCtl* ctl,
                      unsigned* cnt, unsigned cap, int count);
// after the passes: flag a BiCGStab fallback (status 4 or 5: not diagonally dominant, or
// stalled), and move the passes' iterate to dp when they ended on an odd pass
void launch_fb_begin(cudaStream_t s, SolveCtl* ctl);
template <typename T>
void launch_settle_fb(const Launch& L, const SolveCtl* ctl, const T* x2, T* dp, size_t n, int K);
// copy the stage's solve statistics (cnt: [pass pairs, BiCGStab pairs])
void launch_solve_stats(cudaStream_t s, const SolveCtl* ctl, const unsigned* cnt, SolveStat* out);

// ---- adjoint of the 2D step (nh_adjoint.cu) ----
template <typename T>
void launch_adj_pbar(const Prm<T>& P, const Launch& L, const T* eta, const T* H, const T* a1o,
                     const T* a2o, const T* wo, T de, T* pbar);
// rows of M^T into tW..tN (coefficients of B), reductions of b, solve set-up in B.sctl
template <typename T>
void launch_transpose(const Prm<T>& P, const Launch& L, const Bufs<T>& B, const T* b, T* tW,
                      T* tE, T* tS, T* tN, double tol2, int max_iter, int kpass);
template <typename T>
void launch_adj_node(const Prm<T>& P, const Launch& L, const T* eta, const T* H, const T* q1,
                     const T* q2, const T* ws, const T* p, const T* lam, const T* wo,
                     double scale, double de, double a, double b, int assign_in, T* Hh, T* Sb,
                     T* A1, T* A2, T* w_in_bar, T* w_base_bar);
template <typename T>
void launch_adj_cell_corr(const Prm<T>& P, const Launch& L, const T* eta, const T* H,
                          const T* p, const T* eo_bar, const T* a1o, const T* a2o, T de, T* Es,
                          T* Hh, T* Sb, T* A1, T* A2);
template <typename T>
void launch_adj_combine(const Launch& L, long long n, T* Es, const T* Hh, const T* Sb, T* Hbar);
template <typename T>
void launch_adj_face(const Prm<T>& P, const Launch& L, const T* eta, const T* q1, const T* q2,
                     const T* H, const T* Es, const T* A1, const T* A2, T bfac, T dt,
                     int frozen, T* Gh, T* Ge, T* Gu, T* Gv);
template <typename T>
void launch_adj_cell_hyp(const Prm<T>& P, const Launch& L, const T* eta, const T* q1,
                         const T* q2, const T* H, const T* Es, const T* A1, const T* A2,
                         const T* Gh, const T* Ge, const T* Gu, const T* Gv, T a, T b,
                         int assign_in, T* ein_b, T* a1in_b, T* a2in_b, T* eb_b, T* a1b_b,
                         T* a2b_b, T* Hbar);

// ---- batched 1D ----
template <typename T>
void launch_hyp1d(const Prm<T>& P, const Launch& L, const T* eta, const T* q, const T* etab,
                  const T* qb, const T* H, T a, T b, T dt, T* eo, T* qo, StepCtl* st,
                  T* fm = nullptr);
// 1D form of launch_wtrans2d (fm: [rows][nx+1] face mass fluxes)
template <typename T>
void launch_wtrans1d(const Prm<T>& P, const Launch& L, const T* etab, const T* etain,
                     const T* etas, const T* H, const T* wb, const T* win, const T* fm, T a,
                     T b, T dt, T* wo);
template <typename T>
void launch_break1d(const Prm<T>& P, const Launch& L, const T* eta, const T* q, const T* H,
                    T de, T* qo);
template <typename T>
void launch_asm1d(const Prm<T>& P, const Launch& L, const Bufs<T>& B, const T* q_pre,
                  const T* qk, const T* w_in, const T* w_base, T a, T b, T de);
template <typename T>
int launch_tridiag1d(const Prm<T>& P, cudaStream_t s, const Bufs<T>& B, T* x);
// Batched tridiagonal solve of `rows` systems of size n (row-major): PCR in shared memory
// when n <= pcr_max_n, else the Thomas algorithm with scratch cp, dp (n * rows each).
// Returns 0, -1 on a launch-attribute error, -2 when scratch is needed but missing.
template <typename T>
int launch_tridiag_raw(int n, int rows, const T* a, const T* b, const T* c, const T* d, T* x,
                       T* cp, T* dp, cudaStream_t s);
template <typename T>
void launch_tridiag_apply1d(const Prm<T>& P, const Launch& L, const Bufs<T>& B, const T* x,
                            T* y);
template <typename T>
void launch_corr1d(const Prm<T>& P, const Launch& L, const Bufs<T>& B, const T* qk, T de,
                   int with_p, T* eo, T* qo, T* wo, int final_stage, double* partials,
                   StepCtl* st);

// ---- relaxation zones (Sec. 4.4) ----
// Per side (west, east, south, north): zone width L, k = the first natural number with
// k d >= L (0: no zone), and the cell sizes d = (dx, dy) in FP64.
struct RelaxZ {
    double L[4];
    int k[4];
    double d[2];
};
// Blend the zone cells (eta, q1, q2) and nodes (w, p) toward the target (et .. pt) after
// a step; dim 1: rows of 1D channels (west / east zones only).
template <typename T>
void launch_relax(const Prm<T>& P, const Launch& L, const RelaxZ& Z, int dim, T* eta, T* q1,
                  T* q2, T* w, T* p, const T* H, const T* et, const T* q1t, const T* q2t,
                  const T* wt, const T* pt);

// ---- shared ----
template <typename T>
void launch_mass(const Prm<T>& P, const Launch& L, const T* eta, const T* H, double* partials,
                 StepCtl* st);
template <typename T>
void launch_lambda(const Prm<T>& P, const Launch& L, const T* eta, const T* q1, const T* q2,
                   const T* H, int dim, double* partials, StepCtl* st);
template <typename T>
void launch_fill(const Launch& L, T* x, size_t n, T v);
template <typename T>
void launch_nonfinite(const Launch& L, const T* x, size_t n, StepCtl* st);   // flags NaN / inf
template <typename T>
void launch_gather(cudaStream_t s, const T* x, const int* idx, int n, T* out);   // out = x[idx]
template <typename T>
void launch_convert_from_double(const Launch& L, const double* src, T* dst, size_t n);

int pcr_max_n(int elem_bytes);

}  // namespace nh
