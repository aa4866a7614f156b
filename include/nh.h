/*
 * nh.h -- C-ABI of libnh, a B300 (sm_103a) implementation of one time step of the
 * depth-integrated non-hydrostatic (Yamazaki) shallow-water system by the two-step
 * projection-correction scheme of Escalante, Morales de Luna & Castro (arXiv:1706.04551).
 *
 * The step (Sec. 4.3 in 1D, Sec. 5 / App. A in 2D, Sec. 6 "steps 1-4 twice"):
 *   for each stage of a second-order TVD Runge-Kutta method (Shu-Osher form),
 *     hyperbolic PVM-HLL finite-volume update with MUSCL-minmod reconstruction,
 *       emerging-bottom treatment and velocity desingularisation (Eqs. 18-23, 30;
 *       Sec. 4.5), semi-implicit Manning friction, optional breaking terms (Eq. 12);
 *     assembly of the compact finite-difference pressure system (App. B Eq. 43 in 1D,
 *       the five-point system of Eqs. 36-41 in 2D);
 *     pressure solve (1D: batched tridiagonal, parallel cyclic reduction; 2D: Jacobi
 *       with Chebyshev-scheduled relaxation, or Jacobi-preconditioned BiCGStab with FP64
 *       dot products);
 *     correction of the discharges and of w (Eqs. 26-28, 36, 41).
 * Options: the energy-consistent w equation (hw)_t + div(hw u) = p (nh_params.w_equation),
 * generating / absorbing relaxation zones of Sec. 4.4 (nh_params.relax_width,
 * nh_set_relax_target), periodic 1D channels (NH_BC_PERIODIC), the hydrostatic step alone
 * (nh_params.nonhydrostatic = 0) and the stopping criterion of Eq. (32) (nh_params.eps_dp).
 *
 * Conventions.
 *   - Cells: row-major [ny][nx], x fastest; cell (i, j) is centred at ((i+1/2)dx, (j+1/2)dy).
 *   - Nodes (p, w): row-major [ny+1][nx+1]; node (I, J) sits at (I dx, J dy).
 *     In 1D (dim = 1) each of the ny rows is an independent channel of nx cells with
 *     nx + 1 nodes (a batch of 1D problems).
 *   - State: eta = h - H (free surface), q1, q2 (discharges), w, p.  H is the still-water
 *     depth, positive below the datum; a dry cell has eta = -H.
 *   - Arrays passed to nh_set_state / nh_get_state have the handle's precision: double
 *     for NH_FP64, float for NH_FP32.  H is always double.
 *   - where = NH_HOST: pointers are host memory (pinned or pageable); NH_DEVICE: device
 *     memory of the current device, laid out densely as above.
 * Ownership: the library allocates and owns every device buffer of a handle (freed by
 *   nh_destroy).  Input pointers are only read during the call.  All work is enqueued on
 *   the stream given to nh_create (0 = legacy default stream); calls that return results
 *   to the host synchronise that stream.
 * Errors: every function returns NH_OK (0) or a negative NH_E* code; the message of the
 *   last error of a handle is returned by nh_last_error.  Device-side failures (solver
 *   not converged, non-finite values) are reported as status codes, never by trapping.
 */
#ifndef NH_H
#define NH_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

#define NH_OK 0
#define NH_EINVAL (-1)      /* invalid argument                                      */
#define NH_ENOMEM (-2)      /* device allocation failed                              */
#define NH_ECUDA (-3)       /* CUDA runtime error                                    */
#define NH_ENOCONV (-4)     /* pressure solve did not reach tol within max_iter      */
#define NH_ENONFINITE (-5)  /* a non-finite value appeared in the state              */
#define NH_ETIMEOUT (-6)    /* a bounded device-side wait (a Chebyshev pass waiting for its
                               staged copies) ran out of polls; the solve was abandoned   */

enum { NH_BC_WALL = 0, NH_BC_OUTFLOW = 1, NH_BC_PERIODIC = 2 /* 1D only, west and east */ };
enum {
    NH_SOLVER_BICGSTAB = 0,  /* Jacobi-preconditioned BiCGStab, FP64 dots                     */
    NH_SOLVER_CHEBYSHEV = 1  /* Jacobi with Chebyshev-scheduled relaxation (Sec. 5's scheduled
                                relaxation Jacobi) on the Gershgorin interval of D^-1 M        */
};
enum { NH_FP64 = 0, NH_FP32 = 1 };
enum {
    NH_W_YAMAZAKI = 0,   /* h w_t = p (Eq. 7)                                             */
    NH_W_TRANSPORT = 1   /* (hw)_t + div(hw u) = p, the energy-consistent system of Sec. 2's
                            reference [7]: hw moved with the hyperbolic step's mass fluxes */
};
enum { NH_HOST = 0, NH_DEVICE = 1 };

typedef struct {
    int dim;            /* 1 or 2                                                        */
    int nx, ny;         /* cells (2D: nx, ny >= 2; 1D: ny = number of independent rows)  */
    double dx, dy;      /* cell sizes (dy unused in 1D)                                  */
    int bc[4];          /* west, east, south, north: NH_BC_WALL / NH_BC_OUTFLOW, or
                           NH_BC_PERIODIC on both west and east of a 1D channel         */
} nh_grid;

typedef struct {
    double g;           /* gravity                                                       */
    double cfl;         /* Courant number for the Eq. (23) time step                     */
    double delta;       /* desingularisation depth of Sec. 4.5 (1e-5)                    */
    double hdry;        /* dry threshold: a cell is dry when h <= hdry                   */
    double manning_n;   /* Gauckler-Manning coefficient (0: no friction)                 */
    double B1, B2;      /* breaking calibration coefficients, Eq. (9)                    */
    int breaking;       /* 1: breaking terms of Eq. (12)                                 */
    int nonhydrostatic; /* 1: full scheme; 0: hydrostatic shallow water only (p = 0)     */
    int solver;         /* 2D pressure solver, NH_SOLVER_CHEBYSHEV (default) or _BICGSTAB  */
    double tol;         /* stop when ||b - M p||_2 <= tol ||b||_2 (BiCGStab), or
                           ||D^-1 (b - M p)||_2 <= tol ||D^-1 b||_2 (Chebyshev; D = diag M)  */
    int max_iter;       /* iteration cap (BiCGStab iterations / Chebyshev sweeps)         */
    int precision;      /* NH_FP64 or NH_FP32 (state and fluxes; dots are FP64 always)   */
    double fixed_dt;    /* > 0: nh_run uses this step instead of Eq. (23)                */
    double eps_dp;      /* > 0: stop a pressure solve on ||p^(k+1) - p^(k)||_inf < eps_dp,
                           the criterion of Eq. (32), instead of the residual test (the
                           Chebyshev sweeps, and BiCGStab -- chosen, or as the fallback --
                           on the change of its iterate per iteration)                   */
    int adjoint_frozen_limiter; /* nh_adjoint_step: 0 = exact derivative of the step; 1 =
                           reconstruction linearised with the limiter ratio held fixed   */
    int cheb_form;      /* single-domain handles, Chebyshev solver: -1 (default) = the
                           kernel form of the pass is chosen by timing the first passes
                           (among the cyclic forms when cheb_cyclic applies, else among the
                           Jacobi forms); 0 .. nh_cheb_forms(precision) - 1 = that Jacobi
                           form; nh_cheb_forms(precision) + k = cyclic form k (k <
                           nh_cheb_cyclic_forms(precision)).  The Jacobi forms give the
                           same iterates, and so do the cyclic forms.                    */
    int w_equation;     /* NH_W_YAMAZAKI (default) or NH_W_TRANSPORT.  With NH_W_TRANSPORT
                           hw lives on the node (dual) cells: each stage moves it with the
                           mean of the surrounding cells' face mass fluxes, upwind in w,
                           and the Runge-Kutta combination acts on hw.  Single-domain
                           handles only; batches and nh_step_taped reject it.            */
    double relax_width[4]; /* L_Rel of the generating / absorbing relaxation zone of Sec.
                           4.4 on the west, east, south, north side (0: none; 1D: west and
                           east only; not on periodic sides; at most the domain's length).
                           After every step, the k + 1 cells nearest the side (k the first
                           natural number with k dx >= L_Rel) blend toward a target as
                           U <- m U + (1 - m) U*, m = sqrt(max(0, 1 - (d / L_Rel)^2)), d the
                           distance from the zone's inner cell (m = 0 at the boundary
                           cell); w, p at the nodes with the mean m of the two cells.  In
                           2D m is the product of the x and y factors.  The
                           target is the lake at rest (absorbing) until
                           nh_set_relax_target sets another.  Single-domain handles only. */
    int dry_zero;       /* 1 (default): q = 0 in dry cells (h <= hdry) at the end of each
                           stage, i.e. the premise of App. B A.2 (q = w = 0 where the depth
                           vanishes) imposed; 0: the second step exactly as Sec. 4.5 states
                           it, with no special treatment and no truncation at wet/dry
                           fronts (the correction's p (2 eta - h)_x term then gives dry
                           cells next to the shoreline a small discharge).  nh_step_taped
                           and nh_adjoint_step require 1.                                */
    int wait_polls;     /* polls of each bounded wait of the register-form Chebyshev pass
                           for its staged copies (<= 0: the default, 2^22).  A wait that
                           runs out ends the solve with NH_ETIMEOUT; the pass issues no
                           further copies and drains those in flight (bounded) first.   */
    int capture;        /* 1 (default): 2D steps (Chebyshev solver once its pass form is
                           known, or the hydrostatic step) run as one CUDA graph per step,
                           the solver loops as conditional WHILE nodes on the device, the
                           host waiting once per step; 0: every kernel launched eagerly and
                           the solve polled from the host.  Results are the same bits.    */
    int refine_fp32;    /* FP64 2D Chebyshev handles (residual test, eps_dp = 0): 1 = solve
                           each pressure system by defect correction, FP32 inner solves of
                           M d = r (r = b - M x in FP64, scaled by an exact power of two) to
                           a relative 1e-4 by the same scheduled relaxation, x += d in
                           FP64, until the FP64 scaled residual meets tol; the sweeps run
                           at the FP32 rate.  0 (default): FP64 sweeps.  Such handles step
                           eagerly (capture does not apply).                              */
    int fallback_block_nodes; /* batches: a domain of at most this many nodes whose rows
                           fail the Gershgorin test at assembly runs its whole BiCGStab
                           solve in one thread block, beside the Chebyshev passes of the
                           other domains (default 70000); 0: every fallback solve uses the
                           grid-wide BiCGStab after the passes.  Single-domain handles
                           ignore it.                                                     */
    int cheb_cyclic;    /* single-domain 2D handles, Chebyshev solver, cheb_form = -1 and
                           eps_dp = 0: the cyclic form of the pass.  The five-point rows
                           couple each node with nodes of the other colour (I + J) mod 2
                           only, and the Chebyshev interval is centred at 1, so the nodes of
                           one colour at the odd steps and of the other at the even steps
                           form a closed recurrence (Golub and Varga's cyclic Chebyshev
                           method): each step updates one colour in place, half the work of
                           a Jacobi sweep, and every node takes the values of the full
                           iteration at the steps of its colour.  Its stopping test measures
                           a vector whose colours lie one step apart, which takes more steps
                           than the Jacobi forms' sweeps (58 against 53 per stage on the
                           4096^2 island, 36 against 32 on the 1024^2 shoals), and is still
                           faster on every grid measured.  1 (default) = the cyclic form;
                           0 = the Jacobi forms (cheb_form).  Its kernel forms
                           (nh_cheb_cyclic_forms) are chosen by timing.  last_iters and
                           solver_iters count its steps.  The FP32 inner solves of
                           refine_fp32 use it too.  Batches ignore it.                   */
} nh_params;

typedef struct {
    double t;              /* simulated time                                             */
    double dt;             /* last step taken                                            */
    double dt_next;        /* Eq. (23) step of the current state                         */
    long long steps;       /* steps taken since creation / nh_set_state                  */
    long long solver_iters;/* total pressure-solver iterations                           */
    int last_iters[2];     /* iterations of the two stages of the last step              */
    double last_resid[2];  /* relative residuals of those solves                         */
    double mass;           /* sum of h dx dy over all cells (FP64)                        */
    int nonfinite;         /* 1 if a non-finite value was detected                       */
    int fallbacks;         /* Chebyshev solves finished by BiCGStab (stalled, or a system
                              that is not diagonally dominant)                           */
    long long fallback_iters; /* BiCGStab iterations of those (part of solver_iters)     */
    int cheb_form;         /* kernel form of the Chebyshev pass in use (nh_params.cheb_form,
                              or the one chosen by timing; nh_cheb_forms(precision) + k for
                              cyclic form k, nh_params.cheb_cyclic); -1 while the forms are
                              timed, or for a batch / a handle that does not run the
                              Chebyshev solver                                            */
} nh_stats_t;

typedef struct nh_handle nh_handle;

/* Fill p with the paper's defaults: g = 9.81, CFL 0.9, delta = 1e-5, hdry = delta,
 * n = 0, B1 = 0.15, B2 = 0.5 (Sec. 7.4), breaking off, non-hydrostatic on, Chebyshev
 * solver, tol 1e-12, max_iter 2000, FP64, fixed_dt 0, eps_dp 0, exact adjoint, pass
 * form chosen by timing (cheb_form = -1), w equation h w_t = p (NH_W_YAMAZAKI), q = 0 in
 * dry cells (dry_zero = 1), default wait limit (wait_polls = 0), captured steps (capture = 1),
 * defect correction off (refine_fp32 = 0), batched block fallback up to 70000 nodes, cyclic
 * form of the pass (cheb_cyclic = 1). */
int nh_default_params(nh_params *p);

/* Number of kernel forms of the Chebyshev-scheduled Jacobi pass (Sec. 5's scheduled
 * relaxation; nh_params.cheb_form) for precision NH_FP32 or NH_FP64; NH_EINVAL otherwise.
 * No GPU work. */
int nh_cheb_forms(int precision);

/* Number of kernel forms of the cyclic pass (nh_params.cheb_cyclic; the handle times them
 * against each other and reports the one in use as nh_stats_t.cheb_form =
 * nh_cheb_forms(precision) + k) for NH_FP32 or NH_FP64; NH_EINVAL otherwise.  No GPU work. */
int nh_cheb_cyclic_forms(int precision);

/* Create a simulation on the current CUDA device.  H: host array [ny][nx] (double) of
 * still-water depths.  stream: a cudaStream_t (or 0).  The state is lake at rest
 * (eta = max(0, H) - H, q = w = p = 0) until nh_set_state.  Returns NH_EINVAL for bad
 * sizes / parameters, NH_ENOMEM when allocation fails. */
int nh_create(const nh_grid *grid, const double *H, const nh_params *params, void *stream,
              nh_handle **out);

/* Set the state.  eta, q1, q2: [ny][nx]; w, p: [ny+1][nx+1] (may be NULL: set to 0);
 * q2 may be NULL in 1D.  t: simulation time of the state.  Recomputes the Eq. (23)
 * step of the new state.  NH_ENONFINITE when a value of the input is NaN or infinite
 * (checked on the device; the state is then undefined until a successful call). */
int nh_set_state(nh_handle *h, const void *eta, const void *q1, const void *q2,
                 const void *w, const void *p, double t, int where);

/* Copy the state out (any pointer may be NULL to skip it); t may be NULL. */
int nh_get_state(nh_handle *h, void *eta, void *q1, void *q2, void *w, void *p, double *t,
                 int where);

/* Gauges: eta at n cells (row-major indices j nx + i, cells[k] in [0, nx ny)) into out[k],
 * as the time series at wave gauges that the paper's experiments record (Sec. 7).  cells
 * and out are device memory of the current device (out in the handle's precision); the
 * gather is one kernel enqueued on the handle's stream, so a series can be recorded every
 * step without a host round trip.  n = 0 does nothing.  NH_EINVAL for null pointers or
 * n < 0; indices out of range are not checked on the device (the caller validates them). */
int nh_gauges(nh_handle *h, const int *cells, int n, void *out);

/* Advance one time step.  dt > 0: use it; dt <= 0: the Eq. (23) step of the current
 * state (or params.fixed_dt when that is > 0).  *dt_taken (may be NULL) receives it.
 * Returns NH_ENOCONV when a pressure solve stopped at max_iter or broke down (the step is
 * still taken, with that solve's last iterate), NH_ENONFINITE when the new state holds a
 * NaN or infinity, NH_ETIMEOUT when a bounded device-side wait ran out (nh_params.
 * wait_polls); after NH_ENONFINITE or NH_ETIMEOUT the state is undefined until the next
 * nh_set_state. */
int nh_step(nh_handle *h, double dt, double *dt_taken);

/* Advance until t >= t_end (last step shortened to land on t_end; t_end <= 0: no time
 * limit) or max_steps steps.  *steps_taken may be NULL. */
int nh_run(nh_handle *h, double t_end, long long max_steps, long long *steps_taken);

/* Target (eta*, q1*, q2*, w*, p*) of the relaxation zones (Sec. 4.4), used from the next
 * step on: cell arrays [ny][nx], node arrays as in nh_set_state, handle precision; only
 * the zone entries are read.  A NULL pointer leaves that field's target as it is (the
 * lake at rest: eta* = max(H, 0) - H, q* = w* = p* = 0, until set).  A target depth
 * eta* + H below 0 counts as 0.  NH_EINVAL when the handle has no zone.  For a generating
 * boundary, set the target of time t + dt before each step. */
int nh_set_relax_target(nh_handle *h, const void *eta, const void *q1, const void *q2,
                        const void *w, const void *p, int where);

/* Counters and the FP64 mass of the current state (synchronises the stream). */
int nh_stats(nh_handle *h, nh_stats_t *out);

/* Message of the last error on this handle ("" if none); valid until the next call. */
const char *nh_last_error(const nh_handle *h);

void nh_destroy(nh_handle *h);

/* ---- per-kernel timing (CUDA events around every launch, on the handle's stream) ---- */

enum {
    NH_K_HYPERBOLIC = 0,  /* PVM-HLL update + friction + clamp + RK combination        */
    NH_K_BREAKING,        /* breaking terms at cells                                    */
    NH_K_ASSEMBLY,        /* w*, pressure-system rows and right-hand side               */
    NH_K_SOLVE_INIT,      /* BiCGStab initial residual                                  */
    NH_K_BICG_A,          /* BiCGStab: p^ update and v = M D^-1 p^                       */
    NH_K_BICG_B,          /* BiCGStab: t = M D^-1 s                                      */
    NH_K_BICG_C,          /* BiCGStab: x, r updates and convergence test                */
    NH_K_CHEB_PASS,       /* Chebyshev-scheduled Jacobi: K sweeps per launch             */
    NH_K_TRIDIAG,         /* 1D batched tridiagonal solve                               */
    NH_K_CORRECTION,      /* correction of q and w, Eq. (23) rate                        */
    NH_K_ADJ_HYPERBOLIC,  /* adjoint: hyperbolic step (faces, cells)                     */
    NH_K_ADJ_ASSEMBLY,    /* adjoint: transposed rows, assembly / solve terms            */
    NH_K_ADJ_CORRECTION,  /* adjoint: correction terms                                   */
    NH_K_W_TRANSPORT,     /* w* of the (hw)_t + div(hw u) = p form (NH_W_TRANSPORT)      */
    NH_K_RELAX,           /* relaxation zones (Sec. 4.4) and the Eq. (23) rate after them */
    NH_K_BICG_BLOCK,      /* batches: whole BiCGStab solves of small domains, a block each */
    NH_K_COUNT
};

typedef struct {
    long long launches[NH_K_COUNT];
    double ms[NH_K_COUNT];          /* summed device time per kernel class              */
} nh_profile_t;

/* on != 0: start recording an event pair around every kernel launch (counters reset);
 * on == 0: stop.  Recording adds host work per launch; device times are unaffected. */
int nh_profile_enable(nh_handle *h, int on);

/* Accumulated times since nh_profile_enable (synchronises the stream). */
int nh_profile_read(nh_handle *h, nh_profile_t *out);

/* ---- batched tridiagonal solve (the 1D pressure systems, App. B Eqs. 42-43) ---- */

/* Solve `rows` independent systems a[i] x[i-1] + b[i] x[i] + c[i] x[i+1] = d[i],
 * i = 0 .. n-1 (a[0] and c[n-1] are ignored), stored row-major (system r at offset r n).
 * All pointers are device memory of the current device in the given precision
 * (NH_FP64: double, NH_FP32: float); x may not alias the inputs.  Systems must be
 * diagonally dominant (no pivoting), as those of Eq. (43) are.  Systems of n <= 4096
 * (FP64) / 8192 (FP32) are solved by parallel cyclic reduction in shared memory; longer
 * ones by the Thomas algorithm (Sec. 4.3), for which the call allocates 2 n rows
 * elements of scratch with cudaMallocAsync on `stream` and frees them on return.
 * Enqueued on `stream` (asynchronous).  Returns NH_OK, NH_EINVAL, NH_ENOMEM or NH_ECUDA. */
int nh_tridiag_batched(int n, int rows, int precision, const void *a, const void *b,
                       const void *c, const void *d, void *x, void *stream);

/* Size of the fixed device scratch of nh_tridiag_batched_noalloc (8 MiB). */
#define NH_NOALLOC_SCRATCH_BYTES (8u << 20)

/* The same solve as nh_tridiag_batched for callers that cannot allocate device memory
 * during the call -- for example code running inside another framework's memory pool,
 * callbacks or real-time loops where cudaMalloc's latency and implicit synchronisation
 * are not allowed, or processes with a fixed device-memory budget.  It calls no
 * cudaMalloc / cudaFree or other allocating routine.  Systems longer than the
 * shared-memory limit use a file-scope device array of NH_NOALLOC_SCRATCH_BYTES as
 * scratch; each GPU that loads the library holds that array until the process exits.
 * Limit: 2 n rows sizeof(element) <= NH_NOALLOC_SCRATCH_BYTES for those systems (n rows
 * <= 524288 in FP64, 1048576 in FP32); larger sizes return NH_EINVAL and do nothing.
 * The first call on each device looks up the array's device address (with that device
 * current); make that first call before any stream capture.  All calls share the one
 * array: calls whose executions overlap on the GPU (for example on two streams at once)
 * race and give wrong results; serialise them.  No part of the scratch needs to start at
 * zero.  The looked-up address is kept for the life of the process: do not call this
 * entry point on a device after cudaDeviceReset (or any re-creation of its primary
 * context) in the same process, since the kept address would then be stale.  The paper
 * has no counterpart of this entry point.  Same arguments and return codes as
 * nh_tridiag_batched. */
int nh_tridiag_batched_noalloc(int n, int rows, int precision, const void *a, const void *b,
                               const void *c, const void *d, void *x, void *stream);

/* ---- adjoint (reverse-mode derivative) of nh_step ----
 *
 * The paper has no adjoint; these entry points differentiate the discrete 2D step that
 * nh_step takes (Sec. 5 / App. A: the Eq. (30) hyperbolic update with MUSCL-minmod and the
 * PVM-HLL fluctuations of Eqs. (18)-(19), the pressure system of Eqs. (36)-(41) solved
 * exactly (the adjoint solves the transposed system with the handle's solver and tol; a
 * Chebyshev solve that stops improving at the precision's rounding floor is accepted there),
 * and the correction), for a fixed dt.  Limits: 2D handles with the non-hydrostatic step
 * on, no friction (manning_n = 0) and no breaking; minmod, min / max and |.| are
 * differentiated along the branch the forward takes, and depth clamps are not
 * differentiated (states should stay wet).
 *
 * Use: nh_step_taped records what the reverse needs of one step into `tape` (device
 * memory of nh_tape_bytes bytes, 256-byte aligned, in the handle's precision); later,
 * nh_adjoint_step(tape) maps the adjoint of the state after that step to the adjoint of
 * the state before it.  Checkpointing is the caller's: keep the state every K steps
 * (nh_get_state), and before reversing a segment restore it (nh_set_state with p) and
 * retake its K steps with tapes. */

/* Bytes of one step's tape (15 state-sized arrays). */
size_t nh_tape_bytes(nh_handle *h);

/* nh_step (dt <= 0: the Eq. (23) step) that also writes the tape.  2D only. */
int nh_step_taped(nh_handle *h, double dt, void *tape, double *dt_taken);

/* Reverse of the taped step of size dt.  eta_bar, q1_bar, q2_bar ([ny][nx]) and w_bar
 * ([ny+1][nx+1]), device memory in the handle's precision: on entry the adjoint of
 * (eta, q1, q2, w) after the step, on return the adjoint of the state before it.  H_bar
 * ([ny][nx]) accumulates (+=) the derivative with respect to the still-water depth H.
 * p does not carry an adjoint (the solve is exact, so p^{n+1} does not depend on p^n).
 * Returns NH_EINVAL outside the limits above, NH_ENOCONV when a transposed solve does not
 * converge. */
int nh_adjoint_step(nh_handle *h, double dt, const void *tape, void *eta_bar, void *q1_bar,
                    void *q2_bar, void *w_bar, void *H_bar);

/* ---- ensembles: many independent 2D domains of uneven sizes advanced together ----
 *
 * Every domain takes the same step as a single 2D handle (Sec. 5 / App. A scheme, the
 * Chebyshev-scheduled Jacobi solve of NH_SOLVER_CHEBYSHEV), with its own grid, boundary
 * conditions, state, time step and solver convergence; the parameters (nh_params) are
 * shared.  Each kernel class runs as ONE launch for the whole ensemble over a work list of
 * (domain, tile) items, largest domain first; a domain whose pressure solve has converged
 * leaves the remaining Chebyshev passes of that stage.  The paper runs one domain at a
 * time and has no counterpart of this form.
 *
 * Layout and precision of per-domain arrays are those of nh_set_state / nh_get_state for
 * that domain's grid.  All work runs on `stream` (0: the batch creates its own non-blocking
 * stream); every call below that returns data synchronises it. */
typedef struct nh_batch nh_batch;

enum {
    NH_BATCH_AUTOTUNE = 1,  /* time the kernel-shape candidates on the ensemble's own state
                               before the first step and keep the fastest               */
    NH_BATCH_GRAPH = 2      /* run each step as one CUDA graph whose solver loops are
                               device-side conditional WHILE nodes (no host round trip) */
};

/* Kernel shapes and launch forms of a batch (candidate indices: nh_batch_candidate). */
typedef struct {
    int hyp;          /* hyperbolic-kernel cell tile                                     */
    int assembly;     /* assembly node tile                                              */
    int cheb;         /* Chebyshev-pass node region                                      */
    int persistent;   /* bit k set: kernel class k (0 hyperbolic, 1 assembly, 2 Chebyshev,
                         3 correction and breaking) runs as a persistent grid of the
                         blocks resident at once looping over the work list (a register-
                         form Chebyshev candidate: blocks of 8 consecutive work items
                         each); clear: one block per work item                            */
    int graph;        /* 1: steps run as a CUDA graph (NH_BATCH_GRAPH)                   */
    int tuned;        /* 1: chosen by the autotuner                                      */
    double ms[3];     /* autotuner's time of the chosen hyperbolic launch, assembly launch
                         and Chebyshev pass (ms, whole ensemble)                          */
} nh_batch_tuning;

/* Create a batch of n domains.  grids[d]: dim 2, nx, ny >= 2; H[d]: still-water depth of
 * domain d ([ny][nx] doubles, host memory).  params->solver must be NH_SOLVER_CHEBYSHEV
 * when nonhydrostatic is on.  Domains start at rest (eta = max(0, H) - H).  flags: OR of
 * NH_BATCH_*.  Returns NH_OK, NH_EINVAL, NH_ENOMEM or NH_ECUDA. */
int nh_create_batch(int n, const nh_grid *grids, const double *const *H,
                    const nh_params *params, void *stream, int flags, nh_batch **out);

/* Set / read the state of domain d (as nh_set_state / nh_get_state). */
int nh_batch_set_state(nh_batch *b, int d, const void *eta, const void *q1, const void *q2,
                       const void *w, const void *p, double t, int where);
int nh_batch_get_state(nh_batch *b, int d, void *eta, void *q1, void *q2, void *w, void *p,
                       double *t, int where);

/* Advance every domain by nsteps steps, each of its own Eq. (23) step (params->fixed_dt
 * when > 0).  Returns NH_ENOCONV when a solve stopped at the iteration cap, broke down or
 * met a system that is not diagonally dominant (the domain's p then keeps its previous
 * value for that stage), NH_ENONFINITE on a non-finite state.  A solve that stops
 * improving before tol (the rounding floor of FP32) ends there and is not an error; its
 * residual is in nh_batch_stats' last_resid. */
int nh_batch_run(nh_batch *b, int nsteps);

/* Counters, time step and FP64 mass of domain d. */
int nh_batch_stats(nh_batch *b, int d, nh_stats_t *out);

/* Per-kernel-class device times of the batch (as nh_profile_enable / nh_profile_read;
 * SOLVE_INIT and BICG_* count the BiCGStab fallback).  While profiling is on, steps run
 * eagerly (not as a graph) so that every launch is bracketed by events. */
int nh_batch_profile_enable(nh_batch *b, int on);
int nh_batch_profile_read(nh_batch *b, nh_profile_t *out);

/* Current kernel choice; set one by hand (disables the autotuner for this batch). */
int nh_batch_get_tuning(nh_batch *b, nh_batch_tuning *out);
int nh_batch_set_tuning(nh_batch *b, const nh_batch_tuning *in);

/* Candidate idx of kernel class kind (0 hyperbolic cell tile, 1 assembly node tile,
 * 2 Chebyshev node region incl. its 4-node halo) for a precision; NH_EINVAL past the
 * last one. */
int nh_batch_candidate(int precision, int kind, int idx, int *tile_x, int *tile_y,
                       int *threads);

const char *nh_batch_last_error(const nh_batch *b);
void nh_batch_destroy(nh_batch *b);

/* ---- kernel-level entry points used to check the stages one by one ---- */

/* Hyperbolic update of the current state alone (Eqs. 18-22 / 30, friction, clamp):
 * writes U + dt L(U) into eta_out, q1_out, q2_out ([ny][nx], handle precision). */
int nh_debug_hyperbolic(nh_handle *h, double dt, void *eta_out, void *q1_out, void *q2_out,
                        int where);

/* Pressure system of the current state taken as the post-hyperbolic state U* with
 * w* = w (App. B Eq. 43 / Eqs. 36-41, effective step dt): writes the right-hand side
 * -(8 dx dy / dt) B(q*, w*) into rhs_out and M x into mx_out (both node arrays; 1D uses
 * dy = dx).  x is a node array in the handle's precision. */
int nh_debug_system(nh_handle *h, double dt, const void *x, void *rhs_out, void *mx_out,
                    int where);

/* Failure injection for the bounded waits (the paper has no counterpart): the next
 * Chebyshev pass of the handle that runs in a register form (nh_params.cheb_form 5-7 in
 * FP32, 3 in FP64, or the cyclic form) lets block `block` announce its first region's bytes on its mbarrier
 * without issuing the copies, so that this block's first wait runs out of
 * nh_params.wait_polls polls with no copy in flight.  The step then returns NH_ETIMEOUT,
 * and the handle's state is undefined until the next nh_set_state.  Later passes are
 * unaffected.  NH_EINVAL for 1D or BiCGStab handles, or block < 0. */
int nh_debug_stall_copies(nh_handle *h, int block);

#ifdef __cplusplus
}
#endif
#endif
