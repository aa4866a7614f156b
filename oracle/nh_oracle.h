/*
 * nh_oracle.h -- plain FP64 CPU oracle for the depth-integrated non-hydrostatic
 * (Yamazaki) system of Escalante, Morales de Luna & Castro, arXiv:1706.04551.
 *
 * TEST INFRASTRUCTURE ONLY.  This header and nh_oracle.c are the reference that the
 * CUDA library is checked against.  Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline / --impl reference legs of bench.py may load it.  It shares no code,
 * header, table or constant with the CUDA library, and the library never loads it.
 *
 * Layout: cell arrays are row-major [ny][nx] (x fastest), node arrays (p, w) are
 * row-major [ny+1][nx+1]; node (I, J) sits at x = I*dx, y = J*dy, i.e. between cells
 * I-1 and I in x and J-1 and J in y.  1D problems use the or1d_* entry points with
 * cells [nx] and nodes [nx+1].  All arrays are double and owned by the caller.
 *
 * Parity status per function (pins live in tests/test_oracle_*.py, marked "not gpu"):
 *   hyperbolic step 1D/2D ................. pinned (exact dam-break solutions, lake at rest,
 *                                           mass, mirror / transpose symmetry)
 *   or1d_nh_matrix (Eq. 43) ................ pinned (operator of Eqs. 24-28, App. B A.2)
 *   or2d_apply_M / or2d_rhs / or2d_solve ... pinned (dense LU, y-invariant reduction to Eq. 43)
 *   full step 1D/2D ........................ pinned (dispersion relation, solitary wave,
 *                                           Table 1 orders, 2D == 1D on y-invariant data)
 *   breaking terms (Sec. 3, Eq. 12) ........ pinned (closed forms on linear fields in 1D and
 *                                           2D, both sides of the switch; lake at rest,
 *                                           switch-off limit, dissipation)
 *   w transport (w_transport = 1, Sec. 2) .. pinned (donor-cell upwind on uniform flow,
 *                                           uniform w kept, sum of h w kept between walls,
 *                                           no new extrema)
 *   relaxation zones (Sec. 4.4) ............ pinned (interior untouched, fixed point at the
 *                                           target, boundary cell = target, absorption of
 *                                           an outgoing solitary wave against a wall)
 *   Manning friction (1D, 2D) .............. pinned (uniform flow on a flat bottom converges
 *                                           at first order to the ODE dq/dt = -k |q| q)
 *   or1d_cfl_dt / or2d_cfl_dt (Eq. 23) ..... pinned (uniform states with u != v, dx != dy;
 *                                           fastest cell; mesh scaling; 2D -> 1D limit)
 *   wet/dry fronts of the second step ...... measured (the Sec. 4.5 literal form against
 *                                           the dry_zero option: dry-cell discharge, dry-node
 *                                           pressure, rounding sensitivity)
 * Threads: the 2D loops run under OpenMP (or_set_threads); results are bitwise the same for
 * every thread count (only loops over disjoint entries are parallel, all sums are serial).
 */
#ifndef NH_ORACLE_H
#define NH_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

/* Threads of the 2D loops (OpenMP; n <= 0 leaves the count unchanged); returns the count
 * before the call.  Results do not depend on it: only loops over disjoint entries run in
 * parallel and every sum is serial. */
int or_set_threads(int n);

enum { OR_WALL = 0, OR_OUTFLOW = 1, OR_PERIODIC = 2 };

typedef struct {
    int nx, ny;          /* cells; 1D entry points ignore ny                          */
    double dx, dy;
    int bc[4];           /* west, east, south, north (OR_WALL / OR_OUTFLOW / OR_PERIODIC;
                            periodic only in 1D)                                      */
    double g, cfl;
    double delta;        /* desingularisation depth of Sec. 4.5 (1e-5)                 */
    double hdry;         /* a cell is dry when h <= hdry                              */
    double manning;      /* Gauckler-Manning n                                         */
    double B1, B2;       /* breaking calibration, Eq. (9)                              */
    int breaking;        /* 1: breaking terms of Eq. (12)                              */
    int nonhydro;        /* 1: full scheme; 0: hydrostatic SWE only (p = 0)            */
    double tol;          /* 2D Krylov relative-residual tolerance                       */
    int max_iter;
    int w_transport;     /* 1: energy-consistent w equation (hw)_t + div(hw u) = p of the
                            system of [7] (Sec. 2), hw moved upwind on the node (dual)
                            cells; 0: Yamazaki's h w_t = p                                */
    double relax[4];     /* L_Rel of the generating / absorbing zone (Sec. 4.4) on the west,
                            east, south, north side; 0: none (1D: west, east)             */
    int dry_zero;        /* 0: the second step as Sec. 4.5 states it, no truncation at
                            wet/dry fronts; 1: q = 0 in dry cells (h <= hdry) after each
                            stage (App. B A.2's premise q = w = 0 where h vanishes; the
                            default of the Python wrapper's cfg())                        */
} or_cfg;

typedef struct {
    int iters[2];        /* solver iterations of the two RK stages                      */
    double resid[2];     /* final relative residual ||b - M p|| / ||b||                 */
    int clamped;         /* cells whose depth went negative and was clamped             */
} or_stats;

/* ---- 1D (Sec. 4) ---- */
double or1d_cfl_dt(const or_cfg *c, const double *H, const double *h, const double *q);
int or1d_step(const or_cfg *c, const double *H, double *h, double *q, double *w, double *p,
              double dt, or_stats *st);
int or1d_hyperbolic(const or_cfg *c, const double *H, const double *h, const double *q,
                    double dt, double *ho, double *qo);
int or1d_nh_matrix(const or_cfg *c, const double *H, const double *h, const double *q,
                   const double *w, double dt, double *a, double *b, double *cc, double *rhs);
int or1d_affine_apply(const or_cfg *c, const double *H, const double *h, const double *p,
                      double dt, double *out);
int or1d_nh_solve(const or_cfg *c, const double *H, const double *h, const double *q,
                  const double *w, double dt, double *p);
int or1d_thomas(int n, const double *a, const double *b, const double *c, const double *d,
                double *x);
long long or1d_run(const or_cfg *c, const double *H, double *h, double *q, double *w,
                   double *p, double t_end, long long max_steps, double fixed_dt, double *t_out);
/* Generating / absorbing relaxation zones of Sec. 4.4 (zone widths c->relax): blends
 * (h, q) at the zone cells and (w, p) at the zone nodes toward the target (eta_t = h* - H,
 * q_t, w_t, p_t); a NULL target is the lake at rest (h* = max(H, 0), q* = w* = p* = 0),
 * which makes the zone absorbing.  or1d_run / or2d_run apply the absorbing form after
 * every step when a width is set; or1d_step / or2d_step never relax. */
void or1d_relax(const or_cfg *c, const double *H, double *h, double *q, double *w, double *p,
                const double *eta_t, const double *q_t, const double *w_t, const double *p_t);
/* The breaking terms of Sec. 3 / Eq. (12) alone (cells: q += dt 2 nu u_x H_x; nodes:
 * w += dt 2 nu u_x / h), in place. */
void or1d_breaking(const or_cfg *c, const double *H, const double *h, double *q, double *w,
                   double dt);

/* ---- 2D (Sec. 5, App. A) ---- */
double or2d_cfl_dt(const or_cfg *c, const double *H, const double *h, const double *q1,
                   const double *q2);
int or2d_step(const or_cfg *c, const double *H, double *h, double *q1, double *q2, double *w,
              double *p, double dt, or_stats *st);
int or2d_stage(const or_cfg *c, const double *H, const double *h, const double *q1,
               const double *q2, const double *w, double *p, double dt, double *ho,
               double *q1o, double *q2o, double *wo, int *iters, double *resid);
int or2d_hyperbolic(const or_cfg *c, const double *H, const double *h, const double *q1,
                    const double *q2, double dt, double *ho, double *q1o, double *q2o);
int or2d_rhs(const or_cfg *c, const double *H, const double *h, const double *q1,
             const double *q2, const double *w, double dt, double *rhs);
int or2d_apply_M(const or_cfg *c, const double *H, const double *h, const double *p,
                 double dt, double *out);
int or2d_solve(const or_cfg *c, const double *H, const double *h, const double *rhs,
               double dt, double *p, int *iters, double *resid);
long long or2d_run(const or_cfg *c, const double *H, double *h, double *q1, double *q2,
                   double *w, double *p, double t_end, long long max_steps, double fixed_dt,
                   double *t_out, long long *iters_total);
void or2d_relax(const or_cfg *c, const double *H, double *h, double *q1, double *q2,
                double *w, double *p, const double *eta_t, const double *q1_t,
                const double *q2_t, const double *w_t, const double *p_t);
void or2d_breaking(const or_cfg *c, const double *H, const double *h, double *q1, double *q2,
                   double *w, double dt);

#ifdef __cplusplus
}
#endif
#endif
