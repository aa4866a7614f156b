/*
 * nh_oracle.c -- plain, slow FP64 CPU oracle for one time step of the depth-integrated
 * non-hydrostatic (Yamazaki) system, discretised as in Escalante, Morales de Luna &
 * Castro, "Non-hydrostatic pressure shallow flows: GPU implementation using finite
 * volume and finite difference scheme" (arXiv:1706.04551).
 *
 * TEST INFRASTRUCTURE ONLY.  The CUDA library is checked against this file; it is loaded
 * by tests/, __graft_entry__.smoke() and bench.py's cpu_baseline / reference legs and by
 * nothing else.  It shares no code with the CUDA path.  It is written for a reader who
 * checks it against the paper: every loop follows one equation, in the paper's order,
 * with no fusion or blocking.
 *
 * What it computes, per time step (Sec. 4.3, Sec. 5, Sec. 6 "steps 1-4 twice"):
 *   for each of the two stages of the TVD Runge-Kutta method:
 *     (i)   ghost cells (Sec. 4.4; walls are mirror ghosts -- reading, see below),
 *     (ii)  MUSCL-minmod reconstruction of h, eta, u (and v) (Sec. 4.1, Eqs. 20-22),
 *     (iii) PVM / HLL path-conservative update (Eqs. 18-19, 20-22; 2D Eq. 30),
 *     (iv)  semi-implicit Manning friction, breaking terms (Sec. 3, Eq. 12),
 *     (v)   compact finite-difference pressure system (Eqs. 24-29, 37-41, App. B Eq. 43),
 *     (vi)  projection / correction of q and w (Eqs. 26-28, 36, 41);
 *   in the Shu-Osher form of the second-order TVD Runge-Kutta method: stage 2 projects
 *   the combination (U^n + U^(1) + dt L(U^(1))) / 2 with the step dt / 2.
 * Readings of the paper used here:
 *   - App. B prints the right-hand side of Eq. (43) without its minus sign; substituting
 *     the correction into Eq. (28) gives A p = -(8 dx^2 / dt) B(q*, w*).  Used here.
 *   - The w equation of Eq. (28) adds dt*R_w without the 1/h that Eq. (14) implies; we
 *     divide by h (desingularised) as the units require.  In the pressure matrix the
 *     2 h w term contributes 2 dt p exactly (h cancels), as in Eq. (43).
 *   - Eq. (40) divides by 2 where dx (dy) is meant.
 *   - Walls (not in the paper) are mirror ghosts: h, eta, H, tangential q, p, w even,
 *     normal q odd.  Outflow ghosts copy the first interior cell (Sec. 4.4); boundary
 *     pressure nodes are unknowns whose outside neighbour mirrors the inside one.
 *   - Emerging bottoms (Sec. 4.5): a cell is dry when h <= hdry; at a face whose dry
 *     side's bed is at or above the wet side's free surface, the free-surface jump in
 *     T_p and in the alpha_0 term is set to 0; eta slopes are 0 next to dry cells.
 *   - 2D PVM (Sec. 5 cites [18] without the formulas): per face in the normal frame,
 *     Eq. (18) for (h, q_n) and the same (1 +- alpha_1) / alpha_0 weights for q_t with
 *     convective flux q_n q_t / h.
 *   - 2D breaking (Sec. 5 refers to Sec. 3): q_x -> div q and u_x -> div u.  The switch
 *     is stateless: active where |div q| >= U_1 and B > 0.
 *   - Runge-Kutta (Sec. 4.3, Sec. 6 "steps 1-4 are repeated twice"): the projection of the
 *     second stage acts on the Shu-Osher combination, so U^{n+1} itself satisfies the
 *     discrete constraint; p^{n+1} is that projection's pressure.
 *   - Wet/dry fronts in the second step (Sec. 4.5 states that they need no special
 *     treatment): the correction T_NH has a term p (2 eta - h)_x that does not vanish
 *     with h, so a dry cell next to the shoreline takes up a small discharge.  Whether a
 *     later step clamps that cell's depth (and zeroes the discharge) then hangs on depths
 *     of 1e-20 m and below that the flux arithmetic leaves in dry cells.  dry_zero = 1
 *     sets q = 0 in dry cells after each stage (App. B A.2 takes q = w = 0 where the depth
 *     vanishes), which removes that dependence; dry_zero = 0 is the literal form.
 *   - dt (Eq. 23) in 2D: CFL / max((|u|+c)/dx + (|v|+c)/dy), from the current state.
 *   - The 2D system is solved by unpreconditioned BiCGStab to a relative residual tol.
 *   - Energy-consistent w equation (w_transport = 1; Sec. 2 names the system of [7] and
 *     says the scheme extends to it, without a discretisation): hw is moved on the node
 *     (dual) cells by the hyperbolic step's face mass fluxes, upwind in w, and the
 *     Runge-Kutta combination acts on hw (wtransport1d / wtransport2d).
 *   - Relaxation zones (Sec. 4.4): each zone is the k + 1 cells nearest its boundary, the
 *     distance in m is measured from the zone's inner cell on both sides (the paper's two
 *     index sets disagree), m is clamped at 0, overlapping zones multiply, the absorbing
 *     target is the lake at rest (eta* = max(H, 0) - H, not h* = 0), and the blend acts on
 *     the state after each whole time step (relax_m1, or1d_relax, or2d_relax).
 */
#include "nh_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* Threads of the 2D loops.  Only loops whose iterations write disjoint entries carry an
 * OpenMP pragma; every sum (the dot products of BiCGStab) stays serial, so the results
 * do not depend on the thread count, bit for bit. */
int or_set_threads(int n)
{
#ifdef _OPENMP
    int old = omp_get_max_threads();
    if (n > 0) omp_set_num_threads(n);
    return old;
#else
    (void)n;
    return 1;
#endif
}

/* ------------------------------------------------------------------------- */
/* scalar helpers                                                             */
/* ------------------------------------------------------------------------- */

/* minmod limiter used by the MUSCL reconstruction (Sec. 4.1). */
static double minmod(double a, double b)
{
    if (a > 0.0 && b > 0.0) return a < b ? a : b;
    if (a < 0.0 && b < 0.0) return a > b ? a : b;
    return 0.0;
}

/* Velocity desingularisation formula of Sec. 4.5: u = sqrt(2) h q / sqrt(h^4 + max(h^4, d^4)).
 * With q = 1 it gives the desingularised 1/h used in the w update. */
static double desing(double h, double q, double delta)
{
    double h4 = h * h * h * h;
    double d4 = delta * delta * delta * delta;
    double den = sqrt(h4 + (h4 > d4 ? h4 : d4));
    return sqrt(2.0) * h * q / den;
}

/* Path-conservative PVM-HLL fluctuations at one face, Eqs. (18)-(19), in the face-normal
 * frame: component 0 = h, 1 = normal discharge, 2 = tangential discharge.
 * L / R are the reconstructed states on the two sides (h, eta, u_n, u_t). */
static void pvm_face(double g, double hdry,
                     double hL, double etaL, double unL, double utL,
                     double hR, double etaR, double unR, double utR,
                     double Dm[3], double Dp[3])
{
    double qnL = hL * unL, qnR = hR * unR;
    double qtL = hL * utL, qtR = hR * utR;

    /* Roe averages (Sec. 4.1). */
    double hbar = 0.5 * (hL + hR);
    double sL = sqrt(hL), sR = sqrt(hR);
    double ubar = (sL + sR > 0.0) ? (unL * sL + unR * sR) / (sL + sR) : 0.0;

    /* HLL wave-speed bounds S_L, S_R (Sec. 4.1). */
    double cbar = sqrt(g * hbar);
    double SL = fmin(ubar - cbar, unL - sqrt(g * hL));
    double SR = fmax(ubar + cbar, unR + sqrt(g * hR));

    /* Emerging bottom (Sec. 4.5): the dry side's bed at or above the wet free surface. */
    double deta = etaR - etaL;
    if (hR <= hdry && (etaR - hR) >= etaL) deta = 0.0;
    if (hL <= hdry && (etaL - hL) >= etaR) deta = 0.0;

    for (int k = 0; k < 3; ++k) { Dm[k] = 0.0; Dp[k] = 0.0; }
    if (!(SR - SL > 0.0)) return;

    /* PVM coefficients of Q = alpha_0 Id + alpha_1 A (Sec. 4.1). */
    double a0 = (SR * fabs(SL) - SL * fabs(SR)) / (SR - SL);
    double a1 = (fabs(SR) - fabs(SL)) / (SR - SL);

    /* R = F_c(U_R) - F_c(U_L) + T_p, Eq. (19); F_c = (q_n, q_n^2/h, q_n q_t/h). */
    double R[3], V[3];
    R[0] = qnR - qnL;
    R[1] = qnR * unR - qnL * unL + g * hbar * deta;
    R[2] = qnR * utR - qnL * utL;
    /* U_R - U_L - (H_R - H_L) e_1 : the h component becomes the free-surface jump. */
    V[0] = deta;
    V[1] = qnR - qnL;
    V[2] = qtR - qtL;

    /* Eq. (18). */
    for (int k = 0; k < 3; ++k) {
        Dm[k] = 0.5 * ((1.0 - a1) * R[k] - a0 * V[k]);
        Dp[k] = 0.5 * ((1.0 + a1) * R[k] + a0 * V[k]);
    }
}

/* Breaking eddy viscosity, Eq. (9), stateless switch: nu = B h |d| where d is q_x
 * (div q in 2D), B = 1 - d / U_1, U_1 = B_1 sqrt(g h); zero unless |d| >= U_1, B > 0. */
static double breaking_nu(const or_cfg *c, double h, double d)
{
    if (!(h > c->hdry)) return 0.0;
    double U1 = c->B1 * sqrt(c->g * h);
    if (!(fabs(d) >= U1) || !(U1 > 0.0)) return 0.0;
    double B = 1.0 - d / U1;
    return B > 0.0 ? B * h * fabs(d) : 0.0;
}

/* ------------------------------------------------------------------------- */
/* 1D (Sec. 4)                                                               */
/* ------------------------------------------------------------------------- */

#define G1 2 /* ghost cells per side */

/* Fill the two ghost cells on each side of an extended 1D cell array of n + 4 entries
 * (interior at 2 .. n+1).  parity: +1 for fields even under reflection (h, H), -1 for the
 * discharge.  First layer on both sides, then the second (which may reflect a first-layer
 * ghost when n == 1). */
static void ghost1d(const or_cfg *c, int n, double *v, double parity)
{
    switch (c->bc[0]) {
    case OR_WALL:     v[1] = parity * v[2]; break;
    case OR_OUTFLOW:  v[1] = v[2]; break;
    case OR_PERIODIC: v[1] = v[n + 1]; break;
    }
    switch (c->bc[1]) {
    case OR_WALL:     v[n + 2] = parity * v[n + 1]; break;
    case OR_OUTFLOW:  v[n + 2] = v[n + 1]; break;
    case OR_PERIODIC: v[n + 2] = v[2]; break;
    }
    switch (c->bc[0]) {
    case OR_WALL:     v[0] = parity * v[3]; break;
    case OR_OUTFLOW:  v[0] = v[2]; break;
    case OR_PERIODIC: v[0] = v[n]; break;
    }
    switch (c->bc[1]) {
    case OR_WALL:     v[n + 3] = parity * v[n]; break;
    case OR_OUTFLOW:  v[n + 3] = v[n + 1]; break;
    case OR_PERIODIC: v[n + 3] = v[3]; break;
    }
}

static int periodic1d(const or_cfg *c) { return c->bc[0] == OR_PERIODIC; }

/* Relaxation coefficient of Sec. 4.4 for cell i (0-based) of a line of n cells of size d,
 * with zone widths Llo (low side) and Lhi (high side); 1 outside both zones.  k is the
 * first natural number with k d >= L; m = sqrt(1 - (dist / L)^2), clamped at 0.
 * Reading (the paper lists the zone cells as {1..k} on the left, measuring the distance
 * from I_1, and {N-k..N} on the right, measuring it from I_{N-k}; the two disagree, and
 * the left form would leave the boundary cell unrelaxed): each zone is the k + 1 cells
 * nearest its boundary and dist is measured from the zone's inner cell, so m = 1 there
 * and m = 0 at the boundary cell, on both sides.  Where zones overlap the two factors
 * multiply (the two blends applied one after the other). */
static int relax_k(double L, double d)
{
    int k = 0;
    while ((double)k * d < L) ++k;
    return k;
}
static double relax_m1(int i, int n, double d, double Llo, double Lhi)
{
    double m = 1.0;
    if (Llo > 0.0) {
        int k = relax_k(Llo, d);
        if (i <= k) {
            double r = (double)(k - i) * d / Llo, v = 1.0 - r * r;
            m *= v > 0.0 ? sqrt(v) : 0.0;
        }
    }
    if (Lhi > 0.0) {
        int k = relax_k(Lhi, d);
        if (i >= n - 1 - k) {
            double r = (double)(i - (n - 1 - k)) * d / Lhi, v = 1.0 - r * r;
            m *= v > 0.0 ? sqrt(v) : 0.0;
        }
    }
    return m;
}
/* Node coefficient m_{i-1/2} = (m_{i-1} + m_i) / 2 for node I between cells I-1 and I
 * (Sec. 4.4); the cell beyond an end takes the end cell's m. */
static double relax_node1(int I, int n, double d, double Llo, double Lhi)
{
    int a = I - 1 < 0 ? 0 : I - 1, b = I > n - 1 ? n - 1 : I;
    return 0.5 * (relax_m1(a, n, d, Llo, Lhi) + relax_m1(b, n, d, Llo, Lhi));
}

void or1d_relax(const or_cfg *c, const double *H, double *h, double *q, double *w, double *p,
                const double *eta_t, const double *q_t, const double *w_t, const double *p_t)
{
    const int n = c->nx;
    for (int i = 0; i < n; ++i) {
        double m = relax_m1(i, n, c->dx, c->relax[0], c->relax[1]);
        if (m == 1.0) continue;
        double hs = eta_t ? eta_t[i] + H[i] : (H[i] > 0.0 ? H[i] : 0.0);
        if (hs < 0.0) hs = 0.0;
        h[i] = m * h[i] + (1.0 - m) * hs;
        q[i] = m * q[i] + (1.0 - m) * (q_t ? q_t[i] : 0.0);
    }
    for (int I = 0; I <= n; ++I) {
        double m = relax_node1(I, n, c->dx, c->relax[0], c->relax[1]);
        if (m == 1.0) continue;
        w[I] = m * w[I] + (1.0 - m) * (w_t ? w_t[I] : 0.0);
        p[I] = m * p[I] + (1.0 - m) * (p_t ? p_t[I] : 0.0);
    }
}

double or1d_cfl_dt(const or_cfg *c, const double *H, const double *h, const double *q)
{
    (void)H;
    double lmax = 0.0;
    for (int i = 0; i < c->nx; ++i) {
        double u = desing(h[i], q[i], c->delta);
        double l = fabs(u) + sqrt(c->g * h[i]);      /* Eq. (23) */
        if (l > lmax) lmax = l;
    }
    return lmax > 0.0 ? c->cfl * c->dx / lmax : 0.0;
}

/* Hyperbolic step of Sec. 4.1 (Eqs. 18-22) plus semi-implicit Manning friction and the
 * non-negative depth clamp; writes U^{n+1/2}.  Fm (n + 1 entries, or NULL): the mass flux
 * of every face, F_h(U^-) + D^-_h, seen from its left cell. */
static int hyp1d(const or_cfg *c, const double *H, const double *h, const double *q,
                 double dt, double *ho, double *qo, double *Fm)
{
    const int n = c->nx, ne = n + 2 * G1;
    const double dx = c->dx, g = c->g;
    int clamped = 0;
    double *he = calloc(ne, sizeof(double)), *qe = calloc(ne, sizeof(double));
    double *He = calloc(ne, sizeof(double)), *ee = calloc(ne, sizeof(double));
    double *ue = calloc(ne, sizeof(double));
    double *hE = calloc(ne, sizeof(double)), *hW = calloc(ne, sizeof(double));
    double *eE = calloc(ne, sizeof(double)), *eW = calloc(ne, sizeof(double));
    double *uE = calloc(ne, sizeof(double)), *uW = calloc(ne, sizeof(double));
    double *Dm = calloc(2 * (n + 1), sizeof(double)), *Dp = calloc(2 * (n + 1), sizeof(double));

    for (int i = 0; i < n; ++i) { he[i + G1] = h[i]; qe[i + G1] = q[i]; He[i + G1] = H[i]; }
    ghost1d(c, n, he, 1.0);
    ghost1d(c, n, qe, -1.0);
    ghost1d(c, n, He, 1.0);
    for (int e = 0; e < ne; ++e) {
        ee[e] = he[e] - He[e];                       /* eta = h - H */
        ue[e] = desing(he[e], qe[e], c->delta);      /* Sec. 4.5 */
    }

    /* MUSCL-minmod reconstruction of h, eta and u for cells -1 .. n (Sec. 4.1). */
    for (int e = 1; e <= n + 2; ++e) {
        double sh = minmod(he[e] - he[e - 1], he[e + 1] - he[e]);
        double su = minmod(ue[e] - ue[e - 1], ue[e + 1] - ue[e]);
        int dry = he[e - 1] <= c->hdry || he[e] <= c->hdry || he[e + 1] <= c->hdry;
        double se = dry ? 0.0 : minmod(ee[e] - ee[e - 1], ee[e + 1] - ee[e]);
        hE[e] = he[e] + 0.5 * sh; hW[e] = he[e] - 0.5 * sh;
        eE[e] = ee[e] + 0.5 * se; eW[e] = ee[e] - 0.5 * se;
        uE[e] = ue[e] + 0.5 * su; uW[e] = ue[e] - 0.5 * su;
    }

    /* Fluctuations D^-, D^+ at faces k = 0 .. n (face k between cells k-1 and k). */
    for (int k = 0; k <= n; ++k) {
        int L = k + 1, R = k + 2;
        double dm[3], dp[3];
        pvm_face(g, c->hdry, hE[L], eE[L], uE[L], 0.0, hW[R], eW[R], uW[R], 0.0, dm, dp);
        Dm[2 * k] = dm[0]; Dm[2 * k + 1] = dm[1];
        Dp[2 * k] = dp[0]; Dp[2 * k + 1] = dp[1];
        if (Fm) Fm[k] = hE[L] * uE[L] + dm[0];
    }

    /* Cell update, Eq. (20), with the inner-cell term of Eq. (22) in free-surface form:
     * I = F_c(U^-_{i+1/2}) - F_c(U^+_{i-1/2}) + (0, g h_i (eta^-_{i+1/2} - eta^+_{i-1/2})). */
    for (int i = 0; i < n; ++i) {
        int e = i + G1;
        double I0 = hE[e] * uE[e] - hW[e] * uW[e];
        double I1 = hE[e] * uE[e] * uE[e] - hW[e] * uW[e] * uW[e] + g * he[e] * (eE[e] - eW[e]);
        double hn = he[e] - dt / dx * (Dm[2 * (i + 1)] + Dp[2 * i] + I0);
        double qn = qe[e] - dt / dx * (Dm[2 * (i + 1) + 1] + Dp[2 * i + 1] + I1);
        /* Semi-implicit Manning friction (Sec. 2 and Sec. 4): q_t = -g n^2 |u| q / h^(4/3). */
        if (c->manning > 0.0 && hn > 0.0) {
            double u = desing(hn, qn, c->delta);
            double hd = hn > c->delta ? hn : c->delta;
            qn = qn / (1.0 + dt * g * c->manning * c->manning * fabs(u) / pow(hd, 4.0 / 3.0));
        }
        if (hn < 0.0) { hn = 0.0; qn = 0.0; ++clamped; }
        ho[i] = hn; qo[i] = qn;
    }

    free(he); free(qe); free(He); free(ee); free(ue);
    free(hE); free(hW); free(eE); free(eW); free(uE); free(uW); free(Dm); free(Dp);
    return clamped;
}

int or1d_hyperbolic(const or_cfg *c, const double *H, const double *h, const double *q,
                    double dt, double *ho, double *qo)
{
    return hyp1d(c, H, h, q, dt, ho, qo, NULL);
}

/* Breaking terms of Eq. (12)/(14) in 1D: q += dt * 2 nu u_x H_x at cells (centred
 * differences, Sec. 4.3), w += dt * 2 nu u_x / h at nodes (two-cell differences). */
static void breaking1d(const or_cfg *c, const double *H, const double *h, double *q,
                       double *w, double dt)
{
    const int n = c->nx, ne = n + 2 * G1;
    double *he = calloc(ne, sizeof(double)), *qe = calloc(ne, sizeof(double));
    double *He = calloc(ne, sizeof(double)), *ue = calloc(ne, sizeof(double));
    for (int i = 0; i < n; ++i) { he[i + G1] = h[i]; qe[i + G1] = q[i]; He[i + G1] = H[i]; }
    ghost1d(c, n, he, 1.0); ghost1d(c, n, qe, -1.0); ghost1d(c, n, He, 1.0);
    for (int e = 0; e < ne; ++e) ue[e] = desing(he[e], qe[e], c->delta);
    for (int i = 0; i < n; ++i) {
        int e = i + G1;
        double qx = (qe[e + 1] - qe[e - 1]) / (2.0 * c->dx);
        double ux = (ue[e + 1] - ue[e - 1]) / (2.0 * c->dx);
        double Hx = (He[e + 1] - He[e - 1]) / (2.0 * c->dx);
        double nu = breaking_nu(c, he[e], qx);
        q[i] += dt * 2.0 * nu * ux * Hx;
    }
    int nn = periodic1d(c) ? n : n + 1;
    for (int k = 0; k < nn; ++k) {
        int L = k + 1, R = k + 2;
        double hn = 0.5 * (he[L] + he[R]);
        double qx = (qe[R] - qe[L]) / c->dx;
        double ux = (ue[R] - ue[L]) / c->dx;
        double nu = breaking_nu(c, hn, qx);
        w[k] += dt * 2.0 * nu * ux * desing(hn, 1.0, c->delta);
    }
    if (periodic1d(c)) w[n] = w[0];
    free(he); free(qe); free(He); free(ue);
}

/* Extended (ghosted) h, s = 2 eta - h and the cell values xi_i = dx (2 eta_x - h_x)_i of
 * Eq. (27) (centred), for cells -1 .. n.  Arrays have n + 4 entries. */
static void nh1d_fields(const or_cfg *c, const double *H, const double *h, double *he,
                        double *se, double *xi)
{
    const int n = c->nx, ne = n + 2 * G1;
    double *He = calloc(ne, sizeof(double));
    for (int i = 0; i < n; ++i) { he[i + G1] = h[i]; He[i + G1] = H[i]; }
    ghost1d(c, n, he, 1.0); ghost1d(c, n, He, 1.0);
    for (int e = 0; e < ne; ++e) se[e] = 2.0 * (he[e] - He[e]) - he[e];
    for (int e = 0; e < ne; ++e) xi[e] = 0.0;
    for (int e = 1; e <= n + 2; ++e) xi[e] = 0.5 * (se[e + 1] - se[e - 1]);
    free(He);
}

/* Tridiagonal system of App. B, Eqs. (42)-(43), for nodes k = 0 .. n (node k between
 * cells k-1 and k), with the right-hand side -(8 dx^2/dt) B(q*, w*) of Eq. (24) (sign:
 * reading of Eq. (28)).  Boundary rows fold the outside neighbour onto its mirror.
 * Periodic: n unknowns, a[0] couples node n-1 and cc[n-1] couples node 0. */
int or1d_nh_matrix(const or_cfg *c, const double *H, const double *h, const double *q,
                   const double *w, double dt, double *a, double *b, double *cc, double *rhs)
{
    const int n = c->nx, ne = n + 2 * G1;
    const double dx = c->dx;
    double *he = calloc(ne, sizeof(double)), *se = calloc(ne, sizeof(double));
    double *xi = calloc(ne, sizeof(double)), *qe = calloc(ne, sizeof(double));
    nh1d_fields(c, H, h, he, se, xi);
    for (int i = 0; i < n; ++i) qe[i + G1] = q[i];
    ghost1d(c, n, qe, -1.0);
    int nn = periodic1d(c) ? n : n + 1;
    for (int k = 0; k < nn; ++k) {
        int L = k + 1, R = k + 2;                   /* cells k-1 (i) and k (i+1) */
        double hn = 0.5 * (he[L] + he[R]);          /* h_{i+1/2}, Eq. (25) */
        double xin = se[R] - se[L];                 /* xi_{i+1/2} = dx (2 eta_x - h_x)_{i+1/2} */
        double xL = xi[L], xR = xi[R];
        a[k] = (xL - 2.0 * he[L]) * (xin + 2.0 * hn);
        b[k] = 16.0 * dx * dx + xin * (xL + xR + 2.0 * he[L] - 2.0 * he[R])
             + 2.0 * hn * (xL - xR + 4.0 * hn);
        cc[k] = (xR + 2.0 * he[R]) * (xin - 2.0 * hn);
        /* B(q*, w*) at the node, Eq. (24) with the point values of Eq. (25). */
        double Bs = hn * (qe[R] - qe[L]) / dx - 0.5 * (qe[R] + qe[L]) * xin / dx
                  + 2.0 * hn * w[k];
        rhs[k] = -(8.0 * dx * dx / dt) * Bs;
    }
    if (!periodic1d(c)) {
        cc[0] += a[0]; a[0] = 0.0;
        a[n] += cc[n]; cc[n] = 0.0;
    }
    free(he); free(se); free(xi); free(qe);
    return 0;
}

/* The same operator built generically: p -> (8 dx^2/dt) [B(q* + dt T(p), w* + dt p/h) -
 * B(q*, w*)], i.e. Eq. (24) applied to the correction of Eqs. (26)-(28) with the ghost
 * cells' own corrections (the 2 h w term contributes 2 dt p exactly). */
int or1d_affine_apply(const or_cfg *c, const double *H, const double *h, const double *p,
                      double dt, double *out)
{
    const int n = c->nx, ne = n + 2 * G1;
    const double dx = c->dx;
    double *he = calloc(ne, sizeof(double)), *se = calloc(ne, sizeof(double));
    double *xi = calloc(ne, sizeof(double)), *pe = calloc(n + 3, sizeof(double));
    double *T = calloc(ne, sizeof(double));
    nh1d_fields(c, H, h, he, se, xi);
    /* nodes -1 .. n+1 stored at pe[k + 1] */
    if (periodic1d(c)) {
        for (int k = 0; k < n; ++k) pe[k + 1] = p[k];
        pe[n + 1] = p[0]; pe[0] = p[n - 1]; pe[n + 2] = p[1 % n];
    } else {
        for (int k = 0; k <= n; ++k) pe[k + 1] = p[k];
        pe[0] = p[1]; pe[n + 2] = p[n - 1];
    }
    /* T_NH of Eq. (26) with the point values of Eq. (27), cells -1 .. n */
    for (int e = 1; e <= n + 2; ++e) {
        int i = e - G1;                     /* cell index; west node i, east node i+1 */
        double pw = pe[i + 1], pE = pe[i + 2];
        double pi = 0.5 * (pE + pw), px = (pE - pw) / dx;
        T[e] = -0.5 * (he[e] * px + pi * xi[e] / dx);
    }
    int nn = periodic1d(c) ? n : n + 1;
    for (int k = 0; k < nn; ++k) {
        int L = k + 1, R = k + 2;
        double hn = 0.5 * (he[L] + he[R]);
        double xin = se[R] - se[L];
        double dqL = dt * T[L], dqR = dt * T[R];
        double Bl = hn * (dqR - dqL) / dx - 0.5 * (dqR + dqL) * xin / dx + 2.0 * dt * p[k];
        out[k] = (8.0 * dx * dx / dt) * Bl;
    }
    free(he); free(se); free(xi); free(pe); free(T);
    return 0;
}

/* Thomas algorithm for a[i] x[i-1] + b[i] x[i] + c[i] x[i+1] = d[i] (Sec. 4.3). */
int or1d_thomas(int n, const double *a, const double *b, const double *c, const double *d,
                double *x)
{
    double *cp = malloc(n * sizeof(double)), *dp = malloc(n * sizeof(double));
    cp[0] = c[0] / b[0];
    dp[0] = d[0] / b[0];
    for (int i = 1; i < n; ++i) {
        double m = b[i] - a[i] * cp[i - 1];
        cp[i] = c[i] / m;
        dp[i] = (d[i] - a[i] * dp[i - 1]) / m;
    }
    x[n - 1] = dp[n - 1];
    for (int i = n - 2; i >= 0; --i) x[i] = dp[i] - cp[i] * x[i + 1];
    free(cp); free(dp);
    return 0;
}

/* Cyclic tridiagonal solve (periodic BC of Sec. 4.4, "a modification of the Thomas
 * algorithm"): Sherman-Morrison on top of two Thomas solves. */
static void thomas_cyclic(int n, const double *a, const double *b, const double *c,
                          const double *d, double *x)
{
    double alpha = c[n - 1], beta = a[0];
    double gam = -b[0];
    double *bb = malloc(n * sizeof(double)), *u = calloc(n, sizeof(double));
    double *z = malloc(n * sizeof(double));
    memcpy(bb, b, n * sizeof(double));
    bb[0] = b[0] - gam;
    bb[n - 1] = b[n - 1] - alpha * beta / gam;
    or1d_thomas(n, a, bb, c, d, x);
    u[0] = gam; u[n - 1] = alpha;
    or1d_thomas(n, a, bb, c, u, z);
    double fact = (x[0] + beta * x[n - 1] / gam) / (1.0 + z[0] + beta * z[n - 1] / gam);
    for (int i = 0; i < n; ++i) x[i] -= fact * z[i];
    free(bb); free(u); free(z);
}

/* Assemble Eq. (43) with the RHS of the projection and solve it (Thomas, or the cyclic
 * variant for periodic boundaries); p has nx + 1 entries. */
int or1d_nh_solve(const or_cfg *c, const double *H, const double *h, const double *q,
                  const double *w, double dt, double *p)
{
    const int n = c->nx;
    int nn = periodic1d(c) ? n : n + 1;
    double *A = calloc(nn, sizeof(double)), *B = calloc(nn, sizeof(double));
    double *cc = calloc(nn, sizeof(double)), *r = calloc(nn, sizeof(double));
    or1d_nh_matrix(c, H, h, q, w, dt, A, B, cc, r);
    if (periodic1d(c)) { thomas_cyclic(nn, A, B, cc, r, p); p[n] = p[0]; }
    else or1d_thomas(nn, A, B, cc, r, p);
    free(A); free(B); free(cc); free(r);
    return 0;
}

/* Energy-consistent w equation (Sec. 2, the system of [7]): (hw)_t + (hwu)_x = p in place
 * of h w_t = p.  The paper gives no discretisation; the reading used here: hw lives on the
 * nodes like w.  Node k owns the dual cell between the centres of cells k-1 and k (its
 * inner half at a wall or outflow end), whose depth is the mean depth of those two cells.
 * A dual face at the centre of cell i carries the mean of the mass fluxes of cell i's two
 * faces in the hyperbolic step (F = F_h(U^-) + D^-_h per face); at a wall or outflow end
 * the outer dual face is the boundary face itself.  w is taken upwind at every dual face
 * (first order), and the node's own w at the boundary faces.  Those dual fluxes move the
 * dual-cell depth exactly as the mean of the two cell depths moves, so a uniform w stays
 * uniform and sum(h w) over the dual cells changes only through the boundary faces.  The
 * Runge-Kutta combination acts on the conserved hw:
 *   (hw)* = a h_b w_b + b (h w - dt div(F w)),   w* = (hw)* / h* (desingularised),
 * the node depths h_b, h, h* being those of the base, input and combined states. */
static void wtransport1d(const or_cfg *c, const double *hb, const double *wb,
                         const double *h, const double *w, const double *F,
                         const double *hs, double a, double bw, double dt, double *wo)
{
    const int n = c->nx, ne = n + 2 * G1, per = periodic1d(c);
    double *eb = calloc(ne, sizeof(double)), *ei = calloc(ne, sizeof(double));
    double *es = calloc(ne, sizeof(double));
    for (int i = 0; i < n; ++i) { eb[i + G1] = hb[i]; ei[i + G1] = h[i]; es[i + G1] = hs[i]; }
    ghost1d(c, n, eb, 1.0); ghost1d(c, n, ei, 1.0); ghost1d(c, n, es, 1.0);
    const int nk = per ? n : n + 1;          /* distinct nodes (periodic: node n is node 0) */
    for (int k = 0; k < nk; ++k) {
        const int west_end = !per && k == 0, east_end = !per && k == n;
        const double area = (west_end || east_end) ? 0.5 : 1.0;
        const int kw = k == 0 ? n - 1 : k - 1;   /* west neighbour (periodic wrap at 0) */
        const double FE = east_end ? F[n] : 0.5 * (F[k] + F[k + 1]);
        const double FW = west_end ? F[0] : 0.5 * (F[kw] + F[kw + 1]);
        const double wE = east_end ? w[k] : (FE > 0.0 ? w[k] : w[k + 1]);
        const double wW = west_end ? w[k] : (FW > 0.0 ? w[kw] : w[k]);
        const double hin = 0.5 * (ei[k + 1] + ei[k + 2]);
        const double hbn = 0.5 * (eb[k + 1] + eb[k + 2]);
        const double hsn = 0.5 * (es[k + 1] + es[k + 2]);
        const double m = area * hin * w[k] - dt / c->dx * (FE * wE - FW * wW);
        const double hw = a * hbn * wb[k] + bw * m / area;
        wo[k] = hw * desing(hsn, 1.0, c->delta);
    }
    if (per) wo[n] = wo[0];
    free(eb); free(ei); free(es);
}

/* dry_zero = 1: dry cells carry no discharge, q = 0 where h <= hdry at the end of each
 * stage (the premise of App. B A.2, q = w = 0 where the depth vanishes, imposed).
 * dry_zero = 0 is the second step as Sec. 4.5 states it, with no special treatment and no
 * truncation at wet/dry fronts. */
static void dry_discharge_1d(const or_cfg *c, const double *h, double *q)
{
    if (!c->dry_zero) return;
    for (int i = 0; i < c->nx; ++i)
        if (h[i] <= c->hdry) q[i] = 0.0;
}

/* One stage of the TVD-RK2 method in Shu-Osher form (Sec. 4.3 and Sec. 6: "steps 1-4
 * twice"): the hyperbolic update of (h_in, q_in) (Eqs. 18-22, friction, clamp) is combined
 * as U* = a U_base + b U**, w* = a w_base + b w_in, then breaking terms and the pressure
 * projection of Eq. (28) are applied with the effective step b dt.  Stage 1: a = 0, b = 1;
 * stage 2: a = b = 1/2.  (Reading: projecting the combination keeps U^{n+1} on the
 * discrete constraint; projecting the second stage before averaging leaves U^{n+1} off it
 * by O(dt^2) on nonlinear waves.) */
static int stage1d(const or_cfg *c, const double *H, const double *hb, const double *qb,
                   const double *wb, const double *h, const double *q, const double *w,
                   double a, double bw, double *p, double dt, double *ho, double *qo,
                   double *wo)
{
    const int n = c->nx, ne = n + 2 * G1;
    const double dx = c->dx;
    double *Fm = c->w_transport ? calloc(n + 1, sizeof(double)) : NULL;
    int clamped = hyp1d(c, H, h, q, dt, ho, qo, Fm);
    for (int i = 0; i < n; ++i) {
        ho[i] = a * hb[i] + bw * ho[i];
        qo[i] = a * qb[i] + bw * qo[i];
    }
    if (c->w_transport) {
        wtransport1d(c, hb, wb, h, w, Fm, ho, a, bw, dt, wo);
        free(Fm);
    } else {
        for (int k = 0; k <= n; ++k) wo[k] = a * wb[k] + bw * w[k];
    }
    const double de = bw * dt;                   /* effective projection step */
    if (c->breaking) breaking1d(c, H, ho, qo, wo, de);
    if (!c->nonhydro) {
        for (int k = 0; k <= n; ++k) p[k] = 0.0;
        dry_discharge_1d(c, ho, qo);
        return clamped;
    }
    or1d_nh_solve(c, H, ho, qo, wo, de, p);

    /* Correction, Eq. (28): q += de T_NH(p) (Eq. 26), w += de p / h (desingularised). */
    double *he = calloc(ne, sizeof(double)), *se = calloc(ne, sizeof(double));
    double *xi = calloc(ne, sizeof(double));
    nh1d_fields(c, H, ho, he, se, xi);
    for (int i = 0; i < n; ++i) {
        int e = i + G1;
        double pi = 0.5 * (p[i + 1] + p[i]), px = (p[i + 1] - p[i]) / dx;
        double T = -0.5 * (he[e] * px + pi * xi[e] / dx);
        qo[i] += de * T;
    }
    for (int k = 0; k <= n; ++k) {
        double hn = 0.5 * (he[k + 1] + he[k + 2]);
        wo[k] += de * p[k] * desing(hn, 1.0, c->delta);
    }
    if (periodic1d(c)) wo[n] = wo[0];
    dry_discharge_1d(c, ho, qo);
    free(he); free(se); free(xi);
    return clamped;
}

/* Second-order TVD Runge-Kutta step (Sec. 4.3; Shu-Osher): U1 = P(U^n + dt L(U^n)),
 * U^{n+1} = P_{dt/2}((U^n + U1 + dt L(U1)) / 2); p^{n+1} is the second projection's. */
int or1d_step(const or_cfg *c, const double *H, double *h, double *q, double *w, double *p,
              double dt, or_stats *st)
{
    const int n = c->nx;
    double *h1 = malloc(n * sizeof(double)), *q1 = malloc(n * sizeof(double));
    double *w1 = malloc((n + 1) * sizeof(double));
    double *h2 = malloc(n * sizeof(double)), *q2 = malloc(n * sizeof(double));
    double *w2 = malloc((n + 1) * sizeof(double));
    int cl = stage1d(c, H, h, q, w, h, q, w, 0.0, 1.0, p, dt, h1, q1, w1);
    cl += stage1d(c, H, h, q, w, h1, q1, w1, 0.5, 0.5, p, dt, h2, q2, w2);
    memcpy(h, h2, n * sizeof(double));
    memcpy(q, q2, n * sizeof(double));
    memcpy(w, w2, (n + 1) * sizeof(double));
    if (st) { st->iters[0] = st->iters[1] = 1; st->resid[0] = st->resid[1] = 0.0; st->clamped = cl; }
    free(h1); free(q1); free(w1); free(h2); free(q2); free(w2);
    return 0;
}

long long or1d_run(const or_cfg *c, const double *H, double *h, double *q, double *w,
                   double *p, double t_end, long long max_steps, double fixed_dt, double *t_out)
{
    double t = 0.0;
    long long s = 0;
    while (s < max_steps) {
        if (t_end > 0.0 && t >= t_end) break;
        double dt = fixed_dt > 0.0 ? fixed_dt : or1d_cfl_dt(c, H, h, q);
        if (!(dt > 0.0)) break;
        if (t_end > 0.0 && t + dt > t_end) dt = t_end - t;
        or1d_step(c, H, h, q, w, p, dt, NULL);
        if (c->relax[0] > 0.0 || c->relax[1] > 0.0)
            or1d_relax(c, H, h, q, w, p, NULL, NULL, NULL, NULL);
        t += dt;
        ++s;
    }
    if (t_out) *t_out = t;
    return s;
}

/* ------------------------------------------------------------------------- */
/* 2D (Sec. 5, App. A)                                                       */
/* ------------------------------------------------------------------------- */

/* Extended cell arrays: (nx + 4) x (ny + 4), cell (i, j) at CE(i, j).  Extended node
 * arrays: (nx + 3) x (ny + 3), node (I, J) at NE(I, J). */
#define CE(i, j) ((size_t)((j) + 2) * (size_t)(nx + 4) + (size_t)((i) + 2))
#define NE(I, J) ((size_t)((J) + 1) * (size_t)(nx + 3) + (size_t)((I) + 1))
#define CI(i, j) ((size_t)(j) * (size_t)nx + (size_t)(i))
#define NI(I, J) ((size_t)(J) * (size_t)(nx + 1) + (size_t)(I))

/* Ghost cells of an extended 2D cell array: first the two ghost columns of the interior
 * rows, then the two ghost rows over every column (so corners reflect twice).  px / py:
 * parity (+1 / -1) under reflection across x = const / y = const walls. */
static void ghost2d(const or_cfg *c, double *v, double px, double py)
{
    const int nx = c->nx, ny = c->ny;
#pragma omp parallel for
    for (int j = 0; j < ny; ++j) {
        /* first ghost layer, then second (handles nx == 1) */
        v[CE(-1, j)] = c->bc[0] == OR_WALL ? px * v[CE(0, j)] : v[CE(0, j)];
        v[CE(nx, j)] = c->bc[1] == OR_WALL ? px * v[CE(nx - 1, j)] : v[CE(nx - 1, j)];
        v[CE(-2, j)] = c->bc[0] == OR_WALL ? px * v[CE(1, j)] : v[CE(0, j)];
        v[CE(nx + 1, j)] = c->bc[1] == OR_WALL ? px * v[CE(nx - 2, j)] : v[CE(nx - 1, j)];
    }
#pragma omp parallel for
    for (int i = -2; i < nx + 2; ++i) {
        v[CE(i, -1)] = c->bc[2] == OR_WALL ? py * v[CE(i, 0)] : v[CE(i, 0)];
        v[CE(i, ny)] = c->bc[3] == OR_WALL ? py * v[CE(i, ny - 1)] : v[CE(i, ny - 1)];
        v[CE(i, -2)] = c->bc[2] == OR_WALL ? py * v[CE(i, 1)] : v[CE(i, 0)];
        v[CE(i, ny + 1)] = c->bc[3] == OR_WALL ? py * v[CE(i, ny - 2)] : v[CE(i, ny - 1)];
    }
}

/* Ghost pressure nodes: the outside neighbour of a boundary node mirrors the inside one
 * (walls and outflow alike). */
static void ghostnodes2d(const or_cfg *c, double *pe)
{
    const int nx = c->nx, ny = c->ny;
    for (int J = 0; J <= ny; ++J) {
        pe[NE(-1, J)] = pe[NE(1, J)];
        pe[NE(nx + 1, J)] = pe[NE(nx - 1, J)];
    }
    for (int I = -1; I <= nx + 1; ++I) {
        pe[NE(I, -1)] = pe[NE(I, 1)];
        pe[NE(I, ny + 1)] = pe[NE(I, ny - 1)];
    }
}

static double *ext_cells(const or_cfg *c)
{
    return calloc((size_t)(c->nx + 4) * (size_t)(c->ny + 4), sizeof(double));
}
static double *ext_nodes(const or_cfg *c)
{
    return calloc((size_t)(c->nx + 3) * (size_t)(c->ny + 3), sizeof(double));
}
static void load_cells(const or_cfg *c, const double *src, double *dst)
{
    const int nx = c->nx, ny = c->ny;
#pragma omp parallel for
    for (int j = 0; j < ny; ++j)
        for (int i = 0; i < nx; ++i) dst[CE(i, j)] = src[CI(i, j)];
}

double or2d_cfl_dt(const or_cfg *c, const double *H, const double *h, const double *q1,
                   const double *q2)
{
    (void)H;
    double lmax = 0.0;
    size_t n = (size_t)c->nx * (size_t)c->ny;
#pragma omp parallel for reduction(max : lmax)
    for (size_t k = 0; k < n; ++k) {
        double u = desing(h[k], q1[k], c->delta), v = desing(h[k], q2[k], c->delta);
        double cc = sqrt(c->g * h[k]);
        double l = (fabs(u) + cc) / c->dx + (fabs(v) + cc) / c->dy;
        if (l > lmax) lmax = l;
    }
    return lmax > 0.0 ? c->cfl / lmax : 0.0;
}

/* Hyperbolic step of Sec. 5 / Eq. (30): second-order PVM-HLL with MUSCL-minmod, the
 * cell integral by the midpoint rule, then friction and the depth clamp.  FX ([ny][nx+1])
 * and FY ([ny+1][nx]), or NULL: the mass flux of every x / y face, F_h(U^-) + D^-_h, seen
 * from its west / south cell. */
static int hyp2d(const or_cfg *c, const double *H, const double *h, const double *q1,
                 const double *q2, double dt, double *ho, double *q1o, double *q2o,
                 double *FX, double *FY)
{
    const int nx = c->nx, ny = c->ny;
    const double dx = c->dx, dy = c->dy, g = c->g;
    int clamped = 0;
    double *he = ext_cells(c), *He = ext_cells(c), *ae = ext_cells(c), *be = ext_cells(c);
    double *ee = ext_cells(c), *ue = ext_cells(c), *ve = ext_cells(c);
    load_cells(c, h, he); load_cells(c, H, He); load_cells(c, q1, ae); load_cells(c, q2, be);
    ghost2d(c, he, 1.0, 1.0); ghost2d(c, He, 1.0, 1.0);
    ghost2d(c, ae, -1.0, 1.0); ghost2d(c, be, 1.0, -1.0);
    size_t ne = (size_t)(nx + 4) * (ny + 4);
#pragma omp parallel for
    for (size_t k = 0; k < ne; ++k) {
        ee[k] = he[k] - He[k];
        ue[k] = desing(he[k], ae[k], c->delta);
        ve[k] = desing(he[k], be[k], c->delta);
    }

    /* reconstructed edge values: [field][cell]; fields h, eta, u, v */
    double *xE[4], *xW[4], *yN[4], *yS[4];
    for (int f = 0; f < 4; ++f) {
        xE[f] = ext_cells(c); xW[f] = ext_cells(c); yN[f] = ext_cells(c); yS[f] = ext_cells(c);
    }
    double *fld[4] = {he, ee, ue, ve};

    /* x-direction reconstruction for cells i = -1 .. nx of interior rows */
#pragma omp parallel for
    for (int j = 0; j < ny; ++j)
        for (int i = -1; i <= nx; ++i) {
            int dry = he[CE(i - 1, j)] <= c->hdry || he[CE(i, j)] <= c->hdry ||
                      he[CE(i + 1, j)] <= c->hdry;
            for (int f = 0; f < 4; ++f) {
                double *v = fld[f];
                double s = minmod(v[CE(i, j)] - v[CE(i - 1, j)], v[CE(i + 1, j)] - v[CE(i, j)]);
                if (f == 1 && dry) s = 0.0;
                xE[f][CE(i, j)] = v[CE(i, j)] + 0.5 * s;
                xW[f][CE(i, j)] = v[CE(i, j)] - 0.5 * s;
            }
        }
    /* y-direction reconstruction for cells j = -1 .. ny of interior columns */
#pragma omp parallel for
    for (int j = -1; j <= ny; ++j)
        for (int i = 0; i < nx; ++i) {
            int dry = he[CE(i, j - 1)] <= c->hdry || he[CE(i, j)] <= c->hdry ||
                      he[CE(i, j + 1)] <= c->hdry;
            for (int f = 0; f < 4; ++f) {
                double *v = fld[f];
                double s = minmod(v[CE(i, j)] - v[CE(i, j - 1)], v[CE(i, j + 1)] - v[CE(i, j)]);
                if (f == 1 && dry) s = 0.0;
                yN[f][CE(i, j)] = v[CE(i, j)] + 0.5 * s;
                yS[f][CE(i, j)] = v[CE(i, j)] - 0.5 * s;
            }
        }

    /* x faces (I, j), I = 0 .. nx: normal = x (q1), tangential = y (q2) */
    double *DmX = calloc(3 * (size_t)(nx + 1) * ny, sizeof(double));
    double *DpX = calloc(3 * (size_t)(nx + 1) * ny, sizeof(double));
#pragma omp parallel for
    for (int j = 0; j < ny; ++j)
        for (int I = 0; I <= nx; ++I) {
            size_t L = CE(I - 1, j), R = CE(I, j), f = 3 * ((size_t)j * (nx + 1) + I);
            pvm_face(g, c->hdry, xE[0][L], xE[1][L], xE[2][L], xE[3][L],
                     xW[0][R], xW[1][R], xW[2][R], xW[3][R], DmX + f, DpX + f);
            if (FX) FX[(size_t)j * (nx + 1) + I] = xE[0][L] * xE[2][L] + DmX[f];
        }
    /* y faces (i, J), J = 0 .. ny: normal = y (q2), tangential = x (q1) */
    double *DmY = calloc(3 * (size_t)nx * (ny + 1), sizeof(double));
    double *DpY = calloc(3 * (size_t)nx * (ny + 1), sizeof(double));
#pragma omp parallel for
    for (int J = 0; J <= ny; ++J)
        for (int i = 0; i < nx; ++i) {
            size_t L = CE(i, J - 1), R = CE(i, J), f = 3 * ((size_t)J * nx + i);
            pvm_face(g, c->hdry, yN[0][L], yN[1][L], yN[3][L], yN[2][L],
                     yS[0][R], yS[1][R], yS[3][R], yS[2][R], DmY + f, DpY + f);
            if (FY) FY[(size_t)J * nx + i] = yN[0][L] * yN[3][L] + DmY[f];
        }

    /* cell update, Eq. (30) */
#pragma omp parallel for reduction(+ : clamped)
    for (int j = 0; j < ny; ++j)
        for (int i = 0; i < nx; ++i) {
            size_t e = CE(i, j);
            double hEx = xE[0][e], hWx = xW[0][e], uEx = xE[2][e], uWx = xW[2][e];
            double vEx = xE[3][e], vWx = xW[3][e];
            double hNy = yN[0][e], hSy = yS[0][e], uNy = yN[2][e], uSy = yS[2][e];
            double vNy = yN[3][e], vSy = yS[3][e];
            /* inner-cell terms: convective flux difference + g h (eta^+ - eta^-) */
            double Ix0 = hEx * uEx - hWx * uWx;
            double Ix1 = hEx * uEx * uEx - hWx * uWx * uWx + g * he[e] * (xE[1][e] - xW[1][e]);
            double Ix2 = hEx * uEx * vEx - hWx * uWx * vWx;
            double Iy0 = hNy * vNy - hSy * vSy;
            double Iy1 = hNy * uNy * vNy - hSy * uSy * vSy;
            double Iy2 = hNy * vNy * vNy - hSy * vSy * vSy + g * he[e] * (yN[1][e] - yS[1][e]);
            const double *mx = DmX + 3 * ((size_t)j * (nx + 1) + i + 1);   /* east face D^- */
            const double *px = DpX + 3 * ((size_t)j * (nx + 1) + i);       /* west face D^+ */
            const double *my = DmY + 3 * ((size_t)(j + 1) * nx + i);       /* north face D^- */
            const double *py = DpY + 3 * ((size_t)j * nx + i);             /* south face D^+ */
            double hn = he[e] - dt / dx * (mx[0] + px[0] + Ix0) - dt / dy * (my[0] + py[0] + Iy0);
            double an = ae[e] - dt / dx * (mx[1] + px[1] + Ix1) - dt / dy * (my[2] + py[2] + Iy1);
            double bn = be[e] - dt / dx * (mx[2] + px[2] + Ix2) - dt / dy * (my[1] + py[1] + Iy2);
            if (c->manning > 0.0 && hn > 0.0) {
                double u = desing(hn, an, c->delta), v = desing(hn, bn, c->delta);
                double hd = hn > c->delta ? hn : c->delta;
                double fr = 1.0 + dt * g * c->manning * c->manning * sqrt(u * u + v * v)
                                / pow(hd, 4.0 / 3.0);
                an /= fr; bn /= fr;
            }
            if (hn < 0.0) { hn = 0.0; an = 0.0; bn = 0.0; ++clamped; }
            ho[CI(i, j)] = hn; q1o[CI(i, j)] = an; q2o[CI(i, j)] = bn;
        }
    for (int f = 0; f < 4; ++f) { free(xE[f]); free(xW[f]); free(yN[f]); free(yS[f]); }
    free(DmX); free(DpX); free(DmY); free(DpY);
    free(he); free(He); free(ae); free(be); free(ee); free(ue); free(ve);
    return clamped;
}

int or2d_hyperbolic(const or_cfg *c, const double *H, const double *h, const double *q1,
                    const double *q2, double dt, double *ho, double *q1o, double *q2o)
{
    return hyp2d(c, H, h, q1, q2, dt, ho, q1o, q2o, NULL, NULL);
}

/* 2D breaking terms: Sec. 3 with q_x -> div q, u_x -> div u (reading).  Cells: q +=
 * dt 2 nu (div u) grad H (centred); nodes: w += dt 2 nu (div u) / h from the four cells. */
static void breaking2d(const or_cfg *c, const double *H, const double *h, double *q1,
                       double *q2, double *w, double dt)
{
    const int nx = c->nx, ny = c->ny;
    const double dx = c->dx, dy = c->dy;
    double *he = ext_cells(c), *He = ext_cells(c), *ae = ext_cells(c), *be = ext_cells(c);
    double *ue = ext_cells(c), *ve = ext_cells(c);
    load_cells(c, h, he); load_cells(c, H, He); load_cells(c, q1, ae); load_cells(c, q2, be);
    ghost2d(c, he, 1.0, 1.0); ghost2d(c, He, 1.0, 1.0);
    ghost2d(c, ae, -1.0, 1.0); ghost2d(c, be, 1.0, -1.0);
    size_t ne = (size_t)(nx + 4) * (ny + 4);
    for (size_t k = 0; k < ne; ++k) {
        ue[k] = desing(he[k], ae[k], c->delta);
        ve[k] = desing(he[k], be[k], c->delta);
    }
#pragma omp parallel for
    for (int j = 0; j < ny; ++j)
        for (int i = 0; i < nx; ++i) {
            double dq = (ae[CE(i + 1, j)] - ae[CE(i - 1, j)]) / (2 * dx)
                      + (be[CE(i, j + 1)] - be[CE(i, j - 1)]) / (2 * dy);
            double du = (ue[CE(i + 1, j)] - ue[CE(i - 1, j)]) / (2 * dx)
                      + (ve[CE(i, j + 1)] - ve[CE(i, j - 1)]) / (2 * dy);
            double Hx = (He[CE(i + 1, j)] - He[CE(i - 1, j)]) / (2 * dx);
            double Hy = (He[CE(i, j + 1)] - He[CE(i, j - 1)]) / (2 * dy);
            double nu = breaking_nu(c, he[CE(i, j)], dq);
            q1[CI(i, j)] += dt * 2.0 * nu * du * Hx;
            q2[CI(i, j)] += dt * 2.0 * nu * du * Hy;
        }
#pragma omp parallel for
    for (int J = 0; J <= ny; ++J)
        for (int I = 0; I <= nx; ++I) {
            size_t a = CE(I - 1, J - 1), b = CE(I, J - 1), d = CE(I - 1, J), e = CE(I, J);
            double hc = 0.25 * (he[a] + he[b] + he[d] + he[e]);
            double dq = (ae[b] + ae[e] - ae[a] - ae[d]) / (2 * dx)
                      + (be[d] + be[e] - be[a] - be[b]) / (2 * dy);
            double du = (ue[b] + ue[e] - ue[a] - ue[d]) / (2 * dx)
                      + (ve[d] + ve[e] - ve[a] - ve[b]) / (2 * dy);
            double nu = breaking_nu(c, hc, dq);
            w[NI(I, J)] += dt * 2.0 * nu * du * desing(hc, 1.0, c->delta);
        }
    free(he); free(He); free(ae); free(be); free(ue); free(ve);
}

/* Per-cell fields of the non-hydrostatic step on the extended grid: h, s = 2 eta - h and
 * the centred differences X = dx (2 eta - h)_x, Y = dy (2 eta - h)_y (App. A.2). */
typedef struct { double *h, *s, *X, *Y; } nh2d_cells;

static nh2d_cells nh2d_fields(const or_cfg *c, const double *H, const double *h)
{
    const int nx = c->nx, ny = c->ny;
    nh2d_cells f = {ext_cells(c), ext_cells(c), ext_cells(c), ext_cells(c)};
    double *He = ext_cells(c);
    load_cells(c, h, f.h); load_cells(c, H, He);
    ghost2d(c, f.h, 1.0, 1.0); ghost2d(c, He, 1.0, 1.0);
    size_t ne = (size_t)(nx + 4) * (ny + 4);
#pragma omp parallel for
    for (size_t k = 0; k < ne; ++k) f.s[k] = 2.0 * (f.h[k] - He[k]) - f.h[k];
#pragma omp parallel for
    for (int j = -1; j <= ny; ++j)
        for (int i = -1; i <= nx; ++i) {
            f.X[CE(i, j)] = 0.5 * (f.s[CE(i + 1, j)] - f.s[CE(i - 1, j)]);
            f.Y[CE(i, j)] = 0.5 * (f.s[CE(i, j + 1)] - f.s[CE(i, j - 1)]);
        }
    free(He);
    return f;
}
static void nh2d_free(nh2d_cells *f) { free(f->h); free(f->s); free(f->X); free(f->Y); }

/* dt times the edge approximations of T^Hor_N, T^Hor_S, T^Ver_E, T^Ver_W of App. A.2 for
 * cells -1 .. nx, -1 .. ny, from the extended node pressure pe. */
static void half_T(const or_cfg *c, const nh2d_cells *f, const double *pe, double dt,
                   double *TN, double *TS, double *TE, double *TW)
{
    const int nx = c->nx, ny = c->ny;
    const double dx = c->dx, dy = c->dy;
#pragma omp parallel for
    for (int j = -1; j <= ny; ++j)
        for (int i = -1; i <= nx; ++i) {
            size_t e = CE(i, j);
            double h = f->h[e], X = f->X[e], Y = f->Y[e];
            /* nodes of cell (i, j): SW (i, j), SE (i+1, j), NW (i, j+1), NE (i+1, j+1) */
            double pSW = pe[NE(i, j)], pSE = pe[NE(i + 1, j)];
            double pNW = pe[NE(i, j + 1)], pNE = pe[NE(i + 1, j + 1)];
            /* T^Hor_N = -1/2 h (p_NE - p_NW)/dx - 1/2 (p_NE + p_NW)/2 * X/dx, etc. */
            TN[e] = dt * (-0.5 * h * (pNE - pNW) / dx - 0.5 * 0.5 * (pNE + pNW) * X / dx);
            TS[e] = dt * (-0.5 * h * (pSE - pSW) / dx - 0.5 * 0.5 * (pSE + pSW) * X / dx);
            TE[e] = dt * (-0.5 * h * (pNE - pSE) / dy - 0.5 * 0.5 * (pNE + pSE) * Y / dy);
            TW[e] = dt * (-0.5 * h * (pNW - pSW) / dy - 0.5 * 0.5 * (pNW + pSW) * Y / dy);
        }
}

/* The divergence constraint B at every node, Eqs. (37)-(40), with the edge discharges of
 * Eq. (41): q_{1,E} = (q1_e + q1_b)/2 + (dt T^Hor_S(e) + dt T^Hor_N(b))/2, and so on.
 * Q1, Q2 are (extended) cell discharges, T* are dt times the half corrections (NULL: 0),
 * twohw is the 2 h w term at each node. */
static void B_nodes(const or_cfg *c, const nh2d_cells *f, const double *Q1, const double *Q2,
                    const double *TN, const double *TS, const double *TE, const double *TW,
                    const double *twohw, double *B)
{
    const int nx = c->nx, ny = c->ny;
    const double dx = c->dx, dy = c->dy;
#pragma omp parallel for
    for (int J = 0; J <= ny; ++J)
        for (int I = 0; I <= nx; ++I) {
            size_t a = CE(I - 1, J - 1), b = CE(I, J - 1), d = CE(I - 1, J), e = CE(I, J);
            double q1E = 0.5 * (Q1[e] + Q1[b]), q1W = 0.5 * (Q1[d] + Q1[a]);
            double q2N = 0.5 * (Q2[e] + Q2[d]), q2S = 0.5 * (Q2[b] + Q2[a]);
            if (TN) {
                q1E += 0.5 * (TS[e] + TN[b]);
                q1W += 0.5 * (TS[d] + TN[a]);
                q2N += 0.5 * (TW[e] + TE[d]);
                q2S += 0.5 * (TW[b] + TE[a]);
            }
            double sE = 0.5 * (f->s[e] + f->s[b]), sW = 0.5 * (f->s[d] + f->s[a]);
            double sN = 0.5 * (f->s[e] + f->s[d]), sS = 0.5 * (f->s[b] + f->s[a]);
            double hc = 0.25 * (f->h[a] + f->h[b] + f->h[d] + f->h[e]);        /* Eq. (38) */
            double divQ = (q1E - q1W) / dx + (q2N - q2S) / dy;                 /* Eq. (39) */
            double Qx = 0.5 * (q1E + q1W), Qy = 0.5 * (q2N + q2S);
            double gx = (sE - sW) / dx, gy = (sN - sS) / dy;                   /* Eq. (40) */
            B[NI(I, J)] = hc * divQ - (Qx * gx + Qy * gy) + twohw[NI(I, J)];  /* Eq. (37) */
        }
}

int or2d_rhs(const or_cfg *c, const double *H, const double *h, const double *q1,
             const double *q2, const double *w, double dt, double *rhs)
{
    const int nx = c->nx, ny = c->ny;
    const size_t nn = (size_t)(nx + 1) * (ny + 1);
    nh2d_cells f = nh2d_fields(c, H, h);
    double *Q1 = ext_cells(c), *Q2 = ext_cells(c), *tw = calloc(nn, sizeof(double));
    load_cells(c, q1, Q1); load_cells(c, q2, Q2);
    ghost2d(c, Q1, -1.0, 1.0); ghost2d(c, Q2, 1.0, -1.0);
#pragma omp parallel for
    for (int J = 0; J <= ny; ++J)
        for (int I = 0; I <= nx; ++I) {
            double hc = 0.25 * (f.h[CE(I - 1, J - 1)] + f.h[CE(I, J - 1)] + f.h[CE(I - 1, J)]
                                + f.h[CE(I, J)]);
            tw[NI(I, J)] = 2.0 * hc * w[NI(I, J)];
        }
    B_nodes(c, &f, Q1, Q2, NULL, NULL, NULL, NULL, tw, rhs);
    double sc = -8.0 * c->dx * c->dy / dt;
#pragma omp parallel for
    for (size_t k = 0; k < nn; ++k) rhs[k] *= sc;
    free(Q1); free(Q2); free(tw);
    nh2d_free(&f);
    return 0;
}

/* Linear part of the affine map p -> B(q* + dt T(p), w* + dt p / h), scaled by
 * 8 dx dy / dt: the pentadiagonal matrix of Sec. 5, built without expanding coefficients. */
typedef struct { double *pe, *TN, *TS, *TE, *TW, *Z, *tw; } mwork;

static mwork mwork_new(const or_cfg *c)
{
    size_t nn = (size_t)(c->nx + 1) * (c->ny + 1);
    mwork m = {ext_nodes(c), ext_cells(c), ext_cells(c), ext_cells(c), ext_cells(c),
               ext_cells(c), calloc(nn, sizeof(double))};
    return m;
}
static void mwork_free(mwork *m)
{
    free(m->pe); free(m->TN); free(m->TS); free(m->TE); free(m->TW); free(m->Z); free(m->tw);
}

static void apply_M_f(const or_cfg *c, const nh2d_cells *f, const double *p, double dt,
                      double *out, mwork *m)
{
    const int nx = c->nx, ny = c->ny;
    const size_t nn = (size_t)(nx + 1) * (ny + 1);
#pragma omp parallel for
    for (int J = 0; J <= ny; ++J)
        for (int I = 0; I <= nx; ++I) m->pe[NE(I, J)] = p[NI(I, J)];
    ghostnodes2d(c, m->pe);
    half_T(c, f, m->pe, dt, m->TN, m->TS, m->TE, m->TW);
#pragma omp parallel for
    for (size_t k = 0; k < nn; ++k) m->tw[k] = 2.0 * dt * p[k];   /* 2 h (dt p / h) */
    B_nodes(c, f, m->Z, m->Z, m->TN, m->TS, m->TE, m->TW, m->tw, out);
    double sc = 8.0 * c->dx * c->dy / dt;
#pragma omp parallel for
    for (size_t k = 0; k < nn; ++k) out[k] *= sc;
}

int or2d_apply_M(const or_cfg *c, const double *H, const double *h, const double *p,
                 double dt, double *out)
{
    nh2d_cells f = nh2d_fields(c, H, h);
    mwork m = mwork_new(c);
    apply_M_f(c, &f, p, dt, out, &m);
    mwork_free(&m);
    nh2d_free(&f);
    return 0;
}

static double dot(size_t n, const double *a, const double *b)
{
    double s = 0.0;
    for (size_t k = 0; k < n; ++k) s += a[k] * b[k];
    return s;
}

/* BiCGStab (van der Vorst) on M p = rhs, warm-started from p; restarts from the true
 * residual until ||rhs - M p|| <= tol ||rhs|| or max_iter.  rhs == 0 gives p = 0. */
static int solve_f(const or_cfg *c, const nh2d_cells *f, const double *b, double dt,
                   double *x, int *iters, double *resid)
{
    const size_t n = (size_t)(c->nx + 1) * (c->ny + 1);
    double bn = sqrt(dot(n, b, b));
    *iters = 0; *resid = 0.0;
    if (bn == 0.0) { for (size_t k = 0; k < n; ++k) x[k] = 0.0; return 0; }
    mwork m = mwork_new(c);
    double *r = malloc(n * sizeof(double)), *rh = malloc(n * sizeof(double));
    double *pv = malloc(n * sizeof(double)), *v = malloc(n * sizeof(double));
    double *s = malloc(n * sizeof(double)), *t = malloc(n * sizeof(double));
    int it = 0, status = -1;
    for (int restart = 0; restart < 20 && it < c->max_iter; ++restart) {
        apply_M_f(c, f, x, dt, r, &m);
#pragma omp parallel for
        for (size_t k = 0; k < n; ++k) r[k] = b[k] - r[k];
        double rn = sqrt(dot(n, r, r));
        *resid = rn / bn;
        if (rn <= c->tol * bn) { status = 0; break; }
        memcpy(rh, r, n * sizeof(double));
        double rho = 1.0, alpha = 1.0, omega = 1.0;
#pragma omp parallel for
        for (size_t k = 0; k < n; ++k) { pv[k] = 0.0; v[k] = 0.0; }
        while (it < c->max_iter) {
            ++it;
            double rho1 = dot(n, rh, r);
            if (rho1 == 0.0) break;
            double beta = (rho1 / rho) * (alpha / omega);
#pragma omp parallel for
            for (size_t k = 0; k < n; ++k) pv[k] = r[k] + beta * (pv[k] - omega * v[k]);
            apply_M_f(c, f, pv, dt, v, &m);
            double rv = dot(n, rh, v);
            if (rv == 0.0) break;
            alpha = rho1 / rv;
#pragma omp parallel for
            for (size_t k = 0; k < n; ++k) s[k] = r[k] - alpha * v[k];
            if (sqrt(dot(n, s, s)) <= 0.1 * c->tol * bn) {
#pragma omp parallel for
                for (size_t k = 0; k < n; ++k) x[k] += alpha * pv[k];
                break;
            }
            apply_M_f(c, f, s, dt, t, &m);
            double tt = dot(n, t, t);
            omega = tt > 0.0 ? dot(n, t, s) / tt : 0.0;
#pragma omp parallel for
            for (size_t k = 0; k < n; ++k) {
                x[k] += alpha * pv[k] + omega * s[k];
                r[k] = s[k] - omega * t[k];
            }
            rho = rho1;
            if (sqrt(dot(n, r, r)) <= 0.1 * c->tol * bn || omega == 0.0) break;
        }
    }
    if (status != 0) {
        apply_M_f(c, f, x, dt, r, &m);
#pragma omp parallel for
        for (size_t k = 0; k < n; ++k) r[k] = b[k] - r[k];
        *resid = sqrt(dot(n, r, r)) / bn;
        status = *resid <= c->tol ? 0 : -1;
    }
    *iters = it;
    free(r); free(rh); free(pv); free(v); free(s); free(t);
    mwork_free(&m);
    return status;
}

int or2d_solve(const or_cfg *c, const double *H, const double *h, const double *rhs,
               double dt, double *p, int *iters, double *resid)
{
    nh2d_cells f = nh2d_fields(c, H, h);
    int st = solve_f(c, &f, rhs, dt, p, iters, resid);
    nh2d_free(&f);
    return st;
}

/* Node depth: the mean of the four cells around node (I, J) of an extended, ghosted cell
 * array (at a wall or outflow side the mean of the cells inside). */
static double node_depth2d(const or_cfg *c, const double *e, int I, int J)
{
    const int nx = c->nx;
    return 0.25 * (e[CE(I - 1, J - 1)] + e[CE(I, J - 1)] + e[CE(I - 1, J)] + e[CE(I, J)]);
}

/* 2D form of wtransport1d (energy-consistent w equation (hw)_t + div(hw u) = p): node
 * (I, J) owns the dual cell [x_I - dx/2, x_I + dx/2] x [y_J - dy/2, y_J + dy/2] clipped to
 * the domain (area fraction 1, 1/2 or 1/4 of dx dy), a quarter of each cell around it.  Its
 * east face runs along the centre line of the cells (I, J-1), (I, J) (those inside the
 * grid), through half of each; the x mass flux across a cell's centre line is the mean of
 * its two x faces' fluxes.  On the domain boundary the dual face is the boundary face. */
static void wtransport2d(const or_cfg *c, const double *hb, const double *wb,
                         const double *h, const double *w, const double *FX,
                         const double *FY, const double *hs, double a, double bw, double dt,
                         double *wo)
{
    const int nx = c->nx, ny = c->ny;
    double *eb = ext_cells(c), *ei = ext_cells(c), *es = ext_cells(c);
    load_cells(c, hb, eb); load_cells(c, h, ei); load_cells(c, hs, es);
    ghost2d(c, eb, 1.0, 1.0); ghost2d(c, ei, 1.0, 1.0); ghost2d(c, es, 1.0, 1.0);
#pragma omp parallel for
    for (int J = 0; J <= ny; ++J)
        for (int I = 0; I <= nx; ++I) {
            const double ax = (I == 0 || I == nx) ? 0.5 : 1.0;
            const double ay = (J == 0 || J == ny) ? 0.5 : 1.0;
            /* cs[d]: x-face fluxes of face column I-1+d summed over the rows J-1, J inside;
             * rs[d]: y-face fluxes of face row J-1+d summed over the columns I-1, I inside */
            double cs[3] = {0.0, 0.0, 0.0}, rs[3] = {0.0, 0.0, 0.0};
            for (int d = 0; d < 3; ++d) {
                const int If = I - 1 + d, Jf = J - 1 + d;
                if (If >= 0 && If <= nx)
                    for (int j = J - 1; j <= J; ++j)
                        if (j >= 0 && j < ny) cs[d] += FX[(size_t)j * (nx + 1) + If];
                if (Jf >= 0 && Jf <= ny)
                    for (int i = I - 1; i <= I; ++i)
                        if (i >= 0 && i < nx) rs[d] += FY[(size_t)Jf * nx + i];
            }
            const double FE = I == nx ? 0.5 * cs[1] : 0.25 * (cs[1] + cs[2]);
            const double FW = I == 0 ? 0.5 * cs[1] : 0.25 * (cs[0] + cs[1]);
            const double FN = J == ny ? 0.5 * rs[1] : 0.25 * (rs[1] + rs[2]);
            const double FS = J == 0 ? 0.5 * rs[1] : 0.25 * (rs[0] + rs[1]);
            const double wc = w[NI(I, J)];
            const double wE = I == nx ? wc : (FE > 0.0 ? wc : w[NI(I + 1, J)]);
            const double wW = I == 0 ? wc : (FW > 0.0 ? w[NI(I - 1, J)] : wc);
            const double wN = J == ny ? wc : (FN > 0.0 ? wc : w[NI(I, J + 1)]);
            const double wS = J == 0 ? wc : (FS > 0.0 ? w[NI(I, J - 1)] : wc);
            const double area = ax * ay;
            const double m = area * node_depth2d(c, ei, I, J) * wc
                           - dt / c->dx * (FE * wE - FW * wW) - dt / c->dy * (FN * wN - FS * wS);
            const double hw = a * node_depth2d(c, eb, I, J) * wb[NI(I, J)] + bw * m / area;
            wo[NI(I, J)] = hw * desing(node_depth2d(c, es, I, J), 1.0, c->delta);
        }
    free(eb); free(ei); free(es);
}

/* Dry cells carry no discharge (see dry_discharge_1d). */
static void dry_discharge_2d(const or_cfg *c, const double *h, double *q1, double *q2)
{
    if (!c->dry_zero) return;
    size_t n = (size_t)c->nx * c->ny;
#pragma omp parallel for
    for (size_t k = 0; k < n; ++k)
        if (h[k] <= c->hdry) { q1[k] = 0.0; q2[k] = 0.0; }
}

/* One stage of the TVD-RK2 method in Shu-Osher form for App. A (Eq. 41): hyperbolic update
 * of (h, q1, q2) (Eq. 30, friction, clamp), combination U* = a U_base + b U**, w* =
 * a w_base + b w, breaking terms, pressure solve and correction (Eq. 36, w += de p / h_c)
 * with the effective step de = b dt.  Stage 1: a = 0, b = 1; stage 2: a = b = 1/2. */
static int stage2d(const or_cfg *c, const double *H, const double *hb, const double *q1b,
                   const double *q2b, const double *wb, const double *h, const double *q1,
                   const double *q2, const double *w, double a, double bw, double *p,
                   double dt, double *ho, double *q1o, double *q2o, double *wo, int *iters,
                   double *resid)
{
    const int nx = c->nx, ny = c->ny;
    const size_t n = (size_t)nx * ny, nn = (size_t)(nx + 1) * (ny + 1);
    double *FX = NULL, *FY = NULL;
    if (c->w_transport) {
        FX = calloc((size_t)(nx + 1) * ny, sizeof(double));
        FY = calloc((size_t)nx * (ny + 1), sizeof(double));
    }
    int clamped = hyp2d(c, H, h, q1, q2, dt, ho, q1o, q2o, FX, FY);
#pragma omp parallel for
    for (size_t k = 0; k < n; ++k) {
        ho[k] = a * hb[k] + bw * ho[k];
        q1o[k] = a * q1b[k] + bw * q1o[k];
        q2o[k] = a * q2b[k] + bw * q2o[k];
    }
    if (c->w_transport) {
        wtransport2d(c, hb, wb, h, w, FX, FY, ho, a, bw, dt, wo);
        free(FX); free(FY);
    } else {
#pragma omp parallel for
        for (size_t k = 0; k < nn; ++k) wo[k] = a * wb[k] + bw * w[k];
    }
    const double de = bw * dt;
    if (c->breaking) breaking2d(c, H, ho, q1o, q2o, wo, de);
    *iters = 0; *resid = 0.0;
    if (!c->nonhydro) {
        for (size_t k = 0; k < nn; ++k) p[k] = 0.0;
        dry_discharge_2d(c, ho, q1o, q2o);
        return clamped;
    }
    double *rhs = malloc(nn * sizeof(double));
    or2d_rhs(c, H, ho, q1o, q2o, wo, de, rhs);
    nh2d_cells f = nh2d_fields(c, H, ho);
    solve_f(c, &f, rhs, de, p, iters, resid);

    /* correction: q1 += de (T_N + T_S)/2, q2 += de (T_E + T_W)/2 (Eq. 36); w += de p / h_c */
    double *pe = ext_nodes(c), *TN = ext_cells(c), *TS = ext_cells(c);
    double *TE = ext_cells(c), *TW = ext_cells(c);
#pragma omp parallel for
    for (int J = 0; J <= ny; ++J)
        for (int I = 0; I <= nx; ++I) pe[NE(I, J)] = p[NI(I, J)];
    ghostnodes2d(c, pe);
    half_T(c, &f, pe, de, TN, TS, TE, TW);
#pragma omp parallel for
    for (int j = 0; j < ny; ++j)
        for (int i = 0; i < nx; ++i) {
            size_t e = CE(i, j);
            q1o[CI(i, j)] += 0.5 * (TN[e] + TS[e]);
            q2o[CI(i, j)] += 0.5 * (TE[e] + TW[e]);
        }
#pragma omp parallel for
    for (int J = 0; J <= ny; ++J)
        for (int I = 0; I <= nx; ++I) {
            double hc = 0.25 * (f.h[CE(I - 1, J - 1)] + f.h[CE(I, J - 1)] + f.h[CE(I - 1, J)]
                                + f.h[CE(I, J)]);
            wo[NI(I, J)] += de * p[NI(I, J)] * desing(hc, 1.0, c->delta);
        }
    dry_discharge_2d(c, ho, q1o, q2o);
    free(rhs); free(pe); free(TN); free(TS); free(TE); free(TW);
    nh2d_free(&f);
    return clamped;
}

/* Stage 1 of the step (a = 0, b = 1): U1 = P(U^n + dt L(U^n)). */
int or2d_stage(const or_cfg *c, const double *H, const double *h, const double *q1,
               const double *q2, const double *w, double *p, double dt, double *ho,
               double *q1o, double *q2o, double *wo, int *iters, double *resid)
{
    return stage2d(c, H, h, q1, q2, w, h, q1, q2, w, 0.0, 1.0, p, dt, ho, q1o, q2o, wo,
                   iters, resid);
}

/* TVD-RK2 step: U1 = P(U^n + dt L(U^n)), U^{n+1} = P_{dt/2}((U^n + U1 + dt L(U1)) / 2). */
int or2d_step(const or_cfg *c, const double *H, double *h, double *q1, double *q2, double *w,
              double *p, double dt, or_stats *st)
{
    const size_t n = (size_t)c->nx * c->ny, nn = (size_t)(c->nx + 1) * (c->ny + 1);
    double *h1 = malloc(n * sizeof(double)), *a1 = malloc(n * sizeof(double));
    double *b1 = malloc(n * sizeof(double)), *w1 = malloc(nn * sizeof(double));
    double *h2 = malloc(n * sizeof(double)), *a2 = malloc(n * sizeof(double));
    double *b2 = malloc(n * sizeof(double)), *w2 = malloc(nn * sizeof(double));
    int it0, it1;
    double r0, r1;
    int cl = stage2d(c, H, h, q1, q2, w, h, q1, q2, w, 0.0, 1.0, p, dt, h1, a1, b1, w1,
                     &it0, &r0);
    cl += stage2d(c, H, h, q1, q2, w, h1, a1, b1, w1, 0.5, 0.5, p, dt, h2, a2, b2, w2,
                  &it1, &r1);
    memcpy(h, h2, n * sizeof(double));
    memcpy(q1, a2, n * sizeof(double));
    memcpy(q2, b2, n * sizeof(double));
    memcpy(w, w2, nn * sizeof(double));
    if (st) {
        st->iters[0] = it0; st->iters[1] = it1;
        st->resid[0] = r0; st->resid[1] = r1;
        st->clamped = cl;
    }
    free(h1); free(a1); free(b1); free(w1); free(h2); free(a2); free(b2); free(w2);
    return 0;
}

long long or2d_run(const or_cfg *c, const double *H, double *h, double *q1, double *q2,
                   double *w, double *p, double t_end, long long max_steps, double fixed_dt,
                   double *t_out, long long *iters_total)
{
    double t = 0.0;
    long long s = 0, it = 0;
    while (s < max_steps) {
        if (t_end > 0.0 && t >= t_end) break;
        double dt = fixed_dt > 0.0 ? fixed_dt : or2d_cfl_dt(c, H, h, q1, q2);
        if (!(dt > 0.0)) break;
        if (t_end > 0.0 && t + dt > t_end) dt = t_end - t;
        or_stats st;
        or2d_step(c, H, h, q1, q2, w, p, dt, &st);
        if (c->relax[0] > 0.0 || c->relax[1] > 0.0 || c->relax[2] > 0.0 || c->relax[3] > 0.0)
            or2d_relax(c, H, h, q1, q2, w, p, NULL, NULL, NULL, NULL, NULL);
        it += st.iters[0] + st.iters[1];
        t += dt;
        ++s;
    }
    if (t_out) *t_out = t;
    if (iters_total) *iters_total = it;
    return s;
}

/* 2D relaxation zones (Sec. 4.4 on each side): m(i, j) = m_x(i) m_y(j) at cells, the
 * product of the node means m_x(I - 1/2) m_y(J - 1/2) at nodes (the x and y blends applied
 * one after the other); see or1d_relax. */
void or2d_relax(const or_cfg *c, const double *H, double *h, double *q1, double *q2,
                double *w, double *p, const double *eta_t, const double *q1_t,
                const double *q2_t, const double *w_t, const double *p_t)
{
    const int nx = c->nx, ny = c->ny;
#pragma omp parallel for
    for (int j = 0; j < ny; ++j)
        for (int i = 0; i < nx; ++i) {
            double m = relax_m1(i, nx, c->dx, c->relax[0], c->relax[1]) *
                       relax_m1(j, ny, c->dy, c->relax[2], c->relax[3]);
            if (m == 1.0) continue;
            size_t k = CI(i, j);
            double hs = eta_t ? eta_t[k] + H[k] : (H[k] > 0.0 ? H[k] : 0.0);
            if (hs < 0.0) hs = 0.0;
            h[k] = m * h[k] + (1.0 - m) * hs;
            q1[k] = m * q1[k] + (1.0 - m) * (q1_t ? q1_t[k] : 0.0);
            q2[k] = m * q2[k] + (1.0 - m) * (q2_t ? q2_t[k] : 0.0);
        }
#pragma omp parallel for
    for (int J = 0; J <= ny; ++J)
        for (int I = 0; I <= nx; ++I) {
            double m = relax_node1(I, nx, c->dx, c->relax[0], c->relax[1]) *
                       relax_node1(J, ny, c->dy, c->relax[2], c->relax[3]);
            if (m == 1.0) continue;
            size_t k = NI(I, J);
            w[k] = m * w[k] + (1.0 - m) * (w_t ? w_t[k] : 0.0);
            p[k] = m * p[k] + (1.0 - m) * (p_t ? p_t[k] : 0.0);
        }
}

/* The breaking terms of Sec. 3 (Eq. 12) alone, as the stages apply them to U* and w*
 * with the step dt: public for the tests' closed-form pins. */
void or1d_breaking(const or_cfg *c, const double *H, const double *h, double *q, double *w,
                   double dt)
{
    breaking1d(c, H, h, q, w, dt);
}

void or2d_breaking(const or_cfg *c, const double *H, const double *h, double *q1, double *q2,
                   double *w, double dt)
{
    breaking2d(c, H, h, q1, q2, w, dt);
}
