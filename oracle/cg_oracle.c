/*
 * Plain FP64 CPU oracle of the per-RK-stage right-hand side of the
 * compressible Euler equations in curvilinear form with three shock-capturing
 * families: C-GBR (MEG6 / MIG4), LAD (E4 / C6) and the hybrid LAD-GBR.
 *
 * TEST INFRASTRUCTURE ONLY: it exists to check the CUDA library against the
 * paper.  Nothing in the product path may include, link or call it.  It is
 * deliberately slow and literal: whole padded arrays, one loop per step of
 * the method, in the order the paper (and the published methods it cites)
 * gives them.  Compile with -ffp-contract=off so that every a*b+c rounds twice.
 *
 * Paper: Kumar, Saini, Vadlamani, Chamarthi, arXiv 2511.18042.
 *   Sec. 2.1  governing equations, Eq. (1)-(3): conservative curvilinear form,
 *             convective fluxes, contravariant velocities, viscous stress.
 *   Sec. 2.2  LAD: Eq. (4)-(6) artificial coefficients, switch, spacings.
 *   Sec. 2.3  C-GBR: centralised interpolation Eq. (7), wave-appropriate
 *             selection Eq. (8), HLLC Eq. (9)-(10).
 *   Sec. 4    Algorithms 1-2 (LAD, C-GBR stage order); Sec. 5 Algorithm 3
 *             (hybrid LAD-GBR) and the troubled-cell criteria.
 * Where the paper only cites a method, the published method is followed and
 * named at the function (Suresh & Huynh 1997 MP5; Lele 1992 compact schemes;
 * Gaitonde & Visbal filter; Cook & Cabot truncated Gaussian; Toro HLLC;
 * Shu & Osher TVD-RK3; Thomas & Lombard conservative metrics).
 *
 * Pins (tests/test_oracle_pins.py): exact Riemann star states (Toro's table)
 * and the Sod density profile; HLLC consistency, textbook Cartesian form,
 * rotation / orientation / scaling invariance; MP5 polynomial exactness and
 * hand cases; modified wavenumbers of MEG6, MIG4, E4, C6; transfer functions
 * of the Gaussian and implicit filters; design order from the stencils
 * (sympy); RK3 order; periodic conservation; freestream on curvilinear 2D/3D
 * grids; exact metrics of an affine grid; x<->y symmetry of the 2D Riemann
 * configuration 3; hybrid limits; CFL closed form; hand values of beta*, of
 * kappa* and of the sensor.  C-GBR details (tests/test_oracle_gbr_pins.py):
 * the central states of the entropy and shear waves (Eq. 7-8) make their
 * semi-discrete operator skew-symmetric (energy conserved, the upwind
 * acoustic states dissipate); the characteristic frame diagonalises the
 * primitive Jacobian at the arithmetic mean state; a reflective wall is the
 * mirror plane of the doubled periodic domain; the per-interface hybrid
 * marks exactly the interfaces beside a troubled node (and, with a buffer
 * of B nodes, those beside a node within B of one).  Viscous terms (tests/test_oracle_viscous.py): discrete decay
 * rate of periodic and wall-bounded shear waves (E4 and C6 modified
 * wavenumbers) and their energy source; the isothermal no-slip wall as the
 * mirror of the doubled periodic channel; fourth-order convergence of the 3D
 * viscous terms on Cartesian and curvilinear grids and of heat conduction at
 * rest; a parallel flow fed by its own inflow profile is steady; Sutherland
 * against tabulated air viscosity.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif
#include "cg_oracle.h"

/* Marks the step of the method a function performs, for the flop-counting
 * build of this file (oracle/flopcount.cpp); nothing in this build. */
#ifndef ORC_REGION
#define ORC_REGION(name)
#endif

#define GH 8   /* ghost layers of the padded state */
#define GC 14  /* ghost layers of the extended coordinate box */

typedef struct {
    orc_params p;
    int nd, nv;
    int n[3], g[3], P[3];
    long N, NP;
    double *xh[3][3]; /* node metrics \hat\xi_{l,m} = (d xi_l / d x_m) / J, padded */
    double *jac;      /* J, padded */
    double *xt[3][3]; /* interface metrics \tilde\xi_{l,m} at l-interface i+1/2, stored at node i */
    double *dxl[3][3];/* LAD displacement vector Delta x_l, component m (Eq. 6) */
    double *prof[3][2]; /* per-node inflow profiles (primitive), or NULL */
} ctx_t;

/* ------------------------------------------------------------------ */
/* indexing                                                            */
/* ------------------------------------------------------------------ */
static long pidx(const ctx_t *c, int i, int j, int k)
{
    return (long)(i + c->g[0]) +
           (long)c->P[0] * ((long)(j + c->g[1]) + (long)c->P[1] * (long)(k + c->g[2]));
}
static long iidx(const ctx_t *c, int i, int j, int k)
{
    return (long)i + (long)c->n[0] * ((long)j + (long)c->n[1] * (long)k);
}
static long pstride(const ctx_t *c, int d)
{
    if (d == 0) return 1;
    if (d == 1) return c->P[0];
    return (long)c->P[0] * c->P[1];
}
static int imod(int a, int n) { int r = a % n; return r < 0 ? r + n : r; }
static int idiv_floor(int a, int n) { return (a - imod(a, n)) / n; }

/* box of positions: active dims [lo, hi), inactive dims {0} */
typedef struct { int lo[3], hi[3]; } box_t;
static box_t box_grow(const ctx_t *c, int grow)
{
    box_t b;
    for (int d = 0; d < 3; ++d) {
        if (d < c->nd) { b.lo[d] = -grow; b.hi[d] = c->n[d] + grow; }
        else { b.lo[d] = 0; b.hi[d] = 1; }
    }
    return b;
}
#define FOR_BOX(b, i, j, k)                          \
    for (int k = (b).lo[2]; k < (b).hi[2]; ++k)      \
        for (int j = (b).lo[1]; j < (b).hi[1]; ++j)  \
            for (int i = (b).lo[0]; i < (b).hi[0]; ++i)

/* The same loop shared among OpenMP threads, for bodies that write only
 * their own node (or line) and read nothing another iteration writes: every
 * value is computed by the same arithmetic whatever the thread count, and no
 * floating-point sum runs across iterations, so results do not depend on it. */
#ifdef _OPENMP
#define ORC_PRAGMA(x) _Pragma(#x)
/* loops of fewer than 512 iterations (nodes, or lines of a line loop) run
 * on the calling thread: a parallel region would cost more than the loop */
#define FOR_BOX_PAR(b, i, j, k)                                                          \
    ORC_PRAGMA(omp parallel for collapse(3) schedule(static)                             \
               if ((long)((b).hi[0] - (b).lo[0]) * ((b).hi[1] - (b).lo[1]) *             \
                   ((b).hi[2] - (b).lo[2]) >= 512L))                                      \
    FOR_BOX(b, i, j, k)
/* an element-wise loop over n values, shared the same way */
#define ORC_PAR_FOR(n) ORC_PRAGMA(omp parallel for schedule(static) if ((long)(n) >= 65536L))
#else
#define FOR_BOX_PAR(b, i, j, k) FOR_BOX(b, i, j, k)
#define ORC_PAR_FOR(n)
#endif

static double *padded(const ctx_t *c, int nc)
{
    double *f = (double *)malloc(sizeof(double) * (size_t)c->NP * nc);
    ORC_PAR_FOR(c->NP * nc)
    for (long q = 0; q < c->NP * nc; ++q) f[q] = NAN;
    return f;
}

static double dmin(double a, double b) { return a < b ? a : b; }
static double dmax(double a, double b) { return a > b ? a : b; }

/* ------------------------------------------------------------------ */
/* state conversions (Sec. 2.1: E = e + |u|^2/2, e = p/(rho(gamma-1)); */
/* the fifth conserved variable is energy per unit volume)             */
/* ------------------------------------------------------------------ */
static void cons_to_prim(int nd, double gamma, const double *Q, double *W)
{
    double rho = Q[0];
    double irho = 1.0 / rho;
    double ke = 0.0;
    W[0] = rho;
    for (int k = 0; k < nd; ++k) {
        W[1 + k] = Q[1 + k] * irho;
        ke += Q[1 + k] * W[1 + k];
    }
    W[nd + 1] = (gamma - 1.0) * (Q[nd + 1] - 0.5 * ke);
}
static void prim_to_cons(int nd, double gamma, const double *W, double *Q)
{
    double q = 0.0;
    Q[0] = W[0];
    for (int k = 0; k < nd; ++k) {
        Q[1 + k] = W[0] * W[1 + k];
        q += W[1 + k] * W[1 + k];
    }
    Q[nd + 1] = W[nd + 1] / (gamma - 1.0) + 0.5 * W[0] * q;
}

/* ------------------------------------------------------------------ */
/* ghost nodes by boundary condition, filled direction by direction   */
/* (x, then y over the x-extended range, then z).                     */
/* mode 0: primitive state, 1: conserved state, 2: scalar field.      */
/* extrapolation copies the boundary node; a reflective wall mirrors  */
/* (ghost -q <- node q-1) and negates the wall-normal velocity or      */
/* momentum; inflow holds the given state (constant, or the profile of */
/* the transverse position); periodic wraps.  The isothermal no-slip   */
/* wall mirrors with every velocity component negated, the pressure    */
/* kept and the temperature reflected about the wall value,            */
/* T_ghost = 2 T_w - T_mirror (so u = 0 and T = T_w at the face to      */
/* second order).  A scalar field wraps, mirrors at either wall and    */
/* copies otherwise.                                                   */
/* ------------------------------------------------------------------ */
static void wall_prim(const ctx_t *c, const double *Wm, double *Wg)
{
    int nd = c->nd, ip = nd + 1;
    double gm2 = c->p.gamma * c->p.minf * c->p.minf;
    double Tm = gm2 * Wm[ip] / Wm[0];
    double Tg = 2.0 * c->p.twall - Tm;
    Wg[ip] = Wm[ip];
    Wg[0] = gm2 * Wg[ip] / Tg;
    for (int m = 0; m < nd; ++m) Wg[1 + m] = -Wm[1 + m];
}

static long profile_index(const ctx_t *c, int d, const int *a)
{
    long pi = 0, mul = 1;
    for (int e = 0; e < c->nd; ++e) {
        if (e == d) continue;
        int x = a[e] < 0 ? 0 : (a[e] >= c->n[e] ? c->n[e] - 1 : a[e]);
        pi += (long)x * mul;
        mul *= c->n[e];
    }
    return pi;
}

static void fill_ghosts(const ctx_t *c, double *f, int nc, int mode)
{
    ORC_REGION(ghost);
    int nd = c->nd;
    for (int d = 0; d < nd; ++d) {
        box_t b;
        for (int e = 0; e < 3; ++e) {
            if (e >= nd) { b.lo[e] = 0; b.hi[e] = 1; }
            else if (e < d) { b.lo[e] = -c->g[e]; b.hi[e] = c->n[e] + c->g[e]; }
            else { b.lo[e] = 0; b.hi[e] = c->n[e]; }
        }
        b.lo[d] = 0; b.hi[d] = 1; /* iterate lines along d */
        int n = c->n[d];
        long face = c->N / n;
        for (int side = 0; side < 2; ++side) {
            int bc = c->p.bc[d][side];
            const double *prof = bc == ORC_BC_INFLOW ? c->prof[d][side] : NULL;
            double fixed[5];
            if (bc == ORC_BC_INFLOW && mode != 2) {
                if (mode == 0) for (int v = 0; v < c->nv; ++v) fixed[v] = c->p.inflow[d][side][v];
                else prim_to_cons(nd, c->p.gamma, c->p.inflow[d][side], fixed);
            }
            for (int q = 1; q <= c->g[d]; ++q) {
                int gi = side == 0 ? -q : n - 1 + q;
                int src, flip = 0, isfixed = 0, wall = 0;
                if (bc == ORC_BC_PERIODIC) src = imod(gi, n);
                else if (bc == ORC_BC_REFLECT) { src = side == 0 ? q - 1 : n - q; flip = (mode != 2); }
                else if (bc == ORC_BC_WALL) { src = side == 0 ? q - 1 : n - q; wall = (mode != 2); }
                else if (bc == ORC_BC_INFLOW && mode != 2) { src = 0; isfixed = 1; }
                else src = side == 0 ? 0 : n - 1;
                FOR_BOX_PAR(b, i, j, k) {
                    int a[3] = {i, j, k}, s[3] = {i, j, k};
                    a[d] = gi; s[d] = src;
                    long qa = pidx(c, a[0], a[1], a[2]), qs = pidx(c, s[0], s[1], s[2]);
                    if (isfixed && prof) {
                        long pi = profile_index(c, d, a);
                        double Wf[5], Qf[5];
                        for (int v = 0; v < c->nv; ++v) Wf[v] = prof[v * face + pi];
                        if (mode == 1) prim_to_cons(nd, c->p.gamma, Wf, Qf);
                        for (int v = 0; v < nc; ++v) f[v * c->NP + qa] = mode == 1 ? Qf[v] : Wf[v];
                        continue;
                    }
                    if (wall) {
                        double Wm[5], Wg[5], Q[5];
                        for (int v = 0; v < nc; ++v) Q[v] = f[v * c->NP + qs];
                        if (mode == 1) cons_to_prim(nd, c->p.gamma, Q, Wm);
                        else for (int v = 0; v < nc; ++v) Wm[v] = Q[v];
                        wall_prim(c, Wm, Wg);
                        if (mode == 1) prim_to_cons(nd, c->p.gamma, Wg, Q);
                        else for (int v = 0; v < nc; ++v) Q[v] = Wg[v];
                        for (int v = 0; v < nc; ++v) f[v * c->NP + qa] = Q[v];
                        continue;
                    }
                    for (int v = 0; v < nc; ++v) {
                        if (isfixed) f[v * c->NP + qa] = fixed[v];
                        else if (flip && v == 1 + d) f[v * c->NP + qa] = -f[v * c->NP + qs];
                        else f[v * c->NP + qa] = f[v * c->NP + qs];
                    }
                }
            }
        }
    }
}

/* primitives on the padded box from the interior conserved state */
static double *padded_prims(const ctx_t *c, const double *U)
{
    ORC_REGION(prim);
    double *Wp = padded(c, c->nv);
    box_t b = box_grow(c, 0);
    FOR_BOX_PAR(b, i, j, k) {
        double Q[5], W[5];
        long qi = iidx(c, i, j, k), qp = pidx(c, i, j, k);
        for (int v = 0; v < c->nv; ++v) Q[v] = U[v * c->N + qi];
        cons_to_prim(c->nd, c->p.gamma, Q, W);
        for (int v = 0; v < c->nv; ++v) Wp[v * c->NP + qp] = W[v];
    }
    fill_ghosts(c, Wp, c->nv, 0);
    return Wp;
}

/* ------------------------------------------------------------------ */
/* tridiagonal solvers (general Thomas; cyclic via Sherman-Morrison)   */
/* ------------------------------------------------------------------ */
static void thomas(int m, const double *a, const double *b, const double *cc,
                   const double *r, double *x)
{
    double *cp = (double *)malloc(sizeof(double) * m);
    double *dp = (double *)malloc(sizeof(double) * m);
    cp[0] = cc[0] / b[0];
    dp[0] = r[0] / b[0];
    for (int i = 1; i < m; ++i) {
        double den = b[i] - a[i] * cp[i - 1];
        cp[i] = cc[i] / den;
        dp[i] = (r[i] - a[i] * dp[i - 1]) / den;
    }
    x[m - 1] = dp[m - 1];
    for (int i = m - 2; i >= 0; --i) x[i] = dp[i] - cp[i] * x[i + 1];
    free(cp);
    free(dp);
}

/* a x_{i-1} + x_i + a x_{i+1} = r_i; cyclic: indices mod m; otherwise rows
 * 0 and m-1 are x = r (decoupled closure rows). */
void orc_tridiag(int m, double a, int cyclic, const double *r, double *x)
{
    double *A = (double *)malloc(sizeof(double) * m), *B = (double *)malloc(sizeof(double) * m);
    double *C = (double *)malloc(sizeof(double) * m);
    for (int i = 0; i < m; ++i) { A[i] = a; B[i] = 1.0; C[i] = a; }
    if (!cyclic) {
        A[0] = 0.0; C[0] = 0.0; A[m - 1] = 0.0; C[m - 1] = 0.0;
        thomas(m, A, B, C, r, x);
    } else {
        /* Sherman-Morrison: A = T + u v^T with u = (g,0..0,a), v = (1,0..0,a/g) */
        double gam = -B[0];
        double *u = (double *)calloc(m, sizeof(double)), *z = (double *)malloc(sizeof(double) * m);
        double *B2 = (double *)malloc(sizeof(double) * m);
        for (int i = 0; i < m; ++i) B2[i] = B[i];
        B2[0] = B[0] - gam;
        B2[m - 1] = B[m - 1] - a * a / gam;
        A[0] = 0.0; C[m - 1] = 0.0;
        thomas(m, A, B2, C, r, x);
        u[0] = gam; u[m - 1] = a;
        thomas(m, A, B2, C, u, z);
        double fact = (x[0] + a * x[m - 1] / gam) / (1.0 + z[0] + a * z[m - 1] / gam);
        for (int i = 0; i < m; ++i) x[i] -= fact * z[i];
        free(u); free(z); free(B2);
    }
    free(A); free(B); free(C);
}

/* ------------------------------------------------------------------ */
/* line operators.  f points at node 0 of a line whose values exist on */
/* [-ng, n+ng); s is the stride between nodes.                         */
/* ------------------------------------------------------------------ */
/* MEG6 gradient: explicit sixth-order central first derivative. */
static double op_meg6(const double *f, long s)
{
    return 0.75 * (f[s] - f[-s]) - (3.0 / 20.0) * (f[2 * s] - f[-2 * s]) +
           (1.0 / 60.0) * (f[3 * s] - f[-3 * s]);
}
/* E4: explicit fourth-order central first derivative. */
static double op_e4(const double *f, long s)
{
    return (2.0 / 3.0) * (f[s] - f[-s]) - (1.0 / 12.0) * (f[2 * s] - f[-2 * s]);
}
/* right-hand side of the compact schemes (Lele 1992):
 * MIG4: 1/4 f'_{i-1} + f'_i + 1/4 f'_{i+1} = 3/4 (f_{i+1} - f_{i-1})
 * C6:   1/3 f'_{i-1} + f'_i + 1/3 f'_{i+1} = 7/9 (f_{i+1} - f_{i-1}) + 1/36 (f_{i+2} - f_{i-2}) */
static double op_compact_rhs(int kind, const double *f, long s)
{
    if (kind == 1) return 0.75 * (f[s] - f[-s]);
    return (7.0 / 9.0) * (f[s] - f[-s]) + (1.0 / 36.0) * (f[2 * s] - f[-2 * s]);
}
static double compact_alpha(int kind) { return kind == 1 ? 0.25 : 1.0 / 3.0; }

/* Compact first derivative along a line.  Non-periodic: system on [lo, hi]
 * with explicit E4 closure rows at lo and hi.  Periodic: cyclic system on
 * [0, n-1], results copied to positions [lo, hi] by wrapping.  out indexed
 * like f (stride s). */
static void compact_line(int kind, int n, int periodic, int lo, int hi,
                         const double *f, long s, double *out)
{
    double a = compact_alpha(kind);
    if (periodic) {
        double *r = (double *)malloc(sizeof(double) * n), *x = (double *)malloc(sizeof(double) * n);
        for (int i = 0; i < n; ++i) r[i] = op_compact_rhs(kind, f + i * s, s);
        orc_tridiag(n, a, 1, r, x);
        for (int i = lo; i <= hi; ++i) out[i * s] = x[imod(i, n)];
        free(r); free(x);
    } else {
        int m = hi - lo + 1;
        double *r = (double *)malloc(sizeof(double) * m), *x = (double *)malloc(sizeof(double) * m);
        r[0] = op_e4(f + lo * s, s);
        r[m - 1] = op_e4(f + hi * s, s);
        for (int i = lo + 1; i < hi; ++i) r[i - lo] = op_compact_rhs(kind, f + i * s, s);
        orc_tridiag(m, a, 0, r, x);
        for (int i = lo; i <= hi; ++i) out[i * s] = x[i - lo];
        free(r); free(x);
    }
}

/* truncated Gaussian filter, 9 points (Cook & Cabot 2004, used by Kawai &
 * Lele 2008 for the overbar of Eq. (4)-(5)) */
static const double GAUSS_A0 = 3565.0 / 10368.0, GAUSS_A1 = 3091.0 / 12960.0,
                    GAUSS_A2 = 1997.0 / 25920.0, GAUSS_A3 = 149.0 / 12960.0,
                    GAUSS_A4 = 107.0 / 103680.0;
static double op_gauss(const double *f, long s)
{
    return GAUSS_A0 * f[0] + GAUSS_A1 * (f[-s] + f[s]) + GAUSS_A2 * (f[-2 * s] + f[2 * s]) +
           GAUSS_A3 * (f[-3 * s] + f[3 * s]) + GAUSS_A4 * (f[-4 * s] + f[4 * s]);
}

/* eighth-order implicit low-pass filter (Gaitonde & Visbal):
 * af fh_{i-1} + fh_i + af fh_{i+1} = sum_{m=0}^{4} (a_m/2)(f_{i+m} + f_{i-m}) */
static void filter_coeffs(double af, double b[5])
{
    b[0] = (93.0 + 70.0 * af) / 128.0;
    b[1] = 0.5 * ((7.0 + 18.0 * af) / 16.0);
    b[2] = 0.5 * ((-7.0 + 14.0 * af) / 32.0);
    b[3] = 0.5 * ((1.0 - 2.0 * af) / 16.0);
    b[4] = 0.5 * ((-1.0 + 2.0 * af) / 128.0);
}
static double op_filter_rhs(const double b[5], const double *f, long s)
{
    return b[0] * f[0] + b[1] * (f[s] + f[-s]) + b[2] * (f[2 * s] + f[-2 * s]) +
           b[3] * (f[3 * s] + f[-3 * s]) + b[4] * (f[4 * s] + f[-4 * s]);
}
/* Filter one line: non-periodic system on [-1, n] whose end rows keep the
 * ghost values; periodic: cyclic on [0, n-1].  Writes out[0..n-1]. */
static void filter_line(int n, int periodic, double af, const double *f, long s, double *out)
{
    double b[5];
    filter_coeffs(af, b);
    if (periodic) {
        double *r = (double *)malloc(sizeof(double) * n), *x = (double *)malloc(sizeof(double) * n);
        for (int i = 0; i < n; ++i) r[i] = op_filter_rhs(b, f + i * s, s);
        orc_tridiag(n, af, 1, r, x);
        for (int i = 0; i < n; ++i) out[i * s] = x[i];
        free(r); free(x);
    } else {
        int m = n + 2;
        double *r = (double *)malloc(sizeof(double) * m), *x = (double *)malloc(sizeof(double) * m);
        r[0] = f[-s];
        r[m - 1] = f[n * s];
        for (int i = 0; i < n; ++i) r[i + 1] = op_filter_rhs(b, f + i * s, s);
        orc_tridiag(m, af, 0, r, x);
        for (int i = 0; i < n; ++i) out[i * s] = x[i + 1];
        free(r); free(x);
    }
}

int orc_line_op(int kind, int n, int ng, int periodic, double alpha_f,
                const double *in, double *out)
{
    const double *f = in + ng;
    double *o = out + ng;
    for (int i = 0; i < n + 2 * ng; ++i) out[i] = NAN;
    switch (kind) {
    case 0: for (int i = -ng + 3; i <= n + ng - 4; ++i) o[i] = op_meg6(f + i, 1); break;
    case 2: for (int i = -ng + 2; i <= n + ng - 3; ++i) o[i] = op_e4(f + i, 1); break;
    case 1: case 3: compact_line(kind, n, periodic, -ng + 2, n + ng - 3, f, 1, o); break;
    case 4: for (int i = -ng + 4; i <= n + ng - 5; ++i) o[i] = op_gauss(f + i, 1); break;
    case 5: filter_line(n, periodic, alpha_f, f, 1, o); break;
    default: return -1;
    }
    return 0;
}

/* ------------------------------------------------------------------ */
/* gradient of a padded field along d, on every line of the padded box */
/* kind 0 MEG6 -> positions [-2, n+1]; 1 MIG4 / 3 C6 (compact) and     */
/* 2 E4 -> positions [-3, n+2].                                         */
/* ------------------------------------------------------------------ */
static void grad_field(const ctx_t *c, const double *f, int nc, int d, int kind, double *out)
{
    ORC_REGION(grad);
    int n = c->n[d], g = c->g[d];
    int periodic = c->p.bc[d][0] == ORC_BC_PERIODIC;
    long s = pstride(c, d);
    box_t b = box_grow(c, GH);
    b.lo[d] = 0; b.hi[d] = 1;
    FOR_BOX_PAR(b, i, j, k) {
        long q0 = pidx(c, i, j, k);
        for (int v = 0; v < nc; ++v) {
            const double *fl = f + v * c->NP + q0;
            double *ol = out + v * c->NP + q0;
            if (kind == 0) {
                for (int t = -g + 3; t <= n + g - 4; ++t) ol[t * s] = op_meg6(fl + t * s, s);
            } else if (kind == 2) {
                for (int t = -g + 2; t <= n + g - 3; ++t) ol[t * s] = op_e4(fl + t * s, s);
            } else {
                compact_line(kind, n, periodic, -g + 2, n + g - 3, fl, s, ol);
            }
        }
    }
}

/* ------------------------------------------------------------------ */
/* convective flux (Eq. 2) and HLLC (Eq. 9-10)                          */
/* ------------------------------------------------------------------ */
void orc_euler_flux(int nd, double gamma, const double *W, const double *xi, double *F)
{
    ORC_REGION(node_flux);
    int ip = nd + 1;
    double rho = W[0], p = W[ip], U = 0.0, q = 0.0;
    for (int m = 0; m < nd; ++m) {
        U += xi[m] * W[1 + m];
        q += W[1 + m] * W[1 + m];
    }
    double E = p / (gamma - 1.0) + 0.5 * rho * q;
    F[0] = rho * U;
    for (int m = 0; m < nd; ++m) F[1 + m] = rho * W[1 + m] * U + xi[m] * p;
    F[ip] = (E + p) * U;
}

/* HLLC with interface metrics xi (not normalised).  Wave speeds with Roe
 * averages (reading: the Roe sound speed is scaled by |xi| like the others);
 * star states as in Eq. (10), with E^K inside the braces read as the
 * specific total energy; star-region flux F^K + S^K (Q*^K - Q^K) (Toro). */
void orc_hllc(int nd, double gamma, const double *WL, const double *WR,
              const double *xi, double *F)
{
    ORC_REGION(hllc);
    int ip = nd + 1;
    double g2 = 0.0;
    for (int m = 0; m < nd; ++m) g2 += xi[m] * xi[m];
    double g = sqrt(g2);
    double rL = WL[0], pL = WL[ip], rR = WR[0], pR = WR[ip];
    double UL = 0.0, UR = 0.0, qL = 0.0, qR = 0.0;
    for (int m = 0; m < nd; ++m) {
        UL += xi[m] * WL[1 + m];
        UR += xi[m] * WR[1 + m];
        qL += WL[1 + m] * WL[1 + m];
        qR += WR[1 + m] * WR[1 + m];
    }
    double EL = pL / (gamma - 1.0) + 0.5 * rL * qL;
    double ER = pR / (gamma - 1.0) + 0.5 * rR * qR;
    double cL = sqrt(gamma * pL / rL), cR = sqrt(gamma * pR / rR);
    /* Roe averages */
    double sL = sqrt(rL), sR = sqrt(rR);
    double iden = 1.0 / (sL + sR);
    double qh = 0.0, Uh = 0.0;
    for (int m = 0; m < nd; ++m) {
        double uh = (sL * WL[1 + m] + sR * WR[1 + m]) * iden;
        qh += uh * uh;
        Uh += xi[m] * uh;
    }
    double HL = (EL + pL) / rL, HR = (ER + pR) / rR;
    double Hh = (sL * HL + sR * HR) * iden;
    double ch = sqrt((gamma - 1.0) * (Hh - 0.5 * qh));
    double SL = dmin(UL - cL * g, Uh - ch * g);
    double SR = dmax(UR + cR * g, Uh + ch * g);
    double Ss = (rR * UR * (SR - UR) - rL * UL * (SL - UL) + (pL - pR) * g2) /
                (rR * (SR - UR) - rL * (SL - UL));
    const double *W;
    double S, U, E, r, p;
    if (0.0 <= SL) { orc_euler_flux(nd, gamma, WL, xi, F); return; }
    if (0.0 <= Ss) { W = WL; S = SL; U = UL; E = EL; r = rL; p = pL; }
    else if (0.0 <= SR) { W = WR; S = SR; U = UR; E = ER; r = rR; p = pR; }
    else { orc_euler_flux(nd, gamma, WR, xi, F); return; }
    double FK[5], Qs[5], QK[5];
    orc_euler_flux(nd, gamma, W, xi, FK);
    double fac = r * (S - U) / (S - Ss);
    double ig2 = 1.0 / g2;
    Qs[0] = fac;
    QK[0] = r;
    for (int m = 0; m < nd; ++m) {
        /* printed x-row: [xi_x S* + (xi_y^2+xi_z^2) u - xi_y xi_x v - xi_z xi_x w]/|xi|^2
         * which equals u + xi_x (S* - U)/|xi|^2 */
        Qs[1 + m] = fac * (W[1 + m] + xi[m] * (Ss - U) * ig2);
        QK[1 + m] = r * W[1 + m];
    }
    Qs[ip] = fac * (E / r + (Ss - U) * (Ss * ig2 + p / (r * (S - U))));
    QK[ip] = E;
    for (int v = 0; v <= ip; ++v) F[v] = FK[v] + S * (Qs[v] - QK[v]);
}

/* ------------------------------------------------------------------ */
/* MP5 (Suresh & Huynh 1997), left state at i+1/2 from u_{i-2..i+2}     */
/* ------------------------------------------------------------------ */
static double minmod2(double a, double b)
{
    if (a > 0.0 && b > 0.0) return dmin(a, b);
    if (a < 0.0 && b < 0.0) return dmax(a, b);
    return 0.0;
}
static double minmod4(double a, double b, double c, double d)
{
    if (a > 0.0 && b > 0.0 && c > 0.0 && d > 0.0) return dmin(dmin(a, b), dmin(c, d));
    if (a < 0.0 && b < 0.0 && c < 0.0 && d < 0.0) return dmax(dmax(a, b), dmax(c, d));
    return 0.0;
}
double orc_mp5(double um2, double um1, double u0, double up1, double up2, double alpha, double eps)
{
    ORC_REGION(mp5);
    /* fifth-order upwind-biased interpolation */
    double ul = (2.0 * um2 - 13.0 * um1 + 47.0 * u0 + 27.0 * up1 - 3.0 * up2) / 60.0;
    double ump = u0 + minmod2(up1 - u0, alpha * (u0 - um1));
    if ((ul - u0) * (ul - ump) <= eps) return ul;
    double dm1 = um2 - 2.0 * um1 + u0;
    double d0 = um1 - 2.0 * u0 + up1;
    double dp1 = u0 - 2.0 * up1 + up2;
    double dm4p = minmod4(4.0 * d0 - dp1, 4.0 * dp1 - d0, d0, dp1);
    double dm4m = minmod4(4.0 * d0 - dm1, 4.0 * dm1 - d0, d0, dm1);
    double uul = u0 + alpha * (u0 - um1);
    double uav = 0.5 * (u0 + up1);
    double umd = uav - 0.5 * dm4p;
    double ulc = u0 + 0.5 * (u0 - um1) + (4.0 / 3.0) * dm4m;
    double umin = dmax(dmin(dmin(u0, up1), umd), dmin(dmin(u0, uul), ulc));
    double umax = dmin(dmax(dmax(u0, up1), umd), dmax(dmax(u0, uul), ulc));
    return ul + minmod2(umin - ul, umax - ul);
}

/* ------------------------------------------------------------------ */
/* C-GBR interface flux (Sec. 2.3)                                      */
/* ------------------------------------------------------------------ */
typedef struct {
    int nd, nv;
    double gamma, thr, eps, alpha;
    int mp_printed, ac_mp5, pos;
} gbr_cfg;

typedef struct {
    double n[3], t1[3], t2[3];
    double rb, cb, ic2, ha, hb, cr;
} charframe;

/* orthonormal tangents: 2D t = (-n_y, n_x); 3D t1 perpendicular to n built
 * from the two largest components of n (ties: lowest index is "smallest"),
 * t2 = n x t1. */
static void tangents(int nd, const double *n, double *t1, double *t2)
{
    if (nd == 2) { t1[0] = -n[1]; t1[1] = n[0]; return; }
    if (nd != 3) return;
    int s = 0;
    if (fabs(n[1]) < fabs(n[s])) s = 1;
    if (fabs(n[2]) < fabs(n[s])) s = 2;
    int a = (s + 1) % 3, b = (s + 2) % 3;
    double r = 1.0 / sqrt(n[a] * n[a] + n[b] * n[b]);
    t1[s] = 0.0;
    t1[a] = -n[b] * r;
    t1[b] = n[a] * r;
    t2[0] = n[1] * t1[2] - n[2] * t1[1];
    t2[1] = n[2] * t1[0] - n[0] * t1[2];
    t2[2] = n[0] * t1[1] - n[1] * t1[0];
}

/* characteristic variables of primitive W = (rho, u, p) at the frame:
 * waves 1: u_n - c, 2: entropy, 3..: shear, last: u_n + c;
 * l1 = (0, -rho n/(2c), 1/(2c^2)), l2 = (1, 0, -1/c^2), l_shear = (0, t, 0),
 * l_last = (0, rho n/(2c), 1/(2c^2)). */
static void to_char(int nd, const charframe *fr, const double *w, double *cv)
{
    int ip = nd + 1;
    double un = 0.0;
    for (int m = 0; m < nd; ++m) un += fr->n[m] * w[1 + m];
    cv[0] = fr->ha * w[ip] - fr->hb * un;
    cv[1] = w[0] - fr->ic2 * w[ip];
    if (nd >= 2) {
        double s = 0.0;
        for (int m = 0; m < nd; ++m) s += fr->t1[m] * w[1 + m];
        cv[2] = s;
    }
    if (nd == 3) {
        double s = 0.0;
        for (int m = 0; m < nd; ++m) s += fr->t2[m] * w[1 + m];
        cv[3] = s;
    }
    cv[ip] = fr->ha * w[ip] + fr->hb * un;
}
/* inverse: rho = C2 + (C1 + C_last), p = c^2 (C1 + C_last),
 * u_n = (c/rho)(C_last - C1), u = u_n n + C3 t1 + C4 t2 */
static void from_char(int nd, const charframe *fr, const double *cv, double *w)
{
    int ip = nd + 1;
    double s = cv[0] + cv[ip];
    double un = (cv[ip] - cv[0]) * fr->cr;
    w[0] = cv[1] + s;
    w[ip] = (fr->cb * fr->cb) * s;
    for (int m = 0; m < nd; ++m) {
        double u = un * fr->n[m];
        if (nd >= 2) u = u + cv[2] * fr->t1[m];
        if (nd == 3) u = u + cv[3] * fr->t2[m];
        w[1 + m] = u;
    }
}

/* interface frame (Sec. 2.3): unit normal n = xi/|xi| of the interface
 * metrics, its tangents, and the sound speed and density of the arithmetic
 * mean of the primitive states at nodes i and i+1 (reading: mean state) */
static void char_frame(int nd, double gamma, const double *Wi, const double *Wi1,
                       const double *xi, charframe *fr)
{
    int ip = nd + 1;
    double g2 = 0.0;
    for (int m = 0; m < nd; ++m) g2 += xi[m] * xi[m];
    double ig = 1.0 / sqrt(g2);
    for (int m = 0; m < nd; ++m) fr->n[m] = xi[m] * ig;
    tangents(nd, fr->n, fr->t1, fr->t2);
    fr->rb = 0.5 * (Wi[0] + Wi1[0]);
    double pb = 0.5 * (Wi[ip] + Wi1[ip]);
    fr->cb = sqrt(gamma * pb / fr->rb);
    double ic = 1.0 / fr->cb;
    fr->ic2 = ic * ic;
    fr->ha = 0.5 * fr->ic2;
    fr->hb = 0.5 * fr->rb * ic;
    fr->cr = fr->cb / fr->rb;
}

/* The characteristic transform of the interface between nodes with primitive
 * states Wi and Wi1 (exposed for the pins): inverse = 0 gives cv = L w, the
 * characteristic variables of primitive w; inverse = 1 gives w = R cv. */
void orc_char_transform(int nd, double gamma, const double *Wi, const double *Wi1,
                        const double *xi, int inverse, const double *in, double *out)
{
    charframe fr;
    char_frame(nd, gamma, Wi, Wi1, xi, &fr);
    if (inverse) from_char(nd, &fr, in, out);
    else to_char(nd, &fr, in, out);
}

/* Wst[j] = W_{i-2+j} (j = 0..5), Wd[j] = W'_{i-1+j} (j = 0..3), om = interface sensor */
static void gbr_flux(const gbr_cfg *q, const double Wst[6][5], const double Wd[4][5],
                     double om, const double *xi, double *F)
{
    ORC_REGION(reconstruct);
    int nd = q->nd, nv = q->nv, ip = nv - 1;
    const double c12 = 1.0 / 12.0;
    /* second derivatives from values and first derivatives (Chamarthi):
     * W''_j = 2 (W_{j+1} - 2 W_j + W_{j-1}) - (W'_{j+1} - W'_{j-1}) / 2 */
    double W2[2][5];
    for (int v = 0; v < nv; ++v) {
        W2[0][v] = 2.0 * (Wst[3][v] - 2.0 * Wst[2][v] + Wst[1][v]) - 0.5 * (Wd[2][v] - Wd[0][v]);
        W2[1][v] = 2.0 * (Wst[4][v] - 2.0 * Wst[3][v] + Wst[2][v]) - 0.5 * (Wd[3][v] - Wd[1][v]);
    }
    charframe fr;
    char_frame(nd, q->gamma, Wst[2], Wst[3], xi, &fr);

    double C[6][5], Cd[2][5], Cdd[2][5];
    for (int j = 0; j < 6; ++j) to_char(nd, &fr, Wst[j], C[j]);
    to_char(nd, &fr, Wd[1], Cd[0]);
    to_char(nd, &fr, Wd[2], Cd[1]);
    to_char(nd, &fr, W2[0], Cdd[0]);
    to_char(nd, &fr, W2[1], Cdd[1]);

    int disc = om > q->thr;
    double CL[5], CR[5];
    for (int b = 0; b < nv; ++b) {
        double v0 = C[0][b], v1 = C[1][b], v2 = C[2][b], v3 = C[3][b], v4 = C[4][b], v5 = C[5][b];
        /* linear gradient-based states (MEG6 / MIG4) and their average, Eq. (7) */
        double cl = v2 + 0.5 * Cd[0][b] + Cdd[0][b] * c12;
        double cr = v3 - 0.5 * Cd[1][b] + Cdd[1][b] * c12;
        double cc = 0.5 * (cl + cr);
        if (b == 0 || b == ip) {            /* acoustic: sensor (Eq. 8, b = 1, 5) */
            if (disc || q->ac_mp5) {
                CL[b] = orc_mp5(v0, v1, v2, v3, v4, q->alpha, q->eps);
                CR[b] = orc_mp5(v5, v4, v3, v2, v1, q->alpha, q->eps);
            } else { CL[b] = cl; CR[b] = cr; }
        } else if (b == 1) {                /* entropy: MP criterion (Eq. 8, b = 2) */
            double umpL = v2 + minmod2(v3 - v2, q->alpha * (v2 - v1));
            double tL = (cl - v2) * (cl - umpL);
            int limL = q->mp_printed ? (tL <= q->eps) : (tL > q->eps);
            CL[b] = limL ? orc_mp5(v0, v1, v2, v3, v4, q->alpha, q->eps) : cc;
            double umpR = v3 + minmod2(v2 - v3, q->alpha * (v3 - v4));
            double tR = (cr - v3) * (cr - umpR);
            int limR = q->mp_printed ? (tR <= q->eps) : (tR > q->eps);
            CR[b] = limR ? orc_mp5(v5, v4, v3, v2, v1, q->alpha, q->eps) : cc;
        } else {                            /* shear: sensor (Eq. 8, b = 3, 4) */
            if (disc) {
                CL[b] = orc_mp5(v0, v1, v2, v3, v4, q->alpha, q->eps);
                CR[b] = orc_mp5(v5, v4, v3, v2, v1, q->alpha, q->eps);
            } else { CL[b] = cc; CR[b] = cc; }
        }
    }
    double WL[5], WR[5];
    from_char(nd, &fr, CL, WL);
    from_char(nd, &fr, CR, WR);
    if (q->pos && (WL[0] <= 0.0 || WL[ip] <= 0.0 || WR[0] <= 0.0 || WR[ip] <= 0.0)) {
        for (int v = 0; v < nv; ++v) { WL[v] = Wst[2][v]; WR[v] = Wst[3][v]; }
    }
    orc_hllc(nd, q->gamma, WL, WR, xi, F);
}

/* ------------------------------------------------------------------ */
/* discontinuity sensor Omega^d per node (reading: pressure sensor     */
/* max over directions times a Ducros ratio that tends to one in       */
/* irrotational, dilatation-free flow, e.g. a fluid at rest), on the   */
/* box [-4, n+3] so that interface windows reaching 3 nodes past the   */
/* boundary interfaces exist                                           */
/* ------------------------------------------------------------------ */
static void omega_field(const ctx_t *c, const double *Wp, double *const Wd[3], double *om)
{
    ORC_REGION(sensor);
    int nd = c->nd, ip = nd + 1;
    box_t b = box_grow(c, 4);
    FOR_BOX_PAR(b, i, j, k) {
        long q = pidx(c, i, j, k);
        const double *p = Wp + ip * c->NP;
        double phi = 0.0;
        for (int l = 0; l < nd; ++l) {
            long s = pstride(c, l);
            double a = fabs(p[q + s] - 2.0 * p[q] + p[q - s]) / (p[q + s] + 2.0 * p[q] + p[q - s]);
            if (a > phi) phi = a;
        }
        double gu[3][3];
        for (int kk = 0; kk < nd; ++kk)
            for (int m = 0; m < nd; ++m) {
                double s = 0.0;
                for (int l = 0; l < nd; ++l) {
                    double xm = c->jac[q] * c->xh[l][m][q];
                    s += xm * Wd[l][(1 + kk) * c->NP + q];
                }
                gu[kk][m] = s;
            }
        double div = 0.0;
        for (int kk = 0; kk < nd; ++kk) div += gu[kk][kk];
        double curl2 = 0.0;
        if (nd == 2) {
            double w3 = gu[1][0] - gu[0][1];
            curl2 = w3 * w3;
        } else if (nd == 3) {
            double w1 = gu[2][1] - gu[1][2], w2 = gu[0][2] - gu[2][0], w3 = gu[1][0] - gu[0][1];
            curl2 = w1 * w1 + w2 * w2 + w3 * w3;
        }
        double zeta = (div * div + 1e-32) / (div * div + curl2 + 1e-32);
        om[q] = phi * zeta;
    }
}

static gbr_cfg make_gbr_cfg(const ctx_t *c)
{
    gbr_cfg g;
    g.nd = c->nd; g.nv = c->nv; g.gamma = c->p.gamma; g.thr = c->p.sensor_thresh;
    g.eps = c->p.mp_eps; g.alpha = c->p.mp_alpha; g.mp_printed = c->p.read_mp_printed;
    g.ac_mp5 = c->p.read_acoustic_mp5; g.pos = c->p.positivity_fallback;
    return g;
}

/* GBR interface fluxes along d: interior lines, interfaces i+1/2 for
 * i = -1..n-1, stored in Fi (padded, nv comps) at node i.  mask (padded
 * bytes, or NULL) restricts the computation to flagged interfaces. */
static void gbr_dir_fluxes(const ctx_t *c, const double *Wp, double *const Wd[3],
                           const double *om, int d, const unsigned char *mask, double *Fi)
{
    int nd = c->nd, nv = c->nv, n = c->n[d];
    long s = pstride(c, d);
    gbr_cfg cfg = make_gbr_cfg(c);
    box_t b = box_grow(c, 0);
    b.lo[d] = 0; b.hi[d] = 1;
    FOR_BOX_PAR(b, i0, j0, k0) {
        long q0 = pidx(c, i0, j0, k0);
        for (int i = -1; i <= n - 1; ++i) {
            long q = q0 + i * s;
            if (mask && !mask[q]) continue;
            double Wst[6][5], Wdd[4][5], xi[3], F[5];
            for (int jj = 0; jj < 6; ++jj)
                for (int v = 0; v < nv; ++v) Wst[jj][v] = Wp[v * c->NP + q + (jj - 2) * s];
            for (int jj = 0; jj < 4; ++jj)
                for (int v = 0; v < nv; ++v) Wdd[jj][v] = Wd[d][v * c->NP + q + (jj - 1) * s];
            /* interface sensor: largest node value over the window i-w+1 .. i+w
             * (w = 4 covers every node the linear states depend on) */
            int w = c->p.omega_window;
            double ob = om[q];
            for (int jj = 1 - w; jj <= w; ++jj) ob = dmax(ob, om[q + jj * s]);
            for (int m = 0; m < nd; ++m) xi[m] = c->xt[d][m][q];
            gbr_flux(&cfg, Wst, Wdd, ob, xi, F);
            for (int v = 0; v < nv; ++v) Fi[v * c->NP + q] = F[v];
        }
    }
}

/* ------------------------------------------------------------------ */
/* LAD (Sec. 2.2): node fluxes F^c + F^v with artificial beta*, kappa* */
/* ------------------------------------------------------------------ */
typedef struct {
    double *Fn[3];   /* node total flux along each direction, padded nv comps */
    double *beta, *kappa; /* filtered coefficients, padded (ghosts by the scalar rule) */
} lad_out;

/* mode LADF_FULL: F^c - F^v with the artificial coefficients and, when the
 * case is viscous, the physical ones; LADF_NOPHYS: without the physical
 * viscosity; LADF_VISC: the physical viscous flux alone, -F^v (beta* and
 * kappa* are not computed). */
enum { LADF_FULL = 0, LADF_NOPHYS = 1, LADF_VISC = 2 };

/* Sutherland's law in units of the free-stream viscosity and temperature,
 * divided by Re: mu_hat(T) = T^{3/2} (1 + S) / (T + S) / Re (Sec. 2.1). */
static double mu_hat(const ctx_t *c, double T)
{
    double S = c->p.suth;
    return T * sqrt(T) * (1.0 + S) / (T + S) / c->p.re;
}

static void lad_fluxes(const ctx_t *c, const double *Wp, int dkind, int mode, lad_out *out)
{
    ORC_REGION(lad_fluxes);
    int nd = c->nd, nv = c->nv, ip = nd + 1;
    double gamma = c->p.gamma;
    double gm2 = gamma * c->p.minf * c->p.minf;
    /* node scalars: velocities, T = gamma M^2 p / rho, rho, e = p / (rho (gamma-1)) */
    int nf = nd + 3;
    double *fs = padded(c, nf);
    double *cs = padded(c, 1);
    box_t all = box_grow(c, GH);
    FOR_BOX_PAR(all, i, j, k) {
        long q = pidx(c, i, j, k);
        double rho = Wp[q], p = Wp[ip * c->NP + q];
        for (int kk = 0; kk < nd; ++kk) fs[kk * c->NP + q] = Wp[(1 + kk) * c->NP + q];
        fs[nd * c->NP + q] = gm2 * p / rho;
        fs[(nd + 1) * c->NP + q] = rho;
        fs[(nd + 2) * c->NP + q] = p / (rho * (gamma - 1.0));
        cs[q] = sqrt(gamma * p / rho);
    }
    /* computational derivatives along each direction (E4 or C6) */
    double *df[3] = {NULL, NULL, NULL};
    for (int l = 0; l < nd; ++l) {
        df[l] = padded(c, nf);
        grad_field(c, fs, nf, l, dkind, df[l]);
    }
    /* physical gradients by the chain rule, and the dilatation, on [-3, n+2] */
    double *gr = padded(c, nf * nd);     /* gr[(f*nd + m)] = d f / d x_m */
    double *dv = padded(c, 1);
    box_t b3 = box_grow(c, 3);
    FOR_BOX_PAR(b3, i, j, k) {
        long q = pidx(c, i, j, k);
        for (int f = 0; f < nf; ++f)
            for (int m = 0; m < nd; ++m) {
                double s = 0.0;
                for (int l = 0; l < nd; ++l) {
                    double xm = c->jac[q] * c->xh[l][m][q];
                    s += xm * df[l][f * c->NP + q];
                }
                gr[(f * nd + m) * c->NP + q] = s;
            }
        double div = 0.0;
        for (int kk = 0; kk < nd; ++kk) div += gr[(kk * nd + kk) * c->NP + q];
        dv[q] = div;
    }
    /* raw coefficients at interior nodes, Eq. (4)-(6) */
    double *bt = padded(c, 1), *kp = padded(c, 1);
    box_t b0 = box_grow(c, 0);
    double *tmp = padded(c, 1);
    if (mode != LADF_VISC) {
    FOR_BOX_PAR(b0, i, j, k) {
        long q = pidx(c, i, j, k);
        double rho = Wp[q];
        double T = fs[nd * c->NP + q];
        double div = dv[q];
        double curl2 = 0.0;
        if (nd == 2) {
            double w3 = gr[(1 * nd + 0) * c->NP + q] - gr[(0 * nd + 1) * c->NP + q];
            curl2 = w3 * w3;
        } else if (nd == 3) {
            double w1 = gr[(2 * nd + 1) * c->NP + q] - gr[(1 * nd + 2) * c->NP + q];
            double w2 = gr[(0 * nd + 2) * c->NP + q] - gr[(2 * nd + 0) * c->NP + q];
            double w3 = gr[(1 * nd + 0) * c->NP + q] - gr[(0 * nd + 1) * c->NP + q];
            curl2 = w1 * w1 + w2 * w2 + w3 * w3;
        }
        double heav = div < 0.0 ? 1.0 : 0.0;
        double fsw = heav * (div * div) / (div * div + curl2 + 1e-32);
        /* |grad rho|, |grad e| */
        double gmr = 0.0, gme = 0.0;
        for (int m = 0; m < nd; ++m) {
            double a = gr[((nd + 1) * nd + m) * c->NP + q], e = gr[((nd + 2) * nd + m) * c->NP + q];
            gmr += a * a;
            gme += e * e;
        }
        gmr = sqrt(gmr);
        gme = sqrt(gme);
        double sb = 0.0, sk = 0.0;
        for (int l = 0; l < nd; ++l) {
            long s = pstride(c, l);
            const double *e = fs + (nd + 2) * c->NP;
            double d4d = (dv[q - 2 * s] + dv[q + 2 * s]) - 4.0 * (dv[q - s] + dv[q + s]) + 6.0 * dv[q];
            double d4e = (e[q - 2 * s] + e[q + 2 * s]) - 4.0 * (e[q - s] + e[q + s]) + 6.0 * e[q];
            double pr = 0.0, pe = 0.0;
            for (int m = 0; m < nd; ++m) {
                pr += c->dxl[l][m][q] * gr[((nd + 1) * nd + m) * c->NP + q];
                pe += c->dxl[l][m][q] * gr[((nd + 2) * nd + m) * c->NP + q];
            }
            double Db = fabs(pr) / (gmr + 1e-32);
            double Dk = fabs(pe) / (gme + 1e-32);
            sb += d4d * Db * Db;
            sk += d4e * Dk;
        }
        bt[q] = c->p.c_beta * rho * fsw * fabs(sb);
        kp[q] = c->p.c_kappa * (rho * cs[q] / T) * fabs(sk);
    }
    /* truncated-Gaussian overbar, applied along xi, eta, zeta in turn */
    double *fld[2] = {bt, kp};
    for (int w = 0; w < 2; ++w) {
        for (int l = 0; l < nd; ++l) {
            fill_ghosts(c, fld[w], 1, 2);
            long s = pstride(c, l);
            FOR_BOX_PAR(b0, i, j, k) {
                long q = pidx(c, i, j, k);
                tmp[q] = op_gauss(fld[w] + q, s);
            }
            FOR_BOX_PAR(b0, i, j, k) {
                long q = pidx(c, i, j, k);
                fld[w][q] = tmp[q];
            }
        }
        fill_ghosts(c, fld[w], 1, 2);
    }
    }
    /* node fluxes along each direction at positions [-2, n+1] (interior lines):
     * tau = beta* div I (the stress of Eq. 3 with mu = 0: no physical viscosity
     * in the inviscid cases and C_mu not employed), phi_m = u_m tau + kappa* dT/dx_m.
     * Viscous cases (Eq. 3 with Stokes' hypothesis): tau_mi = mu (du_i/dx_m +
     * du_m/dx_i) + delta_mi (beta* - 2/3 mu) div, phi_m = sum_i u_i tau_mi +
     * (kappa* + kappa_hat) dT/dx_m. */
    int conv = mode != LADF_VISC, art = mode != LADF_VISC;
    int phys = c->p.viscous && mode != LADF_NOPHYS;
    double kc = (gamma - 1.0) * c->p.pr * c->p.minf * c->p.minf;
    for (int l = 0; l < nd; ++l) {
        out->Fn[l] = padded(c, nv);
        box_t bl = box_grow(c, 0);
        bl.lo[l] = -2; bl.hi[l] = c->n[l] + 2;
        FOR_BOX_PAR(bl, i, j, k) {
            long q = pidx(c, i, j, k);
            double W[5], xi[3], Fc[5];
            for (int v = 0; v < nv; ++v) W[v] = Wp[v * c->NP + q];
            for (int m = 0; m < nd; ++m) xi[m] = c->xh[l][m][q];
            if (conv) orc_euler_flux(nd, gamma, W, xi, Fc);
            else for (int v = 0; v < nv; ++v) Fc[v] = 0.0;
            if (phys) {
                double T = fs[nd * c->NP + q];
                double mu = mu_hat(c, T);
                double kth = mu / kc;
                double lam = (art ? bt[q] : (double)0.0) - (2.0 / 3.0) * mu;
                double kap = (art ? kp[q] : (double)0.0) + kth;
                double tau[3][3];
                for (int m = 0; m < nd; ++m)
                    for (int a = 0; a < nd; ++a) {
                        double sm = gr[(a * nd + m) * c->NP + q] + gr[(m * nd + a) * c->NP + q];
                        tau[m][a] = mu * sm;
                        if (m == a) tau[m][a] = tau[m][a] + lam * dv[q];
                    }
                double fe = 0.0;
                for (int m = 0; m < nd; ++m) {
                    double phi = W[1] * tau[m][0];
                    for (int a = 1; a < nd; ++a) phi = phi + W[1 + a] * tau[m][a];
                    phi = phi + kap * gr[(nd * nd + m) * c->NP + q];
                    fe = m == 0 ? xi[m] * phi : fe + xi[m] * phi;
                }
                out->Fn[l][q] = Fc[0];
                for (int a = 0; a < nd; ++a) {
                    double fv = xi[0] * tau[0][a];
                    for (int m = 1; m < nd; ++m) fv = fv + xi[m] * tau[m][a];
                    out->Fn[l][(1 + a) * c->NP + q] = Fc[1 + a] + (-fv);
                }
                out->Fn[l][ip * c->NP + q] = Fc[ip] + (-fe);
                continue;
            }
            double tau = bt[q] * dv[q];
            double fe = 0.0;
            for (int m = 0; m < nd; ++m) {
                double phi = W[1 + m] * tau + kp[q] * gr[(nd * nd + m) * c->NP + q];
                fe += xi[m] * phi;
            }
            out->Fn[l][q] = Fc[0];
            for (int m = 0; m < nd; ++m) out->Fn[l][(1 + m) * c->NP + q] = Fc[1 + m] + (-(xi[m] * tau));
            out->Fn[l][ip * c->NP + q] = Fc[ip] + (-fe);
        }
    }
    out->beta = bt;
    out->kappa = kp;
    free(fs); free(cs); free(gr); free(dv); free(tmp);
    for (int l = 0; l < nd; ++l) free(df[l]);
}

/* acc += D_l F_l at interior nodes (E4 explicit, or C6 compact on [0, n-1]
 * with E4 closure rows; periodic: cyclic) */
static void lad_divergence(const ctx_t *c, double *const Fn[3], int dkind, double *acc)
{
    ORC_REGION(lad_div);
    int nd = c->nd, nv = c->nv;
    double *tmp = padded(c, nv);
    for (int l = 0; l < nd; ++l) {
        int n = c->n[l];
        int periodic = c->p.bc[l][0] == ORC_BC_PERIODIC;
        long s = pstride(c, l);
        box_t b = box_grow(c, 0);
        b.lo[l] = 0; b.hi[l] = 1;
        FOR_BOX_PAR(b, i0, j0, k0) {
            long q0 = pidx(c, i0, j0, k0);
            for (int v = 0; v < nv; ++v) {
                const double *f = Fn[l] + v * c->NP + q0;
                double *o = tmp + v * c->NP + q0;
                if (dkind == 2) for (int t = 0; t < n; ++t) o[t * s] = op_e4(f + t * s, s);
                else compact_line(3, n, periodic, 0, n - 1, f, s, o);
            }
        }
        box_t b0 = box_grow(c, 0);
        FOR_BOX_PAR(b0, i, j, k) {
            long q = pidx(c, i, j, k), qi = iidx(c, i, j, k);
            for (int v = 0; v < nv; ++v) acc[v * c->N + qi] += tmp[v * c->NP + q];
        }
    }
    free(tmp);
}

/* ------------------------------------------------------------------ */
/* RHS assembly                                                        */
/* ------------------------------------------------------------------ */
static void free_lad(lad_out *o, int nd)
{
    for (int l = 0; l < nd; ++l) free(o->Fn[l]);
    free(o->beta);
    free(o->kappa);
}

/* acc += F_{i+1/2} - F_{i-1/2} along d */
static void add_iface_diff(const ctx_t *c, const double *Fi, int d, double *acc)
{
    ORC_REGION(flux_diff);
    long s = pstride(c, d);
    box_t b0 = box_grow(c, 0);
    FOR_BOX_PAR(b0, i, j, k) {
        long q = pidx(c, i, j, k), qi = iidx(c, i, j, k);
        for (int v = 0; v < c->nv; ++v)
            acc[v * c->N + qi] += Fi[v * c->NP + q] - Fi[v * c->NP + q - s];
    }
}

static int is_troubled(const ctx_t *c, double rho, double p)
{
    return rho < c->p.hyb_rho || p < c->p.hyb_p;
}

static long global_troubled(const ctx_t *c, const double *Wp)
{
    long cnt = 0;
    box_t b0 = box_grow(c, 0);
    FOR_BOX(b0, i, j, k) {
        long q = pidx(c, i, j, k);
        if (is_troubled(c, Wp[q], Wp[(c->nd + 1) * c->NP + q])) ++cnt;
    }
    return cnt;
}

/* Physical viscous terms of the C-GBR and per-interface hybrid stages
 * (reading: the paper's viscous routines are central differences shared with
 * the LAD framework, without the alpha-damping interface scheme): node
 * fluxes -F^v from E4 gradients, acc += E4 derivative along each direction. */
static void viscous_pass(const ctx_t *c, const double *Wp, double *acc)
{
    lad_out lv;
    lad_fluxes(c, Wp, 2, LADF_VISC, &lv);
    lad_divergence(c, lv.Fn, 2, acc);
    free_lad(&lv, c->nd);
}

/* scheme: the effective scheme of this stage; acc must be zeroed */
static void rhs_acc(const ctx_t *c, const double *Wp, int scheme, double *acc, double *iface_out, int iface_dir)
{
    ORC_REGION(hybrid_mix);
    int nd = c->nd, nv = c->nv;
    if (c->p.viscous && scheme != ORC_LAD_E4 && scheme != ORC_LAD_C6) viscous_pass(c, Wp, acc);
    if (scheme == ORC_MEG6 || scheme == ORC_MIG4) {
        double *Wd[3] = {NULL, NULL, NULL};
        for (int l = 0; l < nd; ++l) {
            Wd[l] = padded(c, nv);
            grad_field(c, Wp, nv, l, scheme == ORC_MEG6 ? 0 : 1, Wd[l]);
        }
        double *om = padded(c, 1);
        omega_field(c, Wp, Wd, om);
        double *Fi = padded(c, nv);
        for (int d = 0; d < nd; ++d) {
            gbr_dir_fluxes(c, Wp, Wd, om, d, NULL, Fi);
            add_iface_diff(c, Fi, d, acc);
            if (iface_out && d == iface_dir) memcpy(iface_out, Fi, sizeof(double) * c->NP * nv);
        }
        free(Fi); free(om);
        for (int l = 0; l < nd; ++l) free(Wd[l]);
    } else if (scheme == ORC_LAD_E4 || scheme == ORC_LAD_C6) {
        lad_out lo;
        lad_fluxes(c, Wp, scheme == ORC_LAD_E4 ? 2 : 3, LADF_FULL, &lo);
        lad_divergence(c, lo.Fn, scheme == ORC_LAD_E4 ? 2 : 3, acc);
        free_lad(&lo, nd);
    } else { /* per-cell hybrid: GBR-MEG6 flux where a neighbour is troubled, else LAD-E4 in flux form */
        double *Wd[3] = {NULL, NULL, NULL};
        for (int l = 0; l < nd; ++l) {
            Wd[l] = padded(c, nv);
            grad_field(c, Wp, nv, l, 0, Wd[l]);
        }
        double *om = padded(c, 1);
        omega_field(c, Wp, Wd, om);
        /* troubled nodes on [-1-B, n+B], then the buffer: a node is marked
         * if any node within B of it (in every direction) is troubled */
        int B = c->p.hybrid_buffer;
        unsigned char *t0 = (unsigned char *)calloc(c->NP, 1);
        unsigned char *tr = (unsigned char *)calloc(c->NP, 1);
        box_t bb = box_grow(c, 1 + B);
        FOR_BOX_PAR(bb, i, j, k) {
            long q = pidx(c, i, j, k);
            int t = is_troubled(c, Wp[q], Wp[(nd + 1) * c->NP + q]);
            if (c->p.hybrid_sensor && om[q] > c->p.sensor_thresh) t = 1;
            t0[q] = (unsigned char)t;
        }
        box_t b1 = box_grow(c, 1);
        FOR_BOX_PAR(b1, i, j, k) {
            int t = 0;
            for (int dk = nd > 2 ? -B : 0; dk <= (nd > 2 ? B : 0); ++dk)
                for (int dj = nd > 1 ? -B : 0; dj <= (nd > 1 ? B : 0); ++dj)
                    for (int di = -B; di <= B; ++di)
                        t |= t0[pidx(c, i + di, j + dj, k + dk)];
            tr[pidx(c, i, j, k)] = (unsigned char)t;
        }
        free(t0);
        lad_out lo;
        lad_fluxes(c, Wp, 2, LADF_NOPHYS, &lo);
        double *Fi = padded(c, nv);
        unsigned char *mask = (unsigned char *)calloc(c->NP, 1);
        for (int d = 0; d < nd; ++d) {
            long s = pstride(c, d);
            box_t b = box_grow(c, 0);
            b.lo[d] = -1;
            FOR_BOX_PAR(b, i, j, k) {
                long q = pidx(c, i, j, k);
                mask[q] = (unsigned char)(tr[q] || tr[q + s]);
            }
            gbr_dir_fluxes(c, Wp, Wd, om, d, mask, Fi);
            FOR_BOX_PAR(b, i, j, k) {
                long q = pidx(c, i, j, k);
                if (mask[q]) continue;
                for (int v = 0; v < nv; ++v) {
                    const double *f = lo.Fn[d] + v * c->NP;
                    Fi[v * c->NP + q] = (7.0 / 12.0) * (f[q] + f[q + s]) - (1.0 / 12.0) * (f[q - s] + f[q + 2 * s]);
                }
            }
            add_iface_diff(c, Fi, d, acc);
            if (iface_out && d == iface_dir) memcpy(iface_out, Fi, sizeof(double) * c->NP * nv);
            FOR_BOX(b, i, j, k) mask[pidx(c, i, j, k)] = 0;
        }
        free(Fi); free(mask); free(tr); free(om);
        free_lad(&lo, nd);
        for (int l = 0; l < nd; ++l) free(Wd[l]);
    }
}

static int stage_scheme(const ctx_t *c, const double *Wp)
{
    int s = c->p.scheme;
    if (s != ORC_HYBRID) return s;
    if (c->p.hybrid_mode == ORC_HYB_CELL) return -1; /* per-cell */
    /* Algorithm 3: the whole stage runs GBR-MEG6 if any cell is troubled, else LAD-E4 */
    return global_troubled(c, Wp) > 0 ? ORC_MEG6 : ORC_LAD_E4;
}

static void rhs_internal(const ctx_t *c, const double *U, double *R)
{
    ORC_REGION(residual);
    int nv = c->nv;
    double *Wp = padded_prims(c, U);
    double *acc = (double *)calloc((size_t)c->N * nv, sizeof(double));
    rhs_acc(c, Wp, stage_scheme(c, Wp), acc, NULL, 0);
    box_t b0 = box_grow(c, 0);
    FOR_BOX_PAR(b0, i, j, k) {
        long q = pidx(c, i, j, k), qi = iidx(c, i, j, k);
        for (int v = 0; v < nv; ++v) R[v * c->N + qi] = -(c->jac[q] * acc[v * c->N + qi]);
    }
    free(acc);
    free(Wp);
}

int orc_rhs(void *ctx, const double *U, double *R)
{
    rhs_internal((const ctx_t *)ctx, U, R);
    return 0;
}

int orc_iface_flux(void *ctx, const double *U, int d, double *F)
{
    const ctx_t *c = (const ctx_t *)ctx;
    int nv = c->nv;
    double *Wp = padded_prims(c, U);
    double *acc = (double *)calloc((size_t)c->N * nv, sizeof(double));
    double *Fi = padded(c, nv);
    int s = stage_scheme(c, Wp);
    if (s == ORC_LAD_E4 || s == ORC_LAD_C6) { free(acc); free(Fi); free(Wp); return -1; }
    rhs_acc(c, Wp, s, acc, Fi, d);
    /* layout [v][line][iface], lines ordered by the remaining dims (lowest first) */
    int n = c->n[d];
    long line = 0;
    box_t b = box_grow(c, 0);
    b.lo[d] = 0; b.hi[d] = 1;
    long nlines = c->N / n;
    long sd = pstride(c, d);
    FOR_BOX(b, i, j, k) {
        long q0 = pidx(c, i, j, k);
        for (int t = -1; t <= n - 1; ++t)
            for (int v = 0; v < nv; ++v)
                F[((long)v * nlines + line) * (n + 1) + (t + 1)] = Fi[v * c->NP + q0 + t * sd];
        ++line;
    }
    free(acc); free(Fi); free(Wp);
    return 0;
}

/* ------------------------------------------------------------------ */
/* implicit filter of the conserved state (LAD-C6, last RK stage)      */
/* ------------------------------------------------------------------ */
static void filter_state(const ctx_t *c, double *U)
{
    ORC_REGION(filter);
    int nd = c->nd, nv = c->nv;
    double *Qp = padded(c, nv);
    box_t b0 = box_grow(c, 0);
    FOR_BOX_PAR(b0, i, j, k) {
        long q = pidx(c, i, j, k), qi = iidx(c, i, j, k);
        for (int v = 0; v < nv; ++v) Qp[v * c->NP + q] = U[v * c->N + qi];
    }
    double *out = padded(c, nv);
    for (int d = 0; d < nd; ++d) {
        fill_ghosts(c, Qp, nv, 1);
        int n = c->n[d];
        int periodic = c->p.bc[d][0] == ORC_BC_PERIODIC;
        long s = pstride(c, d);
        box_t b = box_grow(c, 0);
        b.lo[d] = 0; b.hi[d] = 1;
        FOR_BOX_PAR(b, i0, j0, k0) {
            long q0 = pidx(c, i0, j0, k0);
            if (!c->p.curvilinear) {
                for (int v = 0; v < nv; ++v)
                    filter_line(n, periodic, c->p.alpha_f, Qp + v * c->NP + q0, s, out + v * c->NP + q0);
                continue;
            }
            /* curvilinear: the filter acts on the transformed conserved vector
             * Q/J, the quantity the discrete conservation law advances */
            int P = n + 2 * GH;
            double *ln = (double *)malloc(sizeof(double) * P), *lo = (double *)malloc(sizeof(double) * P);
            for (int v = 0; v < nv; ++v) {
                for (int t = -GH; t < n + GH; ++t) ln[t + GH] = Qp[v * c->NP + q0 + t * s] / c->jac[q0 + t * s];
                filter_line(n, periodic, c->p.alpha_f, ln + GH, 1, lo + GH);
                for (int t = 0; t < n; ++t) out[v * c->NP + q0 + t * s] = lo[t + GH] * c->jac[q0 + t * s];
            }
            free(ln); free(lo);
        }
        FOR_BOX_PAR(b0, i, j, k) {
            long q = pidx(c, i, j, k);
            for (int v = 0; v < nv; ++v) Qp[v * c->NP + q] = out[v * c->NP + q];
        }
    }
    FOR_BOX_PAR(b0, i, j, k) {
        long q = pidx(c, i, j, k), qi = iidx(c, i, j, k);
        for (int v = 0; v < nv; ++v) U[v * c->N + qi] = Qp[v * c->NP + q];
    }
    free(Qp); free(out);
}

int orc_filter(void *ctx, double *U)
{
    filter_state((const ctx_t *)ctx, U);
    return 0;
}

/* ------------------------------------------------------------------ */
/* TVD-RK3 (Shu & Osher)                                               */
/* ------------------------------------------------------------------ */
int orc_rk3_step(void *ctx, double *U, double dt)
{
    ORC_REGION(rk3);
    const ctx_t *c = (const ctx_t *)ctx;
    long M = c->N * c->nv;
    double *Un = (double *)malloc(sizeof(double) * M), *R = (double *)malloc(sizeof(double) * M);
    double *Us = (double *)malloc(sizeof(double) * M);
    memcpy(Un, U, sizeof(double) * M);
    rhs_internal(c, Un, R);
    ORC_PAR_FOR(M)
    for (long q = 0; q < M; ++q) Us[q] = Un[q] + dt * R[q];
    rhs_internal(c, Us, R);
    ORC_PAR_FOR(M)
    for (long q = 0; q < M; ++q) Us[q] = 0.75 * Un[q] + 0.25 * (Us[q] + dt * R[q]);
    rhs_internal(c, Us, R);
    ORC_PAR_FOR(M)
    for (long q = 0; q < M; ++q) U[q] = (1.0 / 3.0) * Un[q] + (2.0 / 3.0) * (Us[q] + dt * R[q]);
    if (c->p.scheme == ORC_LAD_C6 && c->p.filter_on) filter_state(c, U);
    free(Un); free(R); free(Us);
    return 0;
}

/* ------------------------------------------------------------------ */
/* CFL time step (reading: unsplit sum of directional spectral radii)  */
/* ------------------------------------------------------------------ */
double orc_cfl_dt(void *ctx, const double *U)
{
    ORC_REGION(cfl);
    const ctx_t *c = (const ctx_t *)ctx;
    int nd = c->nd, nv = c->nv;
    double mx = 0.0;
    box_t b0 = box_grow(c, 0);
    FOR_BOX(b0, i, j, k) {
        long q = pidx(c, i, j, k), qi = iidx(c, i, j, k);
        double Q[5], W[5];
        for (int v = 0; v < nv; ++v) Q[v] = U[v * c->N + qi];
        cons_to_prim(nd, c->p.gamma, Q, W);
        double cs = sqrt(c->p.gamma * W[nd + 1] / W[0]);
        double s = 0.0;
        for (int l = 0; l < nd; ++l) {
            double dot = 0.0, mag = 0.0;
            for (int m = 0; m < nd; ++m) {
                dot += c->xh[l][m][q] * W[1 + m];
                mag += c->xh[l][m][q] * c->xh[l][m][q];
            }
            s += fabs(dot) + cs * sqrt(mag);
        }
        double r = c->jac[q] * s;
        if (r > mx) mx = r;
    }
    return c->p.cfl / mx;
}

long orc_hybrid_flag(void *ctx, const double *U)
{
    const ctx_t *c = (const ctx_t *)ctx;
    double *Wp = padded_prims(c, U);
    long cnt = global_troubled(c, Wp);
    free(Wp);
    if (c->p.hybrid_mode == ORC_HYB_GLOBAL) return cnt > 0 ? 1 : 0;
    return cnt;
}

int orc_omega(void *ctx, const double *U, double *omega)
{
    const ctx_t *c = (const ctx_t *)ctx;
    int nd = c->nd, nv = c->nv;
    double *Wp = padded_prims(c, U);
    double *Wd[3] = {NULL, NULL, NULL};
    int kind = c->p.scheme == ORC_MIG4 ? 1 : 0;
    for (int l = 0; l < nd; ++l) {
        Wd[l] = padded(c, nv);
        grad_field(c, Wp, nv, l, kind, Wd[l]);
    }
    double *om = padded(c, 1);
    omega_field(c, Wp, Wd, om);
    box_t b0 = box_grow(c, 0);
    FOR_BOX(b0, i, j, k) omega[iidx(c, i, j, k)] = om[pidx(c, i, j, k)];
    free(om); free(Wp);
    for (int l = 0; l < nd; ++l) free(Wd[l]);
    return 0;
}

int orc_lad_coeffs(void *ctx, const double *U, double *beta, double *kappa)
{
    const ctx_t *c = (const ctx_t *)ctx;
    double *Wp = padded_prims(c, U);
    lad_out lo;
    lad_fluxes(c, Wp, c->p.scheme == ORC_LAD_C6 ? 3 : 2, LADF_NOPHYS, &lo);
    box_t b0 = box_grow(c, 0);
    FOR_BOX(b0, i, j, k) {
        beta[iidx(c, i, j, k)] = lo.beta[pidx(c, i, j, k)];
        kappa[iidx(c, i, j, k)] = lo.kappa[pidx(c, i, j, k)];
    }
    free_lad(&lo, c->nd);
    free(Wp);
    return 0;
}

/* ------------------------------------------------------------------ */
/* metrics                                                             */
/* Cartesian: xi_hat = diag(product of the other spacings), J = 1/vol. */
/* Curvilinear: node metrics from derivatives D of the node            */
/* coordinates, with D the scheme's own explicit first derivative      */
/* (sixth order for C-GBR, E4 for LAD-E4 and the hybrid), so that the  */
/* discrete metric identities hold for the flux divergence actually    */
/* used (freestream preservation):                                     */
/* 2D: xi_x = y_eta, xi_y = -x_eta, eta_x = -y_xi, eta_y = x_xi;        */
/* 3D: conservative (Thomas-Lombard) form xi_x = (y_eta z)_zeta -       */
/* (y_zeta z)_eta and cyclic permutations.  Interface metrics are the  */
/* flux-form interpolant H of the node metrics along the interface     */
/* direction, with D = difference of H:                                */
/*  six:  H f_{i+1/2} = 37/60 (f_i+f_{i+1}) - 8/60 (f_{i-1}+f_{i+2})    */
/*                    + 1/60 (f_{i-2}+f_{i+3})                         */
/*  four: H f_{i+1/2} = 7/12 (f_i+f_{i+1}) - 1/12 (f_{i-1}+f_{i+2})     */
/* ------------------------------------------------------------------ */
typedef struct { int nd, n[3], ge[3], PE[3]; long NE; } ebox_t;
static long eidx(const ebox_t *e, int i, int j, int k)
{
    return (long)(i + e->ge[0]) + (long)e->PE[0] * ((long)(j + e->ge[1]) + (long)e->PE[1] * (long)(k + e->ge[2]));
}
static long estride(const ebox_t *e, int d)
{
    if (d == 0) return 1;
    if (d == 1) return e->PE[0];
    return (long)e->PE[0] * e->PE[1];
}
static double *ealloc(const ebox_t *e)
{
    double *f = (double *)malloc(sizeof(double) * e->NE);
    for (long q = 0; q < e->NE; ++q) f[q] = NAN;
    return f;
}
/* op 0: derivative D at nodes; op 1: interpolant H at i+1/2 stored at i.
 * six = 1: sixth-order pair, six = 0: fourth-order (E4) pair. */
static double *eop(const ebox_t *e, const double *f, int d, int op, int six)
{
    double *o = ealloc(e);
    long s = estride(e, d);
    int lo[3], hi[3];
    for (int a = 0; a < 3; ++a) { lo[a] = -e->ge[a]; hi[a] = e->n[a] + e->ge[a]; }
    int r = six ? 3 : 2;
    for (int k = lo[2]; k < hi[2]; ++k)
        for (int j = lo[1]; j < hi[1]; ++j)
            for (int i = lo[0]; i < hi[0]; ++i) {
                int pos[3] = {i, j, k};
                int t = pos[d];
                long q = eidx(e, i, j, k);
                if (op == 0) {
                    if (t - r < lo[d] || t + r >= hi[d]) continue;
                    if (isnan(f[q - r * s]) || isnan(f[q + r * s])) continue;
                    o[q] = six ? op_meg6(f + q, s) : op_e4(f + q, s);
                } else {
                    if (t - r + 1 < lo[d] || t + r >= hi[d]) continue;
                    if (isnan(f[q - (r - 1) * s]) || isnan(f[q + r * s])) continue;
                    if (six)
                        o[q] = (37.0 / 60.0) * (f[q] + f[q + s]) - (8.0 / 60.0) * (f[q - s] + f[q + 2 * s]) +
                               (1.0 / 60.0) * (f[q - 2 * s] + f[q + 3 * s]);
                    else
                        o[q] = (7.0 / 12.0) * (f[q] + f[q + s]) - (1.0 / 12.0) * (f[q - s] + f[q + 2 * s]);
                }
            }
    return o;
}

/* Compact sixth-order (C6) derivative along d on the extended box: the
 * operator of the LAD-C6 flux divergence, so that the metric identities hold
 * for it (reading: the compact operator inside the metrics).  Non-periodic d:
 * the system on nodes [0, n-1] with explicit E4 rows at both ends (reading f
 * at -2 .. n+1), the E4 derivative at the other extended nodes (used only by
 * the chain rule at ghost nodes).  Periodic d: the cyclic system on [0, n-1]
 * applied to f minus its linear trend along the line (detrend = 1, for a
 * coordinate: T = f_n - f_0, its period translation), plus T/n; the
 * extended nodes by wrapping. */
static double *eop_c6(const ebox_t *e, const double *f, int d, int periodic, int detrend)
{
    double *o = eop(e, f, d, 0, 0);
    long s = estride(e, d);
    int n = e->n[d], g = e->ge[d];
    int lo[3], hi[3];
    for (int a = 0; a < 3; ++a) { lo[a] = -e->ge[a]; hi[a] = e->n[a] + e->ge[a]; }
    lo[d] = 0; hi[d] = 1;
    double *gl = (double *)malloc(sizeof(double) * (n + 4)), *og = (double *)malloc(sizeof(double) * (n + 4));
    for (int k = lo[2]; k < hi[2]; ++k)
        for (int j = lo[1]; j < hi[1]; ++j)
            for (int i = lo[0]; i < hi[0]; ++i) {
                long q0 = eidx(e, i, j, k);
                int ok = 1;
                for (int t = -2; t <= n + 1; ++t) ok = ok && !isnan(f[q0 + t * s]);
                if (!ok) continue;
                if (!periodic) {
                    compact_line(3, n, 0, 0, n - 1, f + q0, s, o + q0);
                    continue;
                }
                double T = detrend ? f[q0 + (long)n * s] - f[q0] : (double)0.0;
                for (int t = -2; t <= n + 1; ++t) gl[t + 2] = f[q0 + t * s] - T * (double)t / (double)n;
                compact_line(3, n, 1, 0, n - 1, gl + 2, 1, og + 2);
                for (int t = 0; t < n; ++t) o[q0 + t * s] = og[t + 2] + T / (double)n;
                for (int t = 1; t <= g; ++t) {
                    o[q0 - t * s] = o[q0 + imod(-t, n) * s];
                    o[q0 + (n - 1 + t) * s] = o[q0 + imod(n - 1 + t, n) * s];
                }
            }
    free(gl); free(og);
    return o;
}

static void metrics_curvilinear(ctx_t *c, const double *xyz)
{
    ORC_REGION(metrics);
    int nd = c->nd;
    int six = (c->p.scheme == ORC_MEG6 || c->p.scheme == ORC_MIG4);
    int c6 = c->p.scheme == ORC_LAD_C6;
    ebox_t e;
    e.nd = nd;
    e.NE = 1;
    for (int d = 0; d < 3; ++d) {
        e.n[d] = c->n[d];
        e.ge[d] = d < nd ? GC : 0;
        e.PE[d] = e.n[d] + 2 * e.ge[d];
        e.NE *= e.PE[d];
    }
    /* extended coordinates: linear extrapolation beyond non-periodic ends,
     * periodic translation across periodic ones */
    double *X[3] = {NULL, NULL, NULL};
    for (int m = 0; m < nd; ++m) {
        X[m] = ealloc(&e);
        for (int k = 0; k < c->n[2]; ++k)
            for (int j = 0; j < c->n[1]; ++j)
                for (int i = 0; i < c->n[0]; ++i)
                    X[m][eidx(&e, i, j, k)] = xyz[(long)m * c->N + iidx(c, i, j, k)];
    }
    for (int d = 0; d < nd; ++d) {
        int n = c->n[d];
        int lo[3], hi[3];
        for (int a = 0; a < 3; ++a) {
            if (a < d) { lo[a] = -e.ge[a]; hi[a] = e.n[a] + e.ge[a]; }
            else { lo[a] = 0; hi[a] = e.n[a]; }
        }
        lo[d] = 0; hi[d] = 1;
        long s = estride(&e, d);
        int periodic = c->p.bc[d][0] == ORC_BC_PERIODIC;
        for (int k = lo[2]; k < hi[2]; ++k)
            for (int j = lo[1]; j < hi[1]; ++j)
                for (int i = lo[0]; i < hi[0]; ++i) {
                    long q0 = eidx(&e, i, j, k);
                    for (int m = 0; m < nd; ++m) {
                        double *x = X[m] + q0;
                        for (int t = 1; t <= GC; ++t) {
                            if (periodic) {
                                int a = -t, b = n - 1 + t;
                                x[a * s] = x[imod(a, n) * s] + (double)idiv_floor(a, n) * c->p.period[d][m];
                                x[b * s] = x[imod(b, n) * s] + (double)idiv_floor(b, n) * c->p.period[d][m];
                            } else {
                                x[-t * s] = x[0] + (double)t * (x[0] - x[s]);
                                x[(n - 1 + t) * s] = x[(n - 1) * s] + (double)t * (x[(n - 1) * s] - x[(n - 2) * s]);
                            }
                        }
                    }
                }
    }
    /* node derivatives dX[l][m] = D_l x_m (LAD-C6: its own compact operator) */
    int per[3];
    for (int d = 0; d < 3; ++d) per[d] = d < nd && c->p.bc[d][0] == ORC_BC_PERIODIC;
#define MOP(f, d) (c6 ? eop_c6(&e, (f), (d), per[d], 1) : eop(&e, (f), (d), 0, six))
    double *dX[3][3];
    for (int l = 0; l < nd; ++l)
        for (int m = 0; m < nd; ++m) dX[l][m] = MOP(X[m], l);
    double *node[3][3], *ifc[3][3], *vol = ealloc(&e);
    for (int l = 0; l < 3; ++l) for (int m = 0; m < 3; ++m) { node[l][m] = NULL; ifc[l][m] = NULL; }
    if (nd == 1) {
        node[0][0] = ealloc(&e);
        for (long q = 0; q < e.NE; ++q) { node[0][0][q] = 1.0; vol[q] = dX[0][0][q]; }
    } else if (nd == 2) {
        for (int l = 0; l < 2; ++l) for (int m = 0; m < 2; ++m) node[l][m] = ealloc(&e);
        for (long q = 0; q < e.NE; ++q) {
            node[0][0][q] = dX[1][1][q];
            node[0][1][q] = -dX[1][0][q];
            node[1][0][q] = -dX[0][1][q];
            node[1][1][q] = dX[0][0][q];
            vol[q] = dX[0][0][q] * dX[1][1][q] - dX[1][0][q] * dX[0][1][q];
        }
    } else {
        /* Thomas-Lombard conservative form, (a, b) = (m+1, m+2) mod 3:
         * xi_hat[l][m] = D_{l2}((D_{l1} x_a) x_b) - D_{l1}((D_{l2} x_a) x_b).
         * LAD-C6 (cyclic compact operator along periodic directions): x_b is
         * split into its periodic part and its linear trend s[d][b] k_d across
         * periodic directions d; the trend's terms are exactly
         * (D_{l1} x_a) s[l2][b] - (D_{l2} x_a) s[l1][b], and they cancel in the
         * metric identities as the periodic part's do. */
        double slope[3][3];
        for (int d = 0; d < 3; ++d)
            for (int b = 0; b < 3; ++b) slope[d][b] = c6 && per[d] ? c->p.period[d][b] / (double)c->n[d] : (double)0.0;
        double *Xp[3];
        for (int b = 0; b < 3; ++b) {
            Xp[b] = X[b];
            if (!c6) continue;
            Xp[b] = ealloc(&e);
            for (int k = -e.ge[2]; k < e.n[2] + e.ge[2]; ++k)
                for (int j = -e.ge[1]; j < e.n[1] + e.ge[1]; ++j)
                    for (int i = -e.ge[0]; i < e.n[0] + e.ge[0]; ++i) {
                        long q = eidx(&e, i, j, k);
                        Xp[b][q] = ((X[b][q] - slope[0][b] * (double)i) - slope[1][b] * (double)j) - slope[2][b] * (double)k;
                    }
        }
        double *Pp[3][3];
        for (int lp = 0; lp < 3; ++lp)
            for (int m = 0; m < 3; ++m) {
                int a = (m + 1) % 3, b = (m + 2) % 3;
                Pp[lp][m] = ealloc(&e);
                for (long q = 0; q < e.NE; ++q) Pp[lp][m][q] = dX[lp][a][q] * Xp[b][q];
            }
        for (int l = 0; l < 3; ++l) {
            int l1 = (l + 1) % 3, l2 = (l + 2) % 3;
            for (int m = 0; m < 3; ++m) {
                int a = (m + 1) % 3, b = (m + 2) % 3;
                double *A = c6 ? eop_c6(&e, Pp[l1][m], l2, per[l2], 0) : MOP(Pp[l1][m], l2);
                double *B = c6 ? eop_c6(&e, Pp[l2][m], l1, per[l1], 0) : MOP(Pp[l2][m], l1);
                node[l][m] = ealloc(&e);
                for (long q = 0; q < e.NE; ++q) node[l][m][q] = A[q] - B[q];
                if (c6)
                    for (long q = 0; q < e.NE; ++q)
                        node[l][m][q] = (node[l][m][q] + dX[l1][a][q] * slope[l2][b]) - dX[l2][a][q] * slope[l1][b];
                free(A); free(B);
            }
        }
        if (c6) for (int b = 0; b < 3; ++b) free(Xp[b]);
        for (long q = 0; q < e.NE; ++q) {
            double a11 = dX[0][0][q], a12 = dX[1][0][q], a13 = dX[2][0][q];
            double a21 = dX[0][1][q], a22 = dX[1][1][q], a23 = dX[2][1][q];
            double a31 = dX[0][2][q], a32 = dX[1][2][q], a33 = dX[2][2][q];
            vol[q] = a11 * (a22 * a33 - a23 * a32) - a12 * (a21 * a33 - a23 * a31) + a13 * (a21 * a32 - a22 * a31);
        }
        for (int lp = 0; lp < 3; ++lp) for (int m = 0; m < 3; ++m) free(Pp[lp][m]);
    }
    for (int l = 0; l < nd; ++l)
        for (int m = 0; m < nd; ++m) ifc[l][m] = eop(&e, node[l][m], l, 1, six);
    /* copy onto the padded box */
    box_t bp = box_grow(c, GH);
    FOR_BOX(bp, i, j, k) {
        long q = pidx(c, i, j, k), qe = eidx(&e, i, j, k);
        for (int l = 0; l < nd; ++l)
            for (int m = 0; m < nd; ++m) {
                c->xh[l][m][q] = node[l][m][qe];
                c->xt[l][m][q] = ifc[l][m][qe];
                long s = estride(&e, l);
                c->dxl[l][m][q] = 0.5 * (X[m][qe + s] - X[m][qe - s]);
            }
        c->jac[q] = 1.0 / vol[qe];
    }
    for (int l = 0; l < nd; ++l)
        for (int m = 0; m < nd; ++m) { free(dX[l][m]); free(node[l][m]); free(ifc[l][m]); }
    for (int m = 0; m < nd; ++m) free(X[m]);
    free(vol);
#undef MOP
}

void *orc_create(const orc_params *p, const double *xyz)
{
    ctx_t *c = (ctx_t *)calloc(1, sizeof(ctx_t));
    c->p = *p;
    c->nd = p->ndim;
    c->nv = p->ndim + 2;
    c->N = 1;
    c->NP = 1;
    for (int d = 0; d < 3; ++d) {
        c->n[d] = d < c->nd ? p->n[d] : 1;
        c->g[d] = d < c->nd ? GH : 0;
        c->P[d] = c->n[d] + 2 * c->g[d];
        c->N *= c->n[d];
        c->NP *= c->P[d];
    }
    for (int l = 0; l < 3; ++l)
        for (int m = 0; m < 3; ++m) {
            c->xh[l][m] = padded(c, 1);
            c->xt[l][m] = padded(c, 1);
            c->dxl[l][m] = padded(c, 1);
        }
    c->jac = padded(c, 1);
    if (!p->curvilinear || xyz == NULL) {
        double h0 = p->h[0], h1 = p->h[1], h2 = p->h[2];
        double diag[3] = {1.0, 1.0, 1.0}, J = 1.0;
        if (c->nd == 1) { diag[0] = 1.0; J = 1.0 / h0; }
        if (c->nd == 2) { diag[0] = h1; diag[1] = h0; J = 1.0 / (h0 * h1); }
        if (c->nd == 3) { diag[0] = h1 * h2; diag[1] = h0 * h2; diag[2] = h0 * h1; J = 1.0 / (h0 * h1 * h2); }
        for (long q = 0; q < c->NP; ++q) {
            for (int l = 0; l < c->nd; ++l)
                for (int m = 0; m < c->nd; ++m) {
                    c->xh[l][m][q] = l == m ? diag[l] : (double)0.0;
                    c->xt[l][m][q] = l == m ? diag[l] : (double)0.0;
                    c->dxl[l][m][q] = l == m ? p->h[l] : (double)0.0;
                }
            c->jac[q] = J;
        }
    } else {
        metrics_curvilinear(c, xyz);
    }
    return c;
}

int orc_set_inflow_profile(void *ctx, int d, int side, const double *W)
{
    ctx_t *c = (ctx_t *)ctx;
    if (d < 0 || d >= c->nd || side < 0 || side > 1 || c->p.bc[d][side] != ORC_BC_INFLOW) return -1;
    long face = c->N / c->n[d];
    free(c->prof[d][side]);
    c->prof[d][side] = (double *)malloc(sizeof(double) * (size_t)(face * c->nv));
    memcpy(c->prof[d][side], W, sizeof(double) * (size_t)(face * c->nv));
    return 0;
}

void orc_destroy(void *ctx)
{
    ctx_t *c = (ctx_t *)ctx;
    if (!c) return;
    for (int l = 0; l < 3; ++l)
        for (int m = 0; m < 3; ++m) { free(c->xh[l][m]); free(c->xt[l][m]); free(c->dxl[l][m]); }
    for (int d = 0; d < 3; ++d) { free(c->prof[d][0]); free(c->prof[d][1]); }
    free(c->jac);
    free(c);
}

int orc_metrics(void *ctx, double *node, double *iface)
{
    const ctx_t *c = (const ctx_t *)ctx;
    int nd = c->nd;
    box_t b0 = box_grow(c, 0);
    FOR_BOX(b0, i, j, k) {
        long q = pidx(c, i, j, k), qi = iidx(c, i, j, k);
        for (int l = 0; l < nd; ++l)
            for (int m = 0; m < nd; ++m) {
                node[(l * nd + m) * c->N + qi] = c->xh[l][m][q];
                if (iface) iface[(l * nd + m) * c->N + qi] = c->xt[l][m][q];
            }
        node[nd * nd * c->N + qi] = c->jac[q];
    }
    return 0;
}

int orc_set_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
    return omp_get_max_threads();
#else
    (void)n;
    return 1;
#endif
}
