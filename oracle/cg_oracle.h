/*
 * Plain FP64 CPU oracle of the compressible-flow right-hand side (RHS) of
 * Kumar, Saini, Vadlamani & Chamarthi, "Assessment of gradient-based
 * reconstruction and artificial diffusivity methods in simulating high-speed
 * compressible flows" (arXiv 2511.18042).
 *
 * TEST INFRASTRUCTURE ONLY. Nothing in the product path may include, link or
 * call this code; only the tests, the smoke check and the CPU-baseline leg of
 * the benchmark do. It shares no code, header or constant table with the CUDA
 * library.
 *
 * Every array is FP64, structure-of-arrays: nv = ndim + 2 planes of
 * n0*n1*n2 nodes, index i + n0*(j + n1*k), no ghost nodes.  Conserved order:
 * (rho, rho*u_0 .. rho*u_{ndim-1}, E) with E the total energy per unit volume
 * (Sec. 2.1, governing equations; reading: E per volume).
 */
#ifndef CG_ORACLE_H
#define CG_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

/* ORC_BC_WALL: no-slip isothermal wall at the boundary face (Sec. 3.3: the
 * compression ramps); a supersonic outflow is ORC_BC_EXTRAP. */
enum { ORC_BC_PERIODIC = 0, ORC_BC_EXTRAP = 1, ORC_BC_REFLECT = 2, ORC_BC_INFLOW = 3, ORC_BC_WALL = 4 };
enum { ORC_MEG6 = 0, ORC_MIG4 = 1, ORC_LAD_E4 = 2, ORC_LAD_C6 = 3, ORC_HYBRID = 4 };
enum { ORC_HYB_GLOBAL = 0, ORC_HYB_CELL = 1 };

typedef struct {
    int ndim;                 /* 1, 2 or 3 */
    int n[3];                 /* interior nodes per direction (1 for unused) */
    int bc[3][2];             /* boundary type per direction and side */
    double inflow[3][2][5];   /* primitive (rho, u_0.., p) for ORC_BC_INFLOW faces */
    int curvilinear;          /* 0: uniform Cartesian spacing h; 1: node coordinates */
    double h[3];
    double period[3][3];      /* translation of the coordinates across a periodic direction */
    double gamma, minf;       /* EOS p = rho*T/(gamma*minf^2) */
    int scheme;               /* ORC_MEG6 .. ORC_HYBRID */
    int hybrid_mode;          /* ORC_HYB_GLOBAL or ORC_HYB_CELL */
    int hybrid_sensor;        /* per-cell mode: also flag nodes with Omega > sensor_thresh */
    double hyb_rho, hyb_p;    /* troubled if rho < hyb_rho or p < hyb_p */
    double cfl, c_beta, c_kappa, alpha_f, sensor_thresh, mp_eps, mp_alpha;
    int read_mp_printed;      /* entropy wave: criterion exactly as printed (product <= eps -> MP5) */
    int read_acoustic_mp5;    /* acoustic waves always MP5-limited */
    int omega_window;         /* interface sensor = max of Omega over nodes i-w+1..i+w (1..4) */
    int positivity_fallback;  /* first-order interface states when rho or p <= 0 */
    int filter_on;            /* LAD-C6: implicit filter after the last RK stage */
    /* Physical viscosity (Sec. 2.1, Eq. 3): mu_hat = mu(T)/Re with the
     * Sutherland law mu(T) = T^{3/2} (1 + S)/(T + S) (T, S in units of
     * T_inf), Stokes' hypothesis, kappa_hat = mu_hat/((gamma-1) Pr M^2). */
    int viscous;
    double re, pr;
    double suth;              /* Sutherland constant S / T_inf */
    double twall;             /* temperature of ORC_BC_WALL faces (units of T_inf) */
    int hybrid_buffer;        /* per-cell mode: a troubled node also marks the nodes within
                                 this many nodes (0: the node alone) */
} orc_params;

/* Context: holds the metrics (computed from the coordinates for curvilinear
 * grids; LAD-C6 with its own compact operator).  xyz: ndim planes of node
 * coordinates, or NULL for Cartesian. */
void *orc_create(const orc_params *p, const double *xyz);
void orc_destroy(void *ctx);

/* R = -J * sum_l (F_{l,i+1/2} - F_{l,i-1/2})  (GBR) or -J * sum_l D_l F_l (LAD). */
int orc_rhs(void *ctx, const double *U, double *R);
/* One TVD-RK3 step in place (plus the LAD-C6 filter when enabled). */
int orc_rk3_step(void *ctx, double *U, double dt);
/* dt = cfl / max_i J*sum_l(|xi_l.u| + c|xi_l|) */
double orc_cfl_dt(void *ctx, const double *U);
/* Hybrid: scheme the stage would use (0 LAD, 1 GBR) in global mode, or the
 * number of troubled nodes (interior) in per-cell mode. */
long orc_hybrid_flag(void *ctx, const double *U);
/* Diagnostics on interior nodes. */
int orc_omega(void *ctx, const double *U, double *omega);
int orc_lad_coeffs(void *ctx, const double *U, double *beta, double *kappa);
int orc_filter(void *ctx, double *U);
/* Metrics: node planes xh[l][m] (ndim*ndim) then J; interface planes xt[l][m]
 * at interface i+1/2 along l stored at node i (interior nodes). */
int orc_metrics(void *ctx, double *node, double *iface);
/* Interface fluxes along direction d for all interior lines, interfaces
 * i = -1..n_d-1 (n_d+1 per line), layout [v][line][iface]. */
int orc_iface_flux(void *ctx, const double *U, int d, double *F);

/* Building blocks (exposed for the pins). */
void orc_hllc(int ndim, double gamma, const double *WL, const double *WR,
              const double *xi, double *F);
void orc_euler_flux(int ndim, double gamma, const double *W, const double *xi, double *F);
/* Characteristic transform at the interface between nodes with primitive
 * states Wi, Wi1 and interface metrics xi (Sec. 2.3): inverse = 0: out = L in
 * (primitive -> characteristic); inverse = 1: out = R in. */
void orc_char_transform(int nd, double gamma, const double *Wi, const double *Wi1,
                        const double *xi, int inverse, const double *in, double *out);
double orc_mp5(double um2, double um1, double u0, double up1, double up2,
               double alpha, double eps);
/* Derivative / filter operators on one line of n values with ng ghost values
 * on each side (array length n + 2*ng).  kind: 0 MEG6, 1 MIG4, 2 E4, 3 C6,
 * 4 Gaussian (truncated, 9 points), 5 implicit 8th-order filter.
 * periodic: 1 for a cyclic line.  out has the same layout (n + 2*ng). */
int orc_line_op(int kind, int n, int ng, int periodic, double alpha_f,
                const double *in, double *out);
/* Tridiagonal solve with constant off-diagonal a, unit diagonal, cyclic or not
 * (rows 0 and n-1 decoupled when not cyclic).  Used by the pins. */
void orc_tridiag(int n, double a, int cyclic, const double *rhs, double *x);
/* Inflow face (d, side) holds a per-node primitive profile instead of the
 * constant state: W has nv planes over the face's nodes (the other active
 * directions, lowest first, e.g. j + n1*k for d = 0).  Ghost nodes of the face
 * at any depth take the profile of their transverse position (clamped to the
 * face).  Copied; returns 0, or -1 if the face is not an inflow face. */
int orc_set_inflow_profile(void *ctx, int d, int side, const double *W);
/* Threads of the OpenMP build for the grid loops (n <= 0: unchanged); returns
 * the count in use (1 without OpenMP).  Results do not depend on it. */
int orc_set_threads(int n);

#ifdef __cplusplus
}
#endif
#endif
