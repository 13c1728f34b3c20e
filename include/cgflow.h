/*
 * cgflow: GB300-native right-hand side of the compressible Euler equations in
 * curvilinear form with the shock-capturing families assessed in
 * Kumar, Saini, Vadlamani & Chamarthi, arXiv 2511.18042:
 *   C-GBR  centralised gradient-based reconstruction (MEG6 explicit / MIG4
 *          compact gradients, MP5 limiting, wave-appropriate sensor, HLLC),
 *          Sec. 2.3, Eq. (7)-(10);
 *   LAD    local artificial diffusivity (E4 explicit / C6 compact central
 *          differences, artificial bulk viscosity and conductivity smoothed by
 *          a truncated Gaussian, implicit filter for C6), Sec. 2.2, Eq. (4)-(6);
 *   HYBRID LAD-GBR switching on troubled cells, Sec. 5, Algorithm 3 (whole
 *          stage) or per interface.
 * plus TVD-RK3 time stepping (Sec. 2.1, Sec. 4 Algorithms 1-2), the CFL time
 * step (Sec. 3) and grid metrics on the device (Sec. 2.1, Eq. 1-2).
 *
 * Conventions (every entry point):
 *  - Arrays are FP64, device memory unless the name says _host, structure of
 *    arrays: nv = ndim + 2 planes of n0*n1*n2 nodes, node (i,j,k) at
 *    i + n0*(j + n1*k), no ghost nodes.  Conserved order (rho, rho*u_0, ..,
 *    rho*u_{ndim-1}, E), E the total energy per unit volume.  Caller-owned;
 *    borrowed for the duration of the call (stream-ordered).
 *  - stream: a cudaStream_t passed as void* (NULL = legacy default stream).
 *    All work is enqueued on it; calls return before the GPU finishes unless
 *    stated otherwise.
 *  - Return: 0 (CG_OK) or a negative cg_status; cg_last_error() gives a
 *    thread-local message.  No exception crosses the interface.
 *  - Handles own their device scratch (allocated at create, freed at destroy).
 *    One handle must not be used from two threads at once; separate handles
 *    are independent.
 */
#ifndef CGFLOW_H
#define CGFLOW_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define CG_API __attribute__((visibility("default")))

typedef enum {
    CG_OK = 0,
    CG_ERR_INVALID_ARG = -1,
    CG_ERR_CUDA = -2,
    CG_ERR_OOM = -3,
    CG_ERR_NONPHYSICAL = -4, /* rho <= 0, p <= 0 or NaN produced; see cg_last_bad_index */
    CG_ERR_UNSUPPORTED = -5,
    CG_ERR_TIMEOUT = -6
} cg_status;

/* CG_BC_WALL: isothermal no-slip wall at the boundary face (the compression
 * ramps of Sec. 3.3); ghost nodes mirror the interior with every velocity
 * component negated, the pressure kept and T_ghost = 2 twall - T.  A
 * supersonic outflow is CG_BC_EXTRAP. */
typedef enum { CG_BC_PERIODIC = 0, CG_BC_EXTRAP = 1, CG_BC_REFLECT = 2, CG_BC_INFLOW = 3, CG_BC_WALL = 4 } cg_bc;
typedef enum { CG_MEG6 = 0, CG_MIG4 = 1, CG_LAD_E4 = 2, CG_LAD_C6 = 3, CG_HYBRID = 4 } cg_scheme;
typedef enum { CG_HYBRID_GLOBAL = 0, CG_HYBRID_CELL = 1 } cg_hybrid_mode;
typedef enum { CG_FP64 = 0, CG_MIXED = 1 } cg_precision;

typedef struct cg_grid cg_grid;
typedef struct cg_solver cg_solver;

/* Scheme parameters (Sec. 2.2-2.3, Sec. 3 "CFL 0.2", Sec. 5 thresholds). */
typedef struct {
    double gamma;         /* ratio of specific heats */
    double minf;          /* reference Mach number in p = rho T / (gamma minf^2) */
    int scheme;           /* cg_scheme */
    int precision;        /* cg_precision */
    int hybrid_mode;      /* cg_hybrid_mode (scheme == CG_HYBRID) */
    int hybrid_sensor;    /* per-interface mode: nodes with Omega > sensor_thresh are troubled too */
    double hyb_rho;       /* troubled where rho < hyb_rho (-inf: never) */
    double hyb_p;         /* troubled where p < hyb_p   (-inf: never) */
    double cfl;           /* Courant number of cg_cfl_dt */
    double c_beta, c_kappa; /* LAD coefficients C_beta, C_kappa (Eq. 4-5) */
    double alpha_f;       /* implicit filter parameter (LAD-C6) */
    double sensor_thresh; /* Omega threshold of Eq. (8), 0.01 */
    double mp_eps;        /* MP tolerance of Eq. (8), 1e-20 */
    double mp_alpha;      /* MP5 alpha (Suresh & Huynh), 4 */
    int filter_on;        /* LAD-C6: implicit filter after the last RK stage */
    int omega_window;     /* interface sensor window half-width w (1..4): max over nodes i-w+1..i+w */
    double inflow[3][2][5]; /* primitive (rho, u.., p) held on CG_BC_INFLOW faces [dir][side] */
    /* Physical viscosity (Sec. 2.1, Eq. 3): mu_hat = mu(T) / re with
     * Sutherland's law mu(T) = T^{3/2} (1 + suth) / (T + suth) (T in units of
     * T_inf), Stokes' hypothesis, kappa_hat = mu_hat / ((gamma-1) pr minf^2).
     * LAD schemes add it to their node fluxes; C-GBR and the per-interface
     * hybrid add an E4 central pass of node viscous fluxes. */
    int viscous;          /* 0: inviscid */
    double re, pr;        /* Reynolds number (reference length 1), Prandtl number */
    double suth;          /* Sutherland constant S / T_inf */
    double twall;         /* temperature of CG_BC_WALL faces (units of T_inf) */
    /* FP64 C-GBR interface sweep.  0 (default): every expression in the
     * oracle's operation order, no a*b+c contracted (bitwise reproducible).
     * 1: multiply-adds fused (16 % fewer FP64 instructions in the sweep);
     * results agree to rounding, except where a value sits at a threshold of
     * the selection (Eq. 8) and the branch flips: on the 1792x768 triple point
     * the per-interface hybrid then differs by ~1e-11 after one step.  Other
     * kernels are always exact. */
    int fma_sweep;
    /* Per-interface hybrid: a troubled node also marks every node within
     * hybrid_buffer nodes of it in each direction (0..2; 0, the default, marks
     * the node alone).  A buffer of 1 keeps the C-GBR flux on the LAD-E4 side
     * of a troubled region, where LAD-E4 alone (no artificial shear viscosity)
     * lets an expanding vortex sheet drain the density to zero. */
    int hybrid_buffer;
} cg_params;

/* Fills the defaults: gamma 1.4, minf 1, MEG6, FP64, CFL 0.2, C_beta 1.75,
 * C_kappa 0.01, alpha_f 0.45, Omega threshold 0.01, MP eps 1e-20, alpha 4,
 * window 4, filter on, no hybrid thresholds, inviscid (re 1, pr 0.72,
 * suth 0, twall 1), exact FP64 sweep (fma_sweep 0), no hybrid buffer. */
CG_API void cg_params_default(cg_params *p);

/* Uniform Cartesian grid, node spacing h[d] (Sec. 2.1 with x = xi h).
 * n[d] >= 8 for non-periodic directions, >= 1 otherwise; unused directions 1.
 * bc[2*d + side]: cg_bc.  The metrics are the exact constants. */
CG_API int cg_grid_create_cartesian(int ndim, const int64_t n[3], const double h[3],
                                    const int bc[6], cg_grid **out);
/* Body-fitted grid from node coordinates xyz_dev (device, ndim planes laid out
 * like one state plane).  period[3*d + m]: translation of coordinate m across
 * periodic direction d.  The coordinates are copied; the metrics are computed
 * on the device by cg_solver_create with the scheme's own derivative operator
 * (Sec. 2.1, xi_hat = xi_x / J; conservative metric identities). */
CG_API int cg_grid_create_curvilinear(int ndim, const int64_t n[3], const double *xyz_dev,
                                      const double period[9], const int bc[6], cg_grid **out);
CG_API void cg_grid_destroy(cg_grid *g);

/* Solver = grid + parameters + scratch.  The grid must outlive the solver. */
CG_API int cg_solver_create(const cg_grid *g, const cg_params *p, cg_solver **out);
CG_API void cg_solver_destroy(cg_solver *s);

/* Inflow face (dir, side) holds a per-node primitive profile instead of the
 * constant params.inflow state (e.g. a boundary layer with frozen
 * fluctuations).  W_host: host memory, nv planes over the face's nodes (the
 * other active directions, lowest first: j + n1*k for dir 0), copied to the
 * device (the call synchronises).  Ghost nodes of the face at every depth
 * take the profile of their transverse position, clamped to the face.  Call
 * before stepping (a captured batch graph keeps the profile it saw).
 * CG_ERR_INVALID_ARG if the face is not a CG_BC_INFLOW face. */
CG_API int cg_solver_set_inflow_profile(cg_solver *s, int dir, int side, const double *W_host);

/* Metrics on interior nodes: node_dev gets ndim*ndim planes xi_hat[l][m]
 * then one plane J; iface_dev (may be NULL) gets ndim*ndim planes of the
 * interface metrics of the l-interface i+1/2 stored at node i. */
CG_API int cg_metrics(cg_solver *s, double *node_dev, double *iface_dev, void *stream);

/* Right-hand side of Eq. (1): R = -J sum_l (F_{l,i+1/2} - F_{l,i-1/2}) for C-GBR,
 * R = -J sum_l D_l F_l for LAD, the mixture for the hybrid (Sec. 2, Alg. 1-3). */
CG_API int cg_rhs(cg_solver *s, const double *U, double *R, void *stream);

/* One TVD-RK3 step in place with time step dt (host value); LAD-C6 applies the
 * implicit filter after the third stage when filter_on.  Sets the sticky
 * non-physical flag read by cg_sync_status. */
CG_API int cg_rk3_step(cg_solver *s, double *U, double dt, void *stream);
/* Same with dt read from device memory at run time (graph-capturable). */
CG_API int cg_rk3_step_dev(cg_solver *s, double *U, const double *dt_dev, void *stream);

/* The CFL step size of U (cg_cfl_dt) written to dt_dev (device memory), then
 * one TVD-RK3 step of U in place with it (cg_rk3_step_dev): Sec. 3's time
 * loop body.  The CFL maximum is reduced by stage 1's primitive kernel, so U
 * is read once for both; the results are bitwise those of the two calls.
 * Graph-capturable; nothing waits. */
CG_API int cg_step_dev(cg_solver *s, double *U, double *dt_dev, void *stream);

/* cg_step_dev replayed as a CUDA graph: the solver's first call steps
 * eagerly; then the first call for a given (U, dt_dev) pair and tile shape
 * captures the step on `stream` (which must not be the legacy default
 * stream) and launches it, later calls launch the captured graph, which
 * removes the per-kernel launch gaps of a latency-bound step.  The graph
 * reads U and dt_dev through the pointers it was captured with; a call with
 * other pointers, or after a tile-shape change, captures again.  With kernel
 * timing on (cg_timing_enable) the step runs eagerly.  Nothing waits. */
CG_API int cg_step_graph(cg_solver *s, double *U, double *dt_dev, void *stream);

/* Diagnostic (no counterpart in the paper): the mixed form's FP64 <-> FP32
 * conversions on the integer pipes, applied elementwise: f_out[i] = d_in[i]
 * rounded to binary32 (nearest, ties to even), d_out[i] = f_in[i] widened to
 * binary64.  All four arrays are device memory of n elements, owned by the
 * caller; nothing waits.  They must equal the hardware conversions bit for bit. */
CG_API int cg_convert_check(const double *d_in, float *f_out, const float *f_in, double *d_out, int64_t n,
                            void *stream);

/* CFL time step dt = cfl / max_i J sum_l (|xi_hat_l . u| + c |xi_hat_l|).
 * dt_on_device = 1: *dt_out is device memory, nothing waits; 0: host memory,
 * the call synchronises the stream. */
CG_API int cg_cfl_dt(cg_solver *s, const double *U, double *dt_out, int dt_on_device, void *stream);

/* March with CFL time steps until t_end (last step clipped) or nsteps steps,
 * whichever comes first (t_end <= 0: nsteps only).  Synchronises; returns
 * CG_ERR_NONPHYSICAL if a non-physical state appeared. */
CG_API int cg_advance(cg_solver *s, double *U, int64_t nsteps, double t_end, double *t_out,
                      int64_t *steps_out, void *stream);
/* As cg_advance, but U_host is host memory: copied to the device, advanced,
 * copied back. */
CG_API int cg_advance_host(cg_solver *s, double *U_host, int64_t nsteps, double t_end,
                           double *t_out, void *stream);

/* Diagnostics. */
/* Discontinuity sensor Omega^d (the switch of the wave-appropriate selection,
 * Eq. 8) of state U at the n0*n1*n2 nodes, written to omega in FP64; the mixed
 * form computes and keeps it in FP32 and widens it on return.  Synchronises. */
CG_API int cg_omega(cg_solver *s, const double *U, double *omega, void *stream);
CG_API int cg_lad_coeffs(cg_solver *s, const double *U, double *beta, double *kappa, void *stream);
CG_API int cg_filter(cg_solver *s, double *U, void *stream);
/* Interface fluxes of the C-GBR / per-interface hybrid schemes along dir for all
 * interior lines, interfaces i = -1..n_dir-1: layout [v][line][n_dir+1]. */
CG_API int cg_iface_flux(cg_solver *s, const double *U, int dir, double *F, void *stream);
/* Hybrid: last global decision (0 LAD, 1 GBR) and troubled-node count of the
 * last evaluated stage.  Synchronises. */
CG_API int cg_hybrid_state(cg_solver *s, int *last_flag, int64_t *n_troubled, void *stream);
/* Synchronises and reports (then clears) the sticky non-physical flag. */
CG_API int cg_sync_status(cg_solver *s, void *stream);
CG_API int64_t cg_last_bad_index(const cg_solver *s);
CG_API const char *cg_last_error(void);
/* Number of kernel launches this handle has enqueued since creation. */
CG_API int64_t cg_launch_count(const cg_solver *s);
/* Bytes of device memory the solver holds: its scratch allocated by
 * cg_solver_create plus buffers allocated later on first use (inflow
 * profiles, the host-staging state of cg_advance_host, the scratch of
 * cg_iface_flux); the caller's state arrays are not included.  -1 for NULL.
 * Memory-budget admission (the serving loop) counts with it. */
CG_API int64_t cg_solver_device_bytes(const cg_solver *s);

/* Many independent grids (batched and served workloads).  cg_multi_step
 * advances each solvers[i] by one RK3 step of its own CFL time step on
 * states[i]: the members run concurrently on internal streams forked from
 * `stream` and joined back to it (stream-ordered, capturable in a CUDA graph).
 * Solvers must be distinct; every member keeps its own results (no
 * cross-member reduction), so a member's result does not depend on the batch.
 * cg_batch fixes a member list and its state pointers: the first
 * cg_batch_step runs eagerly, the second captures one step into a CUDA graph,
 * later calls replay it (one graph launch per batch step; `stream` must not
 * be the legacy default stream from the second call on).
 * Work table: a batch whose members are all 2D
 * Cartesian inviscid per-interface hybrids (CG_HYBRID, CG_HYBRID_CELL) of one
 * precision and one sweep tile shape steps phase by phase instead: each
 * launch runs one phase of an RK stage for every member of a group through a
 * table of per-member jobs and block offsets built at the first
 * cg_batch_step (41 launches per RK3 step and group, whatever the member
 * count; groups of members, 1 unless the autotuner chose more, run
 * concurrently on internal streams).  Each member computes what it computes
 * alone.  The table holds the members' buffer addresses:
 * members and states must outlive the batch, as for the stream path. */
typedef struct cg_batch cg_batch;
CG_API int cg_multi_step(cg_solver *const *solvers, double *const *states, int count, void *stream);
CG_API int cg_batch_create(int count, cg_solver *const *solvers, double *const *states, cg_batch **out);
CG_API int cg_batch_step(cg_batch *b, void *stream);
/* Autotunes the batch: every member's tile shape (as cg_autotune; equal
 * shapes share one measurement), then the number of streams the members are
 * spread over (1, 4, 8, 16 or 32), each timed over two batch steps from a saved
 * copy of the states that is restored afterwards: the states are unchanged
 * on return.  Synchronises; not during stream capture; a captured graph is
 * recaptured at the next cg_batch_step.  *width_out (may be NULL) gets the
 * chosen number of streams.  A batch that qualifies for the work table also
 * times the table with each common tile shape, then with 2, 4 and 8 member
 * groups, and keeps the faster path. */
CG_API int cg_batch_autotune(cg_batch *b, void *stream, int *width_out);
/* The path the batch steps by: *path_out = 1 for the work table, 0 for the
 * stream pool; *launches_out (may be NULL) = kernel launches of one table
 * step (41 per group), or -1 for the stream pool (each member counts its own).  Before the
 * first cg_batch_step the table is not built yet and the path reads 0. */
CG_API int cg_batch_path(const cg_batch *b, int *path_out, int *launches_out);
/* Persistent path (*path_out = 2, *launches_out = 3): a work-table batch in one
 * member group advances each RK stage in ONE cooperative launch (all blocks
 * co-resident, as many as the occupancy allows on every SM): the stage's
 * phases run one after another over their blocks with a grid barrier between
 * them.  Every barrier wait is bounded (about a second); a wait that runs out
 * ends the launch early with an error flag that cg_batch_sync reports.  The
 * work table's members compute what they compute alone (bitwise in FP64).
 * cg_batch_set_path chooses the path: 0 the stream pool, 1 the work table in
 * `groups` member groups, 2 the persistent stages; CG_ERR_UNSUPPORTED where
 * the batch does not qualify (the table needs 2D Cartesian inviscid
 * per-interface hybrids of one precision; the persistent stage a tile shape
 * of 4 or 8 lines in both directions).  The next cg_batch_step runs eagerly
 * and the one after recaptures.  cg_batch_autotune times the persistent
 * stages too and keeps the fastest path. */
CG_API int cg_batch_set_path(cg_batch *b, int path, int groups);
/* Synchronises the stream; CG_ERR_TIMEOUT (once, then cleared) if a
 * persistent stage's barrier gave up waiting since the last call. */
CG_API int cg_batch_sync(cg_batch *b, void *stream);
/* Test hook of the bounded barrier wait: from the next cg_batch_step on, every
 * barrier of the persistent stages waits for `extra` more arrivals than the
 * launch has blocks (0 restores the normal count), so each wait runs out after
 * about a second, sets the error flag and ends the launch; the members' states
 * are then incomplete.  CG_ERR_UNSUPPORTED off the persistent path. */
CG_API int cg_batch_debug_barrier(cg_batch *b, int extra);
CG_API void cg_batch_destroy(cg_batch *b);

/* Autotuner of the C-GBR sweep (MEG6, MIG4, hybrid; a no-op for LAD): for
 * each direction, the number of grid lines a tile of 64 interfaces spans
 * (4 or 8 along x; 4, 8 or 16 along y and z) is chosen by timing the
 * right-hand side of the state U with each candidate.  Results are cached
 * for the process by grid shape, grid kind and scheme; force = 1 re-times.
 * U is read only.  Synchronises; not during stream capture.  The choice does
 * not change any result: it only regroups the same per-interface work. */
CG_API int cg_autotune(cg_solver *s, const double *U, int force, void *stream);
/* Lines per sweep tile in use, per direction (0 for unused directions). */
CG_API int cg_tile_shape(const cg_solver *s, int lines_per_tile[3]);
/* Sets the lines per sweep tile per direction (entries of unused directions
 * are ignored); CG_ERR_INVALID_ARG for a value that is not a candidate. */
CG_API int cg_set_tile_shape(cg_solver *s, const int lines_per_tile[3]);

/* Right-hand side of the MEG6 (C-GBR explicit) scheme on a uniform Cartesian
 * grid without allocating any device memory, for callers that cannot call
 * cudaMalloc: code running while a stream is captured into a CUDA graph,
 * plug-ins whose host application owns all device memory, real-time loops that
 * cannot take an allocation's synchronisation.  Same result as cg_rhs of a
 * MEG6 solver on the same grid and parameters.  The paper has no counterpart;
 * this is a deployment convenience.
 *  - Arguments: the grid as for cg_grid_create_cartesian, p->scheme must be
 *    CG_MEG6, p->precision CG_FP64 and p->viscous 0 (inviscid only: the
 *    viscous pass needs the solver's scratch); otherwise CG_ERR_UNSUPPORTED.
 *    Every other parameter is checked as by cg_solver_create
 *    (CG_ERR_INVALID_ARG).  U and R as for cg_rhs.
 *  - Limit: at most 65,536 cells and 2*nv*N + prod(n_d + 8) <= 2^20 scratch
 *    doubles; larger grids return CG_ERR_INVALID_ARG with the sizes.
 *  - Scratch: a fixed 8 MiB array in device memory, held by every GPU that
 *    loads this library until the process exits.  The first call on each
 *    device looks up that array's device address (make it before any stream
 *    capture).  All calls share the array: calls that may overlap on the GPU
 *    (different streams or threads without ordering) race and must be
 *    serialised by the caller.  Nothing in it needs clearing: every element a
 *    call reads was written earlier in the same call. */
CG_API int cg_rhs_meg6_noalloc(int ndim, const int64_t n[3], const double h[3], const int bc[6],
                               const cg_params *p, const double *U, double *R, void *stream);

/* Kernel timing for measurement: while enabled, every launch of a timed
 * kernel class is bracketed by CUDA events on its stream; cg_timing_query
 * synchronises on them, returns the summed duration (ms) and the number of
 * launches of that class since the last query, and forgets them. */
#define CG_TIMING_SWEEP 0 /* the fused C-GBR interface sweep */
CG_API int cg_timing_enable(cg_solver *s, int on);
CG_API int cg_timing_query(cg_solver *s, int kernel_class, double *total_ms, int64_t *count);

#ifdef __cplusplus
}
#endif
#endif
