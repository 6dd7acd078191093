/*
 * fizzy_proj.h -- C ABI of the B300 (sm_103a) variable-density
 * pressure-correction projection.
 *
 * The operation (CaNS-Fizzy paper, "Methods and Implementation strategy":
 * second-order finite differences on a staggered Cartesian grid, pressure
 * correction whose variable-coefficient Poisson equation is turned into a
 * constant-coefficient one by the Dong & Shen / Dodd & Ferrante splitting of
 * Frantzis & Grigoriadis, solved by the fast direct FFT solver of CaNS; and
 * "Mathematical model": density mapped linearly over the phase field):
 *
 *   rho    = rho_g + phi (rho_l - rho_g)              (cell centres)
 *   beta_f = 1 / (mean of the two adjacent centre rho) (faces)
 *   rho0   = min(rho_l, rho_g),   phat = 2 p^n - p^(n-1)
 *   f      = (rho0/dt) D(u*) + D[(1 - rho0 beta_f) G phat]   (mean removed)
 *   D G p  = f      -- real FFT (periodic) or DCT-II (wall) along x and y,
 *                      one tridiagonal solve per (kx, ky) along z,
 *                      inverse transforms; p has zero dzf-weighted mean
 *   u      = u* - dt [G p / rho0 + (beta_f - 1/rho0) G phat]  (non-wall faces)
 *
 * G is the centre-to-face gradient, D the face-to-centre divergence.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - Arrays are double, C order [nz][ny][nx] (x fastest), caller-owned.
 *  - Staggering: u[k][j][i] is the x-face i+1/2, v[k][j][i] the y-face j+1/2,
 *    w[k][j][i] the z-face k+1/2.  x and y are periodic or wall-bounded
 *    (bc_x, bc_y); z is wall-bounded (homogeneous Neumann p) unless the
 *    descriptor sets periodic_z, in which case w[nz-1] is the seam face
 *    joining plane nz-1 to plane 0.  In a wall direction the last face
 *    (i = nx-1, j = ny-1, k = nz-1) is the far wall and must hold 0 on
 *    input; the near wall face is implicit.  Wall faces are 0 on output.
 *  - "stream" is a cudaStream_t passed as void* (NULL = legacy default
 *    stream).  Device work is asynchronous on it unless stated otherwise.
 *  - Return codes: FIZZY_OK (0) or a negative FIZZY_ERR_* value; no entry
 *    point aborts, exits or traps.  fizzy_proj_errstr() names a code and
 *    fizzy_proj_last_error() gives the last message recorded on a plan.
 */
#ifndef FIZZY_PROJ_H
#define FIZZY_PROJ_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
    FIZZY_OK = 0,
    FIZZY_ERR_INVALID = -1,       /* bad argument (null pointer, extent < 2, rho <= 0, dt <= 0, ...) */
    FIZZY_ERR_UNSUPPORTED = -2,   /* nx or ny with a prime factor other than 2 and 3, or too large  */
    FIZZY_ERR_NOMEM = -3,         /* device allocation failed                                       */
    FIZZY_ERR_CUDA = -4,          /* a CUDA call failed; message kept on the plan                   */
    FIZZY_ERR_NOT_CONVERGED = -5, /* mixed mode: refinement stopped above tol (output still written) */
    FIZZY_ERR_TIMEOUT = -6        /* a bounded device wait gave up (batched executor)               */
};

/* Boundary kinds of x and y.  The projection and everything built on it
 * (batch, serving, the unsplit and ACDI steps, the allocation-free entry
 * point) take FIZZY_BC_PERIODIC and FIZZY_BC_NEUMANN (walls): the staggered
 * layout stores one face per cell, so a direction's near face is implicit
 * and must be a wall or periodic.  fizzy_poisson_solve also takes the
 * Dirichlet and mixed kinds of the CaNS fast solver (paper, "Methods and
 * Implementation strategy"): p = 0 on a Dirichlet face, read as a ghost
 * value -p beyond it; a Neumann face has zero flux (ghost value +p). */
enum {
    FIZZY_BC_PERIODIC = 0,
    FIZZY_BC_NEUMANN = 1,            /* zero flux at both faces (DCT-II / DCT-III)                  */
    FIZZY_BC_DIRICHLET = 2,          /* p = 0 at both faces (DST-II / DST-III)                      */
    FIZZY_BC_NEUMANN_DIRICHLET = 3,  /* zero flux at the near face, p = 0 at the far one (DCT-IV;   */
                                     /* even extents only)                                          */
    FIZZY_BC_DIRICHLET_NEUMANN = 4   /* p = 0 at the near face, zero flux at the far one (DST-IV;   */
                                     /* even extents only)                                          */
};

enum {
    FIZZY_PREC_FP64 = 0,  /* every pass in FP64                                           */
    FIZZY_PREC_MIXED = 1  /* FP32 transforms + z-solve, refined by FP64 residuals r = f - L p */
};

/* flags */
#define FIZZY_FLAG_CHECK 1u       /* also compute u_rms, max|D u| and (FP64 mode) relres into the stats */
#define FIZZY_FLAG_ASYNC_ALLOC 2u /* allocate the plan's device memory stream-ordered (cudaMallocAsync  */
                                  /* from the device's default pool) on the plan's stream, and free it  */
                                  /* the same way in fizzy_proj_destroy (no device synchronisation)     */
#define FIZZY_FLAG_FUSED_XY 4u    /* mixed plans with nx = ny = 256 or 512 (periodic or wall x, y): run  */
                                  /* the x and y transforms of each FP32 solve as one pass per          */
                                  /* direction of the solve on a thread-block cluster (a z-plane in     */
                                  /* distributed shared memory) instead of separate x and y passes;     */
                                  /* the same results, bit for bit.  Off by default: on this part the   */
                                  /* separate passes are faster (the cluster's plane fills its SMs'     */
                                  /* shared memory, so loads, exchange and stores cannot overlap)       */

/* Maximum x/y extent of one transform line. */
#define FIZZY_MAX_N 1024
#define FIZZY_DEFAULT_MAX_REFINE 4  /* refinement sweeps when max_refine = 0 */

/* Plan descriptor.  All fields are read at plan time only. */
typedef struct fizzy_proj_desc {
    int nx, ny, nz;       /* cells; nx, ny in [2, FIZZY_MAX_N] with prime factors 2 and 3 only;
                             nz >= 2; nx*ny*nz <= 4e9 and ny*ny*nz < 2^32, else
                             FIZZY_ERR_UNSUPPORTED                                              */
    double dx, dy;        /* uniform x and y spacing (> 0)                                     */
    double dz;            /* uniform z spacing (> 0), used when zf == NULL                      */
    const double *zf;     /* host array of nz+1 increasing z face coordinates, or NULL          */
    int bc_x, bc_y;       /* FIZZY_BC_*: PERIODIC or NEUMANN for the projection; any kind for  */
                          /* fizzy_poisson_solve (3 and 4 need an even extent)                 */
    double rho_l, rho_g;  /* phase densities (> 0, within [1e-30, 1e30]); phi = 1 is rho_l      */
    double dt;            /* time step (> 0)                                                    */
    int precision;        /* FIZZY_PREC_FP64 or FIZZY_PREC_MIXED                                */
    double tol;           /* mixed: stop when max|f - L p| / max|f| <= tol (0 -> 1e-10)         */
    int max_refine;       /* mixed: at most this many sweeps (0 -> FIZZY_DEFAULT_MAX_REFINE, max 16) */
    double div_tol;       /* mixed: also stop only when max|D u| dx / U <= div_tol, with U the   */
                          /* rms of u* and D u = (dt/rho0)(f - L p) (0 -> 1e-10; < 0 -> off)    */
    unsigned flags;       /* FIZZY_FLAG_*                                                       */
    int periodic_z;       /* 0: walls at z = zf[0] and zf[nz] (w[nz-1] is the top wall, 0);    */
                          /* 1: periodic z (triperiodic boxes with bc_x = bc_y = periodic, as  */
                          /* the paper's emulsion in homogeneous isotropic turbulence): the     */
                          /* seam face nz-1/2 joins plane nz-1 to plane 0, centre distance      */
                          /* (dzf_0 + dzf_(nz-1))/2, w[nz-1] is its velocity.  Each z-line is a */
                          /* cyclic tridiagonal system (Sherman-Morrison).  Not accepted by     */
                          /* fizzy_proj_solve_noalloc (FIZZY_ERR_UNSUPPORTED).  Other values:   */
                          /* FIZZY_ERR_INVALID.                                                 */
} fizzy_proj_desc;

/* Diagnostics of the last solve (host memory). */
typedef struct fizzy_proj_stats {
    int iterations;    /* mixed: refinement sweeps run (0 in FP64 mode)                          */
    int converged;     /* mixed: 1 if relres <= tol and the divergence estimate <= div_tol; FP64: 1 */
    double relres;     /* max|f - L p| / max|f| (mixed always; FP64 only with FIZZY_FLAG_CHECK)  */
    double f_max;      /* max|f|                                                                 */
    double div_max;    /* max|D u| over all cells (FIZZY_FLAG_CHECK)                             */
    double u_rms;      /* rms of u* over all face values (mixed always; FP64 with FIZZY_FLAG_CHECK) */
    double div_metric; /* div_max * dx / u_rms (FIZZY_FLAG_CHECK)                                */
} fizzy_proj_stats;

typedef struct fizzy_proj_plan_s *fizzy_proj_plan_t;

/* Build a plan: validates the descriptor, builds the eigenvalue and twiddle
 * tables on the host and the z-factorisation tables on the device, and
 * allocates all device tables and the workspace (fizzy_proj_workspace_bytes()).
 * Grid and precision are fixed per plan; densities and dt can be rebound with
 * fizzy_proj_set_physics.  Synchronous, except with FIZZY_FLAG_ASYNC_ALLOC:
 * then the plan is ready for work queued after it on the same stream (use it
 * on another stream only after that stream's work has completed).  On
 * failure *out is NULL. */
int fizzy_proj_plan(fizzy_proj_plan_t *out, const fizzy_proj_desc *d, void *stream);

/* Device bytes a plan for d would allocate (tables + workspace), 0 if d is invalid. */
size_t fizzy_proj_workspace_bytes(const fizzy_proj_desc *d);

/* One projection on device pointers.
 *   phi, p_n, p_nm1 : in, cell centred.
 *   u, v, w         : in u* (wall faces 0), out u (overwritten in place).
 *   p_np1           : out p^(n+1) with zero dzf-weighted mean; must not alias the inputs.
 *   st              : NULL -> fully asynchronous on stream (graph-capturable);
 *                     non-NULL host pointer -> the call synchronises the stream and fills it.
 * Returns FIZZY_ERR_NOT_CONVERGED (outputs still written) only when st is given. */
int fizzy_proj_solve(fizzy_proj_plan_t p, const double *phi, const double *p_n, const double *p_nm1,
                     double *u, double *v, double *w, double *p_np1, fizzy_proj_stats *st,
                     void *stream);

/* The plan's fast direct Poisson solve on a given right-hand side: L_h p = f
 * with L_h = D G, the 7-point operator of the projection (second-order
 * differences on the staggered grid; z from the plan's face coordinates,
 * walls or periodic) and the plan's x/y boundary kinds, Dirichlet and mixed
 * ones included (the CaNS solver the paper builds on: "Methods and
 * Implementation strategy").  Real transforms along x and y (half-complex
 * FFT, DCT-II, DST-II, DCT-IV or DST-IV per kind), one tridiagonal solve per
 * wavenumber pair along z, inverse transforms.
 *   f     : in, device, [nz][ny][nx] FP64.  Without a Dirichlet face in x or
 *           y the problem is singular: the solve removes f's dzf-weighted
 *           mean and returns the p of zero dzf-weighted mean (a mixed plan's
 *           refinement needs a compatible f, i.e. that mean already 0, to
 *           reach tol).  With a Dirichlet face p is unique.
 *   p_out : out, device, [nz][ny][nx] FP64; must not alias f.
 *   st    : NULL (asynchronous) or host stats: relres = max|f - L_h p| /
 *           max|f|, f_max, and on a mixed plan iterations and converged.
 * FP64 plan: one FP64 solve.  Mixed plan: FP32 transforms and z-solves,
 * refined by FP64 residuals until relres <= the plan's tol (at most
 * max_refine sweeps; max|f| times 1/(4 nx ny) must lie in the FP32 normal
 * range).  Uses the plan's spectral workspace.  Returns
 * FIZZY_ERR_NOT_CONVERGED (p written) when st is given and a mixed solve
 * stopped above tol. */
int fizzy_poisson_solve(fizzy_proj_plan_t p, const double *f, double *p_out, fizzy_proj_stats *st,
                        void *stream);

/* Variable-coefficient projection WITHOUT the constant-coefficient splitting
 * (the equation the splitting replaces; the paper's Hypre path solves it):
 *     D(beta_f G p) = D(u*)/dt,   u = u* - dt beta_f G p,   beta_f = 1/rho_f,
 * with the same grid, staggering, face densities and boundaries as
 * fizzy_proj_solve.  Solved by conjugate gradients preconditioned with
 * M^-1 = L^-1 D(rho_f G) L^-1, L^-1 the plan's constant-coefficient
 * FFT/tridiagonal solve (exact for a constant density); stops when
 * max|D(u*)/dt - D(beta_f G p)| / max|D(u*)/dt| <= tol (0 -> 1e-10) or after
 * max_iter iterations (1 .. 100000).
 *   phi        : in, cell centred (densities and dt from the plan).
 *   u, v, w    : in u* (wall faces 0), out u.
 *   p_np1      : out p with zero dzf-weighted mean (the full pressure; no p^n
 *                enters); must not alias the inputs.
 *   st         : NULL or host stats (iterations = CG iterations, relres,
 *                f_max = max|D(u*)/dt|, div_max, u_rms, div_metric).
 * On an FP64 plan the preconditioner is the FP64 solve; on a mixed plan it is
 * the FP32 solve (applied to r 2^-e, e the exponent of max|b|) with the
 * flexible (Polak-Ribiere) direction update; residuals, the operators and p
 * are FP64 in both.  Allocates 10 fields of workspace on first use (kept
 * with the plan); a mixed plan also uses its FP64 right-hand-side buffer.  Synchronises the stream
 * every 4 iterations to test convergence (not graph-capturable).  Returns
 * FIZZY_ERR_NOT_CONVERGED (outputs written) if tol was not reached. */
int fizzy_proj_solve_vc(fizzy_proj_plan_t p, const double *phi, double *u, double *v, double *w,
                        double *p_np1, int max_iter, double tol, fizzy_proj_stats *st, void *stream);

/* One explicit stage of the ACDI phase-field transport (Jain 2022; the
 * paper's phase-field model), the step that produces phi before a
 * projection, on the plan's grid and boundaries:
 *     d phi/dt = rhs = -div(u phi) + div{ gamma [ eps grad phi
 *                        - 1/4 (1 - tanh^2(psi/(2 eps))) grad psi/|grad psi| ] },
 *     psi = eps ln(max(phi + 1e-100, 1e-100)/max(1 - phi + 1e-100, 1e-100)),
 * in conservative face-flux form: psi and its unit gradient at the centres
 * (central differences, a wall mirrors psi, a zero gradient gives 0), face
 * values as the mean of the two cells, wall faces carry no flux (mass is
 * conserved to round-off).  The bounds inside the logarithm keep psi finite
 * (saturated near +-230 eps) where phi has left [0, 1] by an undershoot or
 * overshoot; for phi in [0, 1] they change nothing.
 *   phi          : in, cell centred.
 *   u, v, w      : in, face velocities (the projection's layout; wall faces 0).
 *   eps, gamma   : interface thickness (> 0) and velocity scale (>= 0).
 *   dt           : stage step; phi_out = phi + dt rhs.
 *   rhs_out      : out rhs, or NULL.
 *   phi_out      : out, or NULL; may alias phi (not u, v, w, rhs_out).
 * Asynchronous on stream.  Uses the plan's face-flux buffers as scratch
 * (a projection queued after it on the same stream is unaffected) and
 * allocates 5 fields on first use.  FP64 in either precision mode. */
int fizzy_acdi_step(fizzy_proj_plan_t p, const double *phi, const double *u, const double *v,
                    const double *w, double eps, double gamma, double dt, double *rhs_out,
                    double *phi_out, void *stream);

/* Rebind the densities and time step of a plan (the grid, its transforms and
 * z-factorisation tables do not depend on them).  Updates four per-plane
 * tables by an asynchronous copy on stream; solves issued after it on the
 * same stream use the new values.  Returns FIZZY_ERR_INVALID for rho <= 0 or
 * dt <= 0. */
int fizzy_proj_set_physics(fizzy_proj_plan_t p, double rho_l, double rho_g, double dt, void *stream);

/* Read the stats of the last solve issued on p (synchronises stream). */
int fizzy_proj_get_stats(fizzy_proj_plan_t p, fizzy_proj_stats *st, void *stream);

/* End-to-end variant on HOST buffers (pinned memory recommended): copies the
 * six inputs to plan-owned device buffers, solves, copies u, v, w and p back,
 * and waits for the copies (fizzy_proj_solve_host_async + fizzy_proj_host_wait).
 * The device staging buffers are allocated on first use and kept by the plan. */
int fizzy_proj_solve_host(fizzy_proj_plan_t p, const double *phi, const double *p_n,
                          const double *p_nm1, double *u, double *v, double *w, double *p_np1,
                          fizzy_proj_stats *st, void *stream);

/* Pipelined end-to-end solves on HOST buffers.  Each call queues the copy of
 * the six inputs (u_in, v_in, w_in hold u*), the solve on stream, and the copy
 * of u, v, w, p_np1 back, and returns at once.  The plan keeps two device
 * staging sets and two copy streams of its own: while one call solves, the
 * next call's inputs and the previous call's results are in transit, so
 * successive calls overlap their copies with the solves.  Host arrays must be
 * pinned (cudaHostAlloc / cudaHostRegister) for the copies to run
 * asynchronously, and must be left untouched (inputs) or unread (outputs)
 * until fizzy_proj_host_wait returns; the outputs may alias the inputs only
 * when each call is waited for before the next.  The two staging sets hold
 * 14 grid fields of device memory (allocated on first use).
 * fizzy_proj_host_wait blocks until every queued result is in host memory;
 * fizzy_proj_get_stats then reports the last solve.  Return FIZZY_OK or a
 * FIZZY_ERR_* code (FIZZY_ERR_NOMEM when the staging cannot be allocated). */
int fizzy_proj_solve_host_async(fizzy_proj_plan_t p, const double *phi, const double *p_n,
                                const double *p_nm1, const double *u_in, const double *v_in,
                                const double *w_in, double *u, double *v, double *w, double *p_np1,
                                void *stream);
int fizzy_proj_host_wait(fizzy_proj_plan_t p);

/* Free everything owned by the plan; NULL is a no-op.  Synchronises the device. */
int fizzy_proj_destroy(fizzy_proj_plan_t p);

const char *fizzy_proj_errstr(int code);
const char *fizzy_proj_last_error(fizzy_proj_plan_t p);

/* Number of kernels one fizzy_proj_solve launches on the plan (for launch accounting). */
int fizzy_proj_launches_per_solve(fizzy_proj_plan_t p);

/* Per-kernel timing (diagnostics).  enable = 1: every kernel launch of a
 * solve is bracketed by CUDA events recorded on the solve's stream; enable =
 * 2 + idx: only the launches of kernel slot idx are (two events per launch,
 * so the rest of the solve runs undisturbed); 0: off.  Up to 8192 launches
 * are kept; later ones are not timed.  Every call resets the totals.
 * fizzy_proj_timing() waits for the recorded events, folds them into
 * per-kernel totals and reports kernel slot idx: its name, total
 * milliseconds and launch count since the last reset.  Both return the
 * number of slots (set_timing: FIZZY_OK), or a negative code. */
int fizzy_proj_set_timing(fizzy_proj_plan_t p, int enable);
int fizzy_proj_timing(fizzy_proj_plan_t p, int idx, const char **name, double *ms, int *launches);

/* ------------------------------------------------------------------------
 * Batched projections.
 *
 * Many independent projections of uneven sizes, each described by its own
 * plan (either precision), replayed from a captured CUDA graph in one of two
 * forms.  Persistent form: one kernel launch works through a list of
 * (instance, pass, tile) items; an item waits (bounded spin) until every tile
 * of its instance's previous pass is done.  Grouped form: one ordinary launch
 * per pass covers that pass of every instance (of a chain), so launch order
 * carries the dependencies.  Solo-chain form: each instance's own
 * stand-alone launch sequence, instances on concurrent chains.  Results are
 * the same in every form and equal each plan's own fizzy_proj_solve (same
 * kernel bodies, same arithmetic per tile), except that a mixed plan with an
 * x or y length the register-resident FP32 transform passes cover runs them
 * alone and in the solo-chain form, and the Stockham passes in the other two
 * forms (the results agree within the mixed tolerance).
 *
 * arrays: 7*n device pointers, for instance i at 7i..7i+6:
 *         phi, p_n, p_nm1, u, v, w (u*, in/out), p_np1 -- fixed for the batch
 *         (the graph is captured with them; write new inputs into the same
 *         buffers between solves).
 * A plan in a batch must not be solved elsewhere at the same time (it lends
 * the batch its workspace and stats); read per-instance stats with
 * fizzy_proj_get_stats(plans[i]) after fizzy_proj_batch_status().
 * ------------------------------------------------------------------------ */
typedef struct fizzy_proj_batch_s *fizzy_proj_batch_t;

typedef struct fizzy_batch_tuning {
    int ctas_per_sm; /* resident CTAs per SM (256-thread kernels); 0 = as many
                        as fit                                                  */
    int flux_planes; /* z planes per flux tile, multiple of 32; 0 = 32           */
    int x_lines;     /* x-pass line pairs per tile (1..16); 0 = per-size default */
    int y_cols;      /* y-pass columns per tile (even, 2..32); 0 = default       */
    int order;       /* persistent form's work-list order: 0 pass-major,
                        1 instance-major, 2 staggered (half of the instances,
                        alternate by size, four passes behind the other half)  */
    int form;        /* 0 persistent launch; 1 grouped: one ordinary launch per
                        pass index and pass kind, covering the tiles of every
                        instance at that pass (no dependency waits); 2 solo
                        chains: each instance's own fizzy_proj_solve launch
                        sequence, captured                                     */
    int chains;      /* forms 1 and 2: instances split (by size, round robin)
                        into this many independent launch chains that the
                        graph runs concurrently (1..16); 0 = 1                 */
} fizzy_batch_tuning;

/* Build the batch (work list, device descriptors) and capture its graph.
 * tuning may be NULL (defaults).  Synchronous. */
int fizzy_proj_batch_create(fizzy_proj_batch_t *out, int n, const fizzy_proj_plan_t *plans,
                            double *const *arrays, const fizzy_batch_tuning *tuning,
                            void *stream);

/* Replay the batch graph on stream (asynchronous). */
int fizzy_proj_batch_solve(fizzy_proj_batch_t b, void *stream);

/* Wait for the stream and return the launch status: FIZZY_OK, or
 * FIZZY_ERR_TIMEOUT if a dependency wait gave up (outputs then invalid). */
int fizzy_proj_batch_status(fizzy_proj_batch_t b, void *stream);

/* Test support for the timeout path (no GPU fault): rebuild the batch graph
 * so that the first dependency wait of instance inst (0 <= inst < n) can
 * never be met, and every dependency wait gives up after spin_limit polls
 * (each about 64 ns; 1 <= spin_limit <= 2^26).  The next solve then ends
 * normally and fizzy_proj_batch_status returns FIZZY_ERR_TIMEOUT (outputs of
 * that solve invalid); the context stays usable.  inst = -1 and
 * spin_limit = 0 restore the defaults (no stall, 2^26 polls).  Returns
 * FIZZY_ERR_INVALID for a null batch or out-of-range arguments,
 * FIZZY_ERR_UNSUPPORTED for a batch built in the grouped or solo-chain form
 * (they have no dependency waits), else the status of the rebuild. */
int fizzy_proj_batch_inject_stall(fizzy_proj_batch_t b, int inst, long long spin_limit);

/* Time candidate tunings (reps replays each, CUDA events on stream), rebuild
 * the batch with the fastest and return it in *chosen and its mean time in
 * *best_ms (either may be NULL).  The candidates cover both forms: the
 * persistent launch with varied CTAs per SM, flux planes per tile, x-pass
 * lines per tile, y-pass columns per tile and work-list order, and the
 * grouped launches with 2, 4 or 8 chains, and the solo chains with 8 or 16.  Overwrites the batch outputs while
 * timing. */
int fizzy_proj_batch_autotune(fizzy_proj_batch_t b, int reps, fizzy_batch_tuning *chosen,
                              double *best_ms, void *stream);

/* Persistent form: work items, grid size and dynamic shared memory of the
 * launch.  Grouped form: launches per solve, the largest grid and the largest
 * dynamic shared memory of one launch. */
int fizzy_proj_batch_info(fizzy_proj_batch_t b, int *n_items, int *grid, size_t *smem_bytes);

int fizzy_proj_batch_destroy(fizzy_proj_batch_t b);

/* ------------------------------------------------------------------------
 * Serving runtime: continuous admission of projection requests.
 *
 * A server owns up to max_slots request slots, each with its own CUDA stream,
 * so requests admitted while others run overlap on the device.  Plans are
 * cached on the device by geometry (extents, spacings, z faces, boundary
 * types, precision and refinement settings) and rebound to each request's
 * densities and dt with fizzy_proj_set_physics, so requests of a geometry
 * already seen start without building tables.  Device memory of plans
 * (cached or in use) plus the seven arrays of every occupied slot is kept
 * within hbm_budget bytes: admission evicts least-recently-used idle plans
 * and otherwise refuses.  All device memory is stream-ordered
 * (cudaMallocAsync from the device's default pool, whose release threshold
 * the server raises to its budget), so admission and release never
 * synchronise the device.
 *
 * Typical use: fizzy_serve_admit -> fill the slot's input arrays on the
 * slot's stream -> fizzy_serve_launch -> fizzy_serve_poll until it reports
 * the slot -> read outputs -> fizzy_serve_release.
 * ------------------------------------------------------------------------ */
typedef struct fizzy_serve_s *fizzy_serve_t;

#define FIZZY_ERR_BUSY (-7) /* fizzy_serve_admit: no free slot right now */

int fizzy_serve_create(fizzy_serve_t *out, size_t hbm_budget, int max_slots);

/* Admit one request.  On FIZZY_OK, *slot is its slot and arrays[0..6] are
 * device arrays of d's shape: phi, p_n, p_nm1, u, v, w (u* in, u out), p_np1,
 * owned by the server until release.  FIZZY_ERR_BUSY: every slot is taken;
 * FIZZY_ERR_NOMEM: it does not fit the budget now.  Neither changes state. */
int fizzy_serve_admit(fizzy_serve_t s, const fizzy_proj_desc *d, int *slot, double **arrays);

/* The slot's stream (fill the inputs on it before launch). */
int fizzy_serve_stream(fizzy_serve_t s, int slot, void **stream);

/* Queue the projection of an admitted slot on its stream.  A mixed plan's
 * solve is queued with at most two refinement sweeps (most solves converge
 * after one); see fizzy_serve_poll for the rest. */
int fizzy_serve_launch(fizzy_serve_t s, int slot);

/* Report up to max launched slots whose projection has finished (without
 * blocking); returns how many were written to slots[].  A mixed solve that
 * has finished its queued sweeps without converging has its remaining sweeps
 * (up to its plan's max_refine) queued here instead, and is reported once
 * they have run: the results equal those of fizzy_proj_solve. */
int fizzy_serve_poll(fizzy_serve_t s, int *slots, int max);

/* Stats of a finished slot's projection. */
int fizzy_serve_stats(fizzy_serve_t s, int slot, fizzy_proj_stats *st);

/* Return the slot (its arrays go back to the pool, its plan to the cache). */
int fizzy_serve_release(fizzy_serve_t s, int slot);

/* Budget in use, cached plans, plans built so far, slots occupied. */
int fizzy_serve_info(fizzy_serve_t s, size_t *bytes_used, int *plans_cached, int *plans_built,
                     int *slots_busy);

int fizzy_serve_destroy(fizzy_serve_t s);

/* Stage one request's inputs from a device-resident source state: a data
 * movement helper for serving, not an operation of the method.
 * src[0..5] (a host array of six device pointers) are phi, p_n, p_nm1, u, v, w
 * of shape (tz, ty, tx), x fastest; dst[0..5] likewise of shape (nz, ny, nx).
 * Each output is a periodic crop,
 *   dst_f[k][j][i] = src_f[(k + oz) mod tz][(j + oy) mod ty][(i + ox) mod tx],
 * except that the wall faces of the staggered velocity are zero: u at
 * i = nx-1 when bc_x is FIZZY_BC_NEUMANN, v at j = ny-1 when bc_y is, and w
 * at k = nz-1 always (the top wall; for a periodic-z request that face is
 * the seam and must be staged by a plain copy instead).  One kernel on `stream` (null: the
 * legacy default stream) moving 96 bytes per output point; dst must not
 * overlap src.  Returns FIZZY_ERR_INVALID for a null pointer, an extent < 1,
 * a negative offset or a bc other than the two above, else FIZZY_OK or
 * FIZZY_ERR_CUDA if the launch failed. */
int fizzy_crop_fill(const double *const *src, int tx, int ty, int tz, double *const *dst,
                    int nx, int ny, int nz, int ox, int oy, int oz, int bc_x, int bc_y,
                    void *stream);

/* Measurement support (no counterpart in the paper): the arithmetic issue
 * rate of the GPU, the peak the FP64-bound projection kernels are measured
 * against.  precision FIZZY_PREC_FP64 times FP64 instructions,
 * FIZZY_PREC_MIXED FP32 ones; op 0 fused multiply-adds, 1 adds, 2 multiplies,
 * 3 multiply-adds and adds in turn, 4 multiply-adds each followed by an
 * independent FP32 multiply-add (not counted), 5 multiply-adds whose
 * multiplicand is another chain's register; chains (4, 8 or 16) independent chains
 * per thread.  One launch of a resident grid (CTAs per SM x SMs, 256
 * threads), 4 x chains x iters instructions per thread, timed with CUDA
 * events on stream, which the call synchronises.  *instr_per_s receives
 * instructions (per lane) per second, *elapsed_ms (nullable) the kernel
 * time.  Choose iters so the launch lasts 100 ms or more.  Returns
 * FIZZY_ERR_INVALID for an argument out of range or a null instr_per_s,
 * FIZZY_ERR_CUDA if the launch fails. */
int fizzy_probe_fma_rate(int precision, int op, int chains, int iters, double *instr_per_s,
                         double *elapsed_ms, void *stream);

/* ------------------------------------------------------------------------
 * Allocation-free projection (FP64 mode, small grids).
 *
 * The paper has no counterpart to this entry point; it exists for callers
 * that cannot call cudaMalloc: host applications that own every byte of
 * device memory through their own allocator or memory pool and forbid
 * allocations by libraries they load, and code that must not trigger an
 * allocation's implicit device synchronisation in the middle of its own
 * stream-ordered work.  It needs no plan: every call rebuilds the eigenvalue,
 * twiddle and z-factorisation tables on the host (a few milliseconds) and
 * copies them into scratch.
 *
 * Scratch: one file-scope static __device__ array of FIZZY_NOALLOC_SCRATCH_BYTES
 * bytes inside the library holds the tables and the workspace.  Every GPU
 * that loads the library holds this array until the process exits.  The
 * caller passes inputs and outputs exactly as for fizzy_proj_solve().
 *
 * Limits: nx * ny * nz <= FIZZY_NOALLOC_MAX_CELLS, nx and ny <= 512 (prime
 * factors 2 and 3), nz <= 4096; larger grids return FIZZY_ERR_UNSUPPORTED
 * without touching the device.  precision must be FIZZY_PREC_FP64 and flags 0.
 *
 * The first call on a device looks up the device address of the scratch
 * array (cudaGetSymbolAddress) with that device current; make that first call
 * before any stream capture.  All calls share the one array and its host-side
 * staging buffer, which keep the previous call's contents: calls that overlap
 * (on different streams, or from several host threads at once) race and must
 * be serialised by the caller.  Returns FIZZY_OK or a FIZZY_ERR_* code; no
 * stats are produced.
 * ------------------------------------------------------------------------ */
#define FIZZY_NOALLOC_MAX_CELLS 262144
#define FIZZY_NOALLOC_SCRATCH_BYTES 12968256
int fizzy_proj_solve_noalloc(const fizzy_proj_desc *d, const double *phi, const double *p_n,
                             const double *p_nm1, double *u, double *v, double *w,
                             double *p_np1, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* FIZZY_PROJ_H */
