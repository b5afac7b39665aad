/*
 * fdlbm.h - C ABI of the GB300 library for the D2Q9 T2S2-FDLBM time step
 * (Chen, Chai, Wang, Shi, "A finite-difference lattice Boltzmann model with
 * second-order accuracy of time and space for incompressible flow",
 * arXiv 1911.12913).
 *
 * One handle = one grid, one parameter set and the distribution state f~ of
 * every node, resident in device memory.  All compute runs in CUDA kernels on
 * the handle's stream; the host only marshals arguments.
 *
 * Conventions for every entry point:
 *  - Return an fdlbm_status; no C++ exception crosses this boundary.  The text
 *    of the last failure of a handle is available from fdlbm_last_error().
 *  - Arrays are row-major [ny][nx] (x fastest); distributions are [9][ny][nx]
 *    with the population order of Sec. 3 of the paper:
 *      i :  0  1  2  3  4  5  6  7  8
 *      xi: (0,0) (1,0) (0,1) (-1,0) (0,-1) (1,1) (-1,1) (-1,-1) (1,-1)
 *  - Arguments tagged `where` are host pointers (FDLBM_MEM_HOST) or device
 *    pointers (FDLBM_MEM_DEVICE) of FP64 values.  They are borrowed for the call
 *    only: host arrays are copied before the call returns, device arrays are
 *    read by work enqueued on the handle's stream (keep them alive until that
 *    work completes).
 *  - fdlbm_step() is asynchronous.  Calls that return host data (get_state and
 *    moments with FDLBM_MEM_HOST, reduce) synchronise the stream.
 */
#ifndef FDLBM_H
#define FDLBM_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

#define FDLBM_ABI_VERSION 3

typedef struct fdlbm_ctx *fdlbm_t;

typedef enum {
    FDLBM_OK = 0,
    FDLBM_EINVAL = -1,        /* invalid argument (sizes, metrics <= 0, NULL, ...) */
    FDLBM_ENOMEM = -2,        /* workspace too small, or device allocation failed */
    FDLBM_ECUDA = -3,         /* CUDA runtime error, or a bounded device-side wait (an mbarrier
                                 of a tensor-copy kernel, a grid barrier of a persistent batch)
                                 that gave up: there is no separate timeout status; the text
                                 of fdlbm_last_error() says which */
    FDLBM_ENONFINITE = -4,    /* a reduction met NaN or Inf (the run diverged) */
    FDLBM_EUNSUPPORTED = -5,  /* option combination not available */
    FDLBM_ETOOBIG = -6        /* size beyond a fixed capacity (see fdlbm_reduce_noalloc) */
} fdlbm_status;

enum { FDLBM_PERIODIC = 0, FDLBM_WALL = 1 };            /* boundary kind of an axis */
enum { FDLBM_FP64 = 0, FDLBM_FP32_DEV = 1 };            /* storage / arithmetic precision */
enum { FDLBM_PATH_AUTO = 0, FDLBM_PATH_FUSED = 1, FDLBM_PATH_STAGED = 2 };
enum { FDLBM_MEM_HOST = 0, FDLBM_MEM_DEVICE = 1 };
/* Equilibrium of the BGK collision.  STANDARD is Eq. 3.2.  INCOMPRESSIBLE is
 * the incompressible equilibrium of He and Luo, which Sec. 2 of the paper says
 * can be combined with both T2S2 schemes without printing it:
 *   f_i^eq = w_i [rho + rho0 (xi.u / cs^2 + ((xi.u)^2 - cs^2 u.u) / (2 cs^4))],
 * with the velocity read from rho0 u = sum xi f~ + (dt/2) rho0 F (Eq. 3.3 with
 * rho0 for rho) and the forcing term of Eq. 3.12 taken with the equilibrium at
 * rho0.  It runs on every step kernel and in batches; the adjoint step
 * returns FDLBM_EUNSUPPORTED with it.  fdlbm_moments returns the density and
 * this velocity. */
enum { FDLBM_EQ_STANDARD = 0, FDLBM_EQ_INCOMPRESSIBLE = 1 };
/* Fused-kernel variant of T2S2-FDLBM1 (Sec. 2D, first sequence):
 *  SCALAR  one column per thread, rows loaded through registers (any nx >= 4);
 *          on a grid with a walled axis, the walls sweep with Eq. 3.10 inside;
 *  WARP    FP32 only, one independent warp per 56-column tile, two adjacent
 *          columns per lane in packed f32x2 arithmetic, x-neighbours by warp
 *          shuffle, rows by bulk tensor copies into a per-warp ring; no
 *          block-level barrier; with or without a force field (nx >= 64, nx %
 *          4 == 0 on a periodic x axis, fewer than 2^32 values in the state).
 *          On a grid with a walled axis it covers the interior, the nodes at
 *          least 4 from every wall whose tiles load nothing outside the grid
 *          (there the walled and the periodic scheme compute the same values),
 *          and a second launch of the walls sweep covers the 4-node frame:
 *          two launches per step (fdlbm_kernels_per_step).
 * AUTO picks WARP where it applies (the fastest measured on GB300 for the
 * periodic 4096^2 throughput case), except on walled grids of fewer than
 * 1.5 M nodes, where the frame launch's fixed cost makes the walls sweep
 * faster, and SCALAR otherwise.  Asking for a variant that does not apply
 * returns FDLBM_EUNSUPPORTED; the values 2 to 4 are not used. */
enum { FDLBM_VARIANT_AUTO = 0, FDLBM_VARIANT_SCALAR = 1, FDLBM_VARIANT_WARP = 5 };
enum { FDLBM_WALL_W = 0, FDLBM_WALL_E = 1, FDLBM_WALL_S = 2, FDLBM_WALL_N = 3 };
/* Time-marching scheme (Sec. 2A):
 *  T2S2_1  f~(n+1) = f~+ + dt L(f*), f* at t_n + A dt (Eq. 2.23; A = 0 gives T1S2);
 *  T2S2_2  f~(n+1) = f~+ + dt/2 [L(f^n) + L(f^{n+1})] with the characteristic
 *          estimate of f^{n+1} over h = dt (Eq. 5.23, second sequence of Sec. 2D).
 *          Runs on its own fused sweeps (FP32 grids of 64 columns and more:
 *          the warp-tile kernel, with the walls sweep on the 4-node frame of a
 *          walled grid; otherwise the scalar sweeps, periodic grids in both
 *          precisions and walled grids in FP32) and on the staged kernels
 *          (walled grids in FP64, or opts.path = FDLBM_PATH_STAGED); A is
 *          ignored. */
enum { FDLBM_SCHEME_T2S2_1 = 0, FDLBM_SCHEME_T2S2_2 = 1 };

/* Tensor-product grid (Sec. 3, Eqs. 3.9 and 3.11).  A periodic axis stores its
 * n unique nodes (node n is node 0 shifted by the period); a walled axis stores
 * both wall nodes.  Coordinates are host arrays, strictly increasing. */
typedef struct {
    int nx, ny;
    const double *x, *y;      /* host, length nx / ny */
    double lx, ly;            /* period of a periodic axis; 0: n * (x[1] - x[0]) */
    int bc_x, bc_y;           /* FDLBM_PERIODIC or FDLBM_WALL */
    double wall_u[4][2];      /* (u, v) of the W, E, S, N walls (Eq. 3.10 boundary data) */
} fdlbm_grid;

/* 1-D grid metrics: d(zeta)/dx at every column and d(mu)/dy at every row, where
 * zeta, mu are the node indices (unit spacing).  d/dx = (dzeta/dx) d/dzeta is
 * applied to the differences of Eqs. 2.36-2.38.  Host arrays, every entry > 0.
 * NULL for an axis means uniform spacing: 1 / (x[1] - x[0]). */
typedef struct {
    const double *dzeta_dx;   /* length nx or NULL */
    const double *dmu_dy;     /* length ny or NULL */
} fdlbm_metrics;

typedef struct {
    double A;                 /* t* = t_n + A dt (Eq. 2.9): 0.5 = T2S2-FDLBM1 (Eq. 2.21), 0 = T1S2 (Eq. 2.16) */
    double rho0;              /* reference density; FP32 storage keeps f~_i - w_i rho0 */
    int precision;            /* FDLBM_FP64 or FDLBM_FP32_DEV */
    int has_force;            /* 1: reserve a body-acceleration field (fdlbm_set_force), Eq. 3.12 */
    int path;                 /* FDLBM_PATH_AUTO: the fused kernel for both schemes on periodic
                                 grids and on walled grids in FP32; the staged kernels for
                                 walled grids in FP64 (bound by the FP64 units, where the
                                 sweep's recomputed halo costs more than the extra traffic) */
    int rows_per_cta;         /* fused kernel tile height; 0 = automatic */
    int variant;              /* FDLBM_VARIANT_*; WARP where it does not apply -> EUNSUPPORTED */
    int scheme;               /* FDLBM_SCHEME_T2S2_1 (default) or FDLBM_SCHEME_T2S2_2 */
    int adjoint;              /* 1: reserve scratch for fdlbm_adjoint_step (periodic grids) */
    int graph_steps;          /* > 0: fdlbm_step replays a CUDA graph of this many steps (rounded
                                 up to even), captured on first use; 0 = direct launches */
    int equilibrium;          /* FDLBM_EQ_STANDARD (Eq. 3.2) or FDLBM_EQ_INCOMPRESSIBLE */
    void *stream;             /* cudaStream_t used for all work; NULL = default stream */
    void *workspace;          /* caller-owned device memory of fdlbm_workspace_bytes() bytes,
                                 256-byte aligned; NULL = the library allocates its own */
    size_t workspace_bytes;
} fdlbm_opts;

/* Fill *o with the defaults: A = 0.5, rho0 = 1, FP64, no force, automatic path,
 * default stream, library-owned workspace. */
void fdlbm_default_opts(fdlbm_opts *o);

/* Eq. 3.1: dt = CFL * dx_min / xi with xi = 1 (lattice speed) and dx_min the
 * smallest node spacing over both axes.  Host only.  Returns a negative value
 * for an invalid grid or cfl <= 0. */
double fdlbm_time_step(const fdlbm_grid *grid, double cfl);

/* Device bytes a handle needs for this grid and options (0 if invalid).  Host only. */
size_t fdlbm_workspace_bytes(const fdlbm_grid *grid, const fdlbm_opts *opts);

/* Create a handle.  nu: kinematic viscosity (tau = nu / cs^2, cs^2 = 1/3);
 * cfl: Eq. 3.1; blend: weight beta of the second-order upwind difference in the
 * mixed difference, D_m = (1 - beta) D_central + beta D_upwind (Eq. 2.36 with the
 * blend read as the upwind weight; see Eq. 4.8).  opts may be NULL (defaults).
 * The state is zero (f~ = w_i rho0, fluid at rest) until initialised.
 * Errors: EINVAL (sizes < 3, non-increasing coordinates, metric <= 0, nu <= 0,
 * cfl <= 0, blend outside [0, 1], A outside [0, 1]), ENOMEM (workspace too
 * small or cudaMalloc failed), ECUDA. */
fdlbm_status fdlbm_create(const fdlbm_grid *grid, const fdlbm_metrics *metrics, double nu,
                          double cfl, double blend, const fdlbm_opts *opts, fdlbm_t *out);

/* Release the handle and any memory the library allocated.  NULL-safe. */
void fdlbm_destroy(fdlbm_t h);

/* Initialise f~ from macroscopic fields.  The physical distribution is
 * f = f^eq(rho, u) (Eq. 3.2), or with grad != NULL the non-equilibrium start of
 * Eq. 3.5, and the stored variable is f~ = f - (dt/2) Omega-bar(f) (Eq. 2.19):
 *   f~_i = f_i^eq - (dt/2) F_i(rho, u) - rho0 w_i (2 tau + dt) / (2 cs^2) xi_i xi_i : grad u,
 * with F_i the forcing term of Eq. 3.12 under the handle's body-acceleration
 * field AS SET AT THE TIME OF THIS CALL (zero without opts.has_force or before
 * the first fdlbm_set_force), so that Eq. 3.3 returns exactly the given u.  A
 * later fdlbm_set_force changes the force of the following steps but not the
 * state: call fdlbm_set_force first to start a forced run from (rho, u).
 * grad = 4 consecutive [ny][nx] fields du/dx, du/dy, dv/dx, dv/dy.
 * rho, ux, uy: [ny][nx] FP64 at `where`. */
fdlbm_status fdlbm_init_fields(fdlbm_t h, const double *rho, const double *ux, const double *uy,
                               const double *grad, int where);
/* The same from FP32 fields ([ny][nx] float at `where`), the density given as
 * its deviation drho = rho - rho0 so that FP32 keeps its small variations.
 * For a handle with FP32 storage nothing is lost against the FP64 call (the
 * arithmetic runs in the storage precision either way) and half the bytes
 * move. */
fdlbm_status fdlbm_init_fields_f32(fdlbm_t h, const float *drho, const float *ux, const float *uy,
                                   const float *grad, int where);

/* Copy f~ ([9][ny][nx] FP64 at `where`) into / out of the handle. */
fdlbm_status fdlbm_set_state(fdlbm_t h, const double *f, int where);
fdlbm_status fdlbm_get_state(fdlbm_t h, double *f, int where);

/* Body acceleration Fbar ([2][ny][nx] FP64 at `where`: x then y component),
 * used by Eqs. 3.3 and 3.12.  Needs opts.has_force. */
fdlbm_status fdlbm_set_force(fdlbm_t h, const double *force, int where);

/* Advance n >= 0 time steps of the scheme (Sec. 2D, Steps 1-3; Eq. 2.23), with
 * the non-equilibrium extrapolation of Eq. 3.10 on walled sides.  Enqueued on
 * the stream; returns ECUDA if a launch fails. */
fdlbm_status fdlbm_step(fdlbm_t h, int n);

/* Density and velocity of Eq. 3.3 into [ny][nx] FP64 arrays at `where`,
 * computed in the storage precision of the handle. */
fdlbm_status fdlbm_moments(fdlbm_t h, double *rho, double *ux, double *uy, int where);
/* The same into FP32 arrays, the density as its deviation rho - rho0. */
fdlbm_status fdlbm_moments_f32(fdlbm_t h, float *drho, float *ux, float *uy, int where);

/* FP64 reductions (warp shuffles, fixed order): *mass = sum rho / (m_x m_y) over all
 * nodes (the Jacobian-weighted mass, exactly conserved on periodic grids), and
 * *resid = the successive-state residual of the cavity section,
 * sqrt(sum |u - u_prev|^2 / sum |u|^2), against the velocity of the previous
 * fdlbm_reduce call (-1 on the first call; for a fluid exactly at rest, where
 * sum |u|^2 = 0, the absolute sqrt(sum |u - u_prev|^2), which is 0 if it was at
 * rest before as well).  Synchronises the stream.  Returns
 * ENONFINITE if either value is NaN/Inf.  Either pointer may be NULL. */
fdlbm_status fdlbm_reduce(fdlbm_t h, double *mass, double *resid);

/* Bind the handle to another stream (cudaStream_t). */
fdlbm_status fdlbm_set_stream(fdlbm_t h, void *stream);

/* Wait for the handle's stream; reports asynchronous CUDA errors as ECUDA. */
fdlbm_status fdlbm_sync(fdlbm_t h);

double fdlbm_dt(fdlbm_t h);              /* the dt of Eq. 3.1 used by the handle */
double fdlbm_tau(fdlbm_t h);             /* nu / cs^2 */
long long fdlbm_steps_done(fdlbm_t h);   /* steps enqueued since creation */
int fdlbm_path(fdlbm_t h);               /* FDLBM_PATH_FUSED or FDLBM_PATH_STAGED */
int fdlbm_kernels_per_step(fdlbm_t h);   /* kernel launches fdlbm_step makes per step */
/* The tiles of the warp-tile kernel's step on a grid (FDLBM_VARIANT_WARP), for
 * the tile height `rows` (> 0) and `scheme` (FDLBM_SCHEME_*): first the
 * interior windows in launch order, then, on a walled grid, the frame tiles,
 * 5 ints each: kind (0: interior, the warp tile, 56 output columns; 1: frame,
 * the walls sweep in one-warp blocks, 24 output columns), x0 (first output
 * column), the end of the columns the tile stores, y0, y1 (rows [y0, y1)).
 * The interior covers the nodes at least 4 from every wall whose tiles load
 * nothing outside the grid (Eq. 3.10 and the central differences next to a
 * wall reach no further), the frame the rest.  Host only, no device work:
 * *count receives the number of tiles and at most cap are written to tiles.
 * EINVAL for bad arguments, EUNSUPPORTED where the warp-tile kernel does not
 * apply. */
fdlbm_status fdlbm_tile_plan(const fdlbm_grid *g, int rows, int scheme, int *tiles, int cap, int *count);
const char *fdlbm_last_error(fdlbm_t h); /* never NULL */
/* Short description of the kernel the handle runs per step, e.g.
 * "fused-warp fp32dev rows=121" (never NULL; valid until the handle is destroyed). */
const char *fdlbm_describe(fdlbm_t h);
const char *fdlbm_status_string(fdlbm_status s);

/* ---------------------------------------------------------------------------
 * Reverse mode.  The paper has no adjoint; this is the discrete adjoint of the
 * step above (Sec. 2D Steps 1-3 on a periodic grid, scheme T2S2_1), written by
 * hand, with the body-acceleration field of Eq. 3.12 as the parameter.  States
 * and cotangents live in device buffers of fdlbm_state_bytes() bytes in the
 * handle's storage layout (precision of the handle, [9][ny][pitch] deviations
 * from w_i rho0; cotangents use the same layout).
 * ------------------------------------------------------------------------- */
size_t fdlbm_state_bytes(fdlbm_t h);
/* Row pitch (elements) and element size (4 or 8 bytes) of the storage layout:
 * value (i, y, x) of a state or cotangent buffer sits at element
 * (i * ny + y) * pitch + x; elements with x >= nx are padding. */
fdlbm_status fdlbm_state_layout(fdlbm_t h, int *pitch, int *elem_bytes);
/* Device copy between the handle's current state and `buf` (storage layout):
 * to_handle = 1 loads buf into the handle, 0 stores the handle's state into buf. */
fdlbm_status fdlbm_copy_state(fdlbm_t h, void *buf, int to_handle);
/* One adjoint step: given the state g^n (state_n) and the cotangent lam_next of
 * g^{n+1} = step(g^n), write the cotangent lam_prev of g^n and, if dforce is
 * not NULL, add the cotangent of the force field to dforce (device, FP64,
 * [2][ny][nx]; a handle without a force field differentiates at zero force).
 * Needs opts.adjoint, both axes periodic and scheme T2S2_1 (else EUNSUPPORTED).
 * lam_next and lam_prev may not alias.  Asynchronous on the stream. */
fdlbm_status fdlbm_adjoint_step(fdlbm_t h, const void *state_n, const void *lam_next,
                                void *lam_prev, double *dforce);
/* Cotangent of a state from a cotangent du ([2][ny][nx] FP64 device) of its
 * velocity (Eq. 3.3): writes lam (storage layout) and adds du * dt/2 to dforce
 * (if not NULL). */
fdlbm_status fdlbm_moments_vjp(fdlbm_t h, const void *state, const double *du, void *lam,
                               double *dforce);
/* Cotangents of the fields of an equilibrium initialisation
 * (fdlbm_init_fields(rho, ux, uy, NULL): Eq. 3.2 or the incompressible
 * equilibrium, minus (dt/2) F_i of Eq. 2.19 under the handle's current force
 * field): given the cotangent lam (storage layout, device) of the state that
 * those fields (device, FP64, [ny][nx] each) produce, ADD their cotangents to
 * drho (may be NULL), dux and duy (device, FP64, [ny][nx]), and the cotangent
 * of the force field through the initial state to dforce (device, FP64,
 * [2][ny][nx]; may be NULL).  With fdlbm_adjoint_step this differentiates a
 * rollout with respect to its initial density and velocity.  Asynchronous on
 * the stream. */
fdlbm_status fdlbm_init_vjp(fdlbm_t h, const double *rho, const double *ux, const double *uy,
                            const void *lam, double *drho, double *dux, double *duy,
                            double *dforce);

/* ---------------------------------------------------------------------------
 * Batched mode: many independent cases (uneven sizes, walls, forces, Reynolds
 * numbers) advanced together.  Every case is an ordinary handle whose memory
 * lies inside one batch workspace: the per-case calls (fdlbm_init_fields,
 * fdlbm_set_force, fdlbm_get_state, fdlbm_moments, fdlbm_reduce, fdlbm_dt) work
 * on fdlbm_batch_case(b, c); stepping, the stream and destruction belong to the
 * batch (fdlbm_step / fdlbm_set_stream on a case return EUNSUPPORTED,
 * fdlbm_destroy ignores it).  Every case runs its own scheme (Sec. 2D) with
 * its own dt (Eq. 3.1), on the kernels that fdlbm_batch_set_mode selects; one
 * batch step advances every case by one of its own time steps.
 * ------------------------------------------------------------------------- */
typedef struct fdlbm_batch_ctx *fdlbm_batch_t;

/* Device bytes of the batch workspace (0 if any case is invalid).  opts may be
 * NULL (defaults) or an array of ncases option blocks. */
size_t fdlbm_batch_workspace_bytes(int ncases, const fdlbm_grid *grids, const fdlbm_opts *opts);

/* Create a batch.  grids, nu, cfl, blend: arrays of ncases; metrics and opts:
 * arrays of ncases or NULL.  All cases must share one precision.  The stream is
 * opts[0].stream, or a private non-blocking stream when NULL (graph capture
 * needs a non-legacy stream).  graph_steps > 0: fdlbm_batch_step replays a CUDA
 * graph of that many steps (rounded up to even) captured on first use, and
 * launches any remainder directly.  autotune != 0: time a few tile shapes
 * (block shapes of the staged node kernels, or tile heights of the fused sweep)
 * on this batch and keep the fastest (cached per batch signature for the
 * process); the states are reset to rest afterwards.
 * workspace: caller device memory of fdlbm_batch_workspace_bytes() bytes,
 * 256-byte aligned, or NULL (the library allocates). */
fdlbm_status fdlbm_batch_create(int ncases, const fdlbm_grid *grids, const fdlbm_metrics *metrics,
                                const double *nu, const double *cfl, const double *blend,
                                const fdlbm_opts *opts, int graph_steps, int autotune,
                                void *workspace, size_t workspace_bytes, fdlbm_batch_t *out);
fdlbm_t fdlbm_batch_case(fdlbm_batch_t b, int c);    /* NULL if out of range */
int fdlbm_batch_size(fdlbm_batch_t b);
long long fdlbm_batch_cells(fdlbm_batch_t b);        /* nodes of all cases */
/* Advance every case by n steps (asynchronous on the batch stream). */
fdlbm_status fdlbm_batch_step(fdlbm_batch_t b, int n);
/* How fdlbm_batch_step advances the cases:
 *  FUSED       the fused sweeps with Eq. 3.10 inside them over tiles of every
 *              case: one launch per step for the T2S2-FDLBM1 cases and one for
 *              the T2S2-FDLBM2 cases (FP32 batches; the default there);
 *  STAGED      one launch per stage and step of the staged kernels (the default
 *              otherwise);
 *  PERSISTENT  one cooperative launch for all the steps of a call (or of a graph
 *              replay): the fused sweep with one grid barrier per step where
 *              every case is T2S2-FDLBM1 in FP32, else the staged stages
 *              separated by grid barriers; every barrier wait is bounded (a timeout sets every case's error flag, which
 *              fdlbm_sync / fdlbm_reduce of a case report).
 * fdlbm_batch_set_mode synchronises the batch stream, drops a captured graph and
 * rebuilds the tables with the mode's default tile shape (no autotuning);
 * EUNSUPPORTED if FUSED does not apply. */
enum { FDLBM_BATCH_FUSED = 0, FDLBM_BATCH_STAGED = 1, FDLBM_BATCH_PERSISTENT = 2 };
fdlbm_status fdlbm_batch_set_mode(fdlbm_batch_t b, int mode);
int fdlbm_batch_mode(fdlbm_batch_t b);               /* -1 for NULL */
/* Synchronise the batch stream, then read the kernel-side failure flag of
 * every case (set when a bounded wait gave up: a grid barrier of PERSISTENT, a
 * row copy of a fused kernel).  Flags that are set are cleared and reported
 * once, as ECUDA with the number of cases in fdlbm_batch_last_error(); the
 * states of those cases are not valid (re-initialise them). */
fdlbm_status fdlbm_batch_sync(fdlbm_batch_t b);
/* Test hook for the failure path of PERSISTENT: the number of polls after which
 * a block gives up waiting at a grid barrier (default 2^24, well over a second
 * with the back-off sleeps).  0 makes every block but the last to arrive give
 * up at the first barrier, which sets the cases' flags without any fault or
 * hang.  Synchronises (fdlbm_batch_sync) and drops a captured graph. */
fdlbm_status fdlbm_batch_set_spin_limit(fdlbm_batch_t b, unsigned polls);
void *fdlbm_batch_stream(fdlbm_batch_t b);           /* cudaStream_t of the batch */
const char *fdlbm_batch_describe(fdlbm_batch_t b);
const char *fdlbm_batch_last_error(fdlbm_batch_t b);
void fdlbm_batch_destroy(fdlbm_batch_t b);           /* NULL-safe; releases every case */

/* Allocation-free reduction, for callers that cannot allocate device memory
 * where they need it (code whose device memory is all owned by a framework's
 * pool, a service loop that must keep a fixed footprint after start-up, a
 * thread that may not call cudaMalloc while other work is in flight).  The
 * paper has no counterpart; this is a library utility.
 *
 * Same quantities as fdlbm_reduce, computed from caller-owned device buffers:
 *   f         device, FP64 [9][ny][nx] f~ (the fdlbm_get_state layout);
 *   dzeta_dx, dmu_dy  device, FP64 metrics of length nx and ny;
 *   uprev     device, FP64 [2][ny][nx] previous velocity (u then v), or NULL;
 *   out       device, 3 FP64: Jacobian-weighted mass, residual against uprev
 *             (-1 without uprev; the absolute sqrt(sum |u - uprev|^2) when
 *             sum |u|^2 = 0), sum |u|^2.  Velocities are sum xi f / sum f, with
 *             no body-force correction.
 * Enqueued on `stream` (cudaStream_t, NULL = default); read `out` after the
 * stream completes.  No allocation of any kind: the scratch (3 doubles per grid
 * row) is a fixed device array of fdlbm_reduce_noalloc_max_rows() rows that
 * every GPU using the library holds until the process exits.  The first call on
 * a device looks up that array's device address, so make it before any stream
 * capture (and, after the device's context has been destroyed and made anew,
 * the next call looks it up again).  Every call shares the array: calls whose
 * kernels overlap on the GPU race and give wrong results.  Errors: EINVAL (NULL
 * pointer, nx or ny < 1), ETOOBIG (ny above the maximum), ECUDA (also, without
 * launching, when an earlier CUDA error is already pending on the thread). */
fdlbm_status fdlbm_reduce_noalloc(const double *f, int nx, int ny, const double *dzeta_dx,
                                  const double *dmu_dy, const double *uprev, double *out,
                                  void *stream);
int fdlbm_reduce_noalloc_max_rows(void);

/* Measurement utility (the paper has no counterpart): a launch of `blocks`
 * blocks of independent FP64 fused multiply-add chains, `iters` FMAs per chain,
 * enqueued on `stream` (cudaStream_t, NULL = default).  *flop (if not NULL) is
 * set to the floating-point operations it performs (2 per FMA).  Time it with
 * CUDA events on the same stream to measure the FP64 rate of the device, the
 * roofline denominator of the FP64 step.  out: device pointer to `blocks`
 * doubles (written only in a case that does not occur; it keeps the work).
 * Errors: EINVAL, ECUDA. */
fdlbm_status fdlbm_probe_fp64_fma(int blocks, int iters, double *out, void *stream, double *flop);

#ifdef __cplusplus
}
#endif

#endif /* FDLBM_H */
