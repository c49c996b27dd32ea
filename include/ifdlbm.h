/*
 * ifdlbm.h - C ABI of the GB300 (sm_103a) IFDLBM library.
 *
 * The library advances the incompressible finite-difference lattice
 * Boltzmann method (IFDLBM) of Chen, Chai, Zhao and Shi (arXiv 2306.07603)
 * for a power-law fluid in a lid-driven isosceles trapezoidal cavity that
 * is mapped to a uniform (xi, eta) computational grid (Sec. 4, Eq. 3.8),
 * and in cavities on general convex quadrilaterals (bilinear map,
 * ifdlbm_create_quad_batch).
 * One call of ifdlbm_step performs Steps (2)-(7) of the paper's calculation
 * process per time step, with Step (8)'s global relative error (Eq. 2.19)
 * formed on the last step of the call.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - Grids are nx x ny nodes; node (i, j) sits at xi = i/(nx-1),
 *    eta = j/(ny-1). j = 0 is the bottom wall, j = ny-1 the lid (Eq. 1.5).
 *    Host and device field arrays are row-major [ny][nx] (xi contiguous);
 *    distribution arrays are [9][ny][nx] in the D2Q9 order of Eq. (2.9).
 *  - Every compute step runs as sm_103a CUDA on the stream given at
 *    creation. There is no CPU fallback: without a CUDA device, creation
 *    fails with IFDLBM_ERR_CUDA.
 *  - The handle owns all device memory it allocates, through the allocator
 *    registered with ifdlbm_set_allocator (cudaMalloc/cudaFree if none).
 *    Pointers passed in are borrowed for the duration of the call only.
 *  - Functions taking HOST buffers synchronise the handle's stream before
 *    they return. Functions suffixed _dev take DEVICE pointers, enqueue
 *    their copies on the handle's stream and return without synchronising.
 *  - Return value: IFDLBM_OK (0) or a negative IFDLBM_ERR_* code; the text
 *    of the last error is available from ifdlbm_last_error(handle), or
 *    ifdlbm_last_error(NULL) for a failed create.
 *  - A handle is not thread safe: calls on one handle must not overlap.
 */
#ifndef IFDLBM_H
#define IFDLBM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define IFDLBM_OK 0
#define IFDLBM_ERR_INVALID_ARG (-1) /* argument out of its documented range */
#define IFDLBM_ERR_CUDA (-2)        /* a CUDA call failed (text in last_error) */
#define IFDLBM_ERR_OOM (-3)         /* the allocator returned NULL */
#define IFDLBM_ERR_DIVERGED (-4)    /* a non-finite velocity appeared in a step */
#define IFDLBM_ERR_TIMEOUT (-5)     /* a bounded device-side wait gave up */

/* Storage / arithmetic form of the distributions (pattern "precision"). */
#define IFDLBM_FP64 0    /* f-hat and all arithmetic in FP64 */
#define IFDLBM_FP32DEV 1 /* f-hat stored and updated in FP32 as deviations
                            g_i = f-hat_i - f^eq_i(P_ref, 0) from the rest
                            equilibrium at a reference pressure (Eq. 2.8 at
                            u = 0), P_ref re-based on the cavity's mean
                            pressure every 1024 steps (a uniform pressure
                            offset is a neutral, drifting mode). The metrics,
                            the power law of Eq. (1.4) (on the FP32 strain
                            rate) and all reductions are FP64 (see power_fp32
                            for an FP32 power); the relaxation-time plane is
                            stored in FP32. Every output includes P_ref. */

/* Step kernel organisation. */
#define IFDLBM_KERNEL_AUTO 0   /* FUSED for FP32DEV, STAGED for FP64 */
#define IFDLBM_KERNEL_STAGED 1 /* three launches per step, no recomputation */
#define IFDLBM_KERNEL_FUSED 2  /* one launch per step, eta-marching window */

/* Geometry of the isosceles trapezoid (Sec. 2, Eq. 3.8.1 with general L, H):
 * bottom edge of length L, height H, base angle theta_deg in (0, 90]; the
 * side walls lean outward so the lid spans L + 2 H cot(theta). theta_deg =
 * 90 is the square cavity (identity map). */
typedef struct {
  double L;
  double H;
  double theta_deg;
} ifdlbm_geometry;

/* Run options. ifdlbm_default_options fills the defaults noted here. */
typedef struct {
  double cfl;       /* Courant number, 0.5 (Sec. 5.1) */
  double c;         /* lattice speed, 1.0 (Sec. 5.1) */
  double eta_b;     /* blend of Eq. (2.5) in [0, 1]; default 0.5 */
  double gamma_min; /* zero-shear clamp of |gamma-dot|; <= 0 means 1e-3 U/H;
                       otherwise >= 1e-100 */
  double dt;        /* time step; <= 0: derived from cfl by dt_mode */
  double rho0;      /* reference density, 1.0 */
  int precision;    /* IFDLBM_FP64 (default) or IFDLBM_FP32DEV */
  int kernel;       /* IFDLBM_KERNEL_*; default AUTO */
  int graph_chunk;  /* steps per captured CUDA graph, even, >= 2; default 32;
                       0 disables graph capture */
  int fused_threads; /* FUSED: threads per CTA, 64, 128 or 256, two per
                        column; each CTA owns at most fused_threads/2 - 8
                        columns; 0 = 128 */
  int fused_rows;    /* FUSED: rows per CTA task (>= 2); 0 = automatic */
  int schedule;      /* FUSED: IFDLBM_SCHED_*; default GRID */
  int dt_mode;       /* IFDLBM_DT_*: how dt follows from cfl when dt <= 0 */
  int lambda_mode;   /* IFDLBM_LAMBDA_*: how Eq. (2.14) meets the strain rate */
  int power_fp32;    /* FP32DEV only, opt-in (default 0): 1 evaluates the power law
                        of Eq. (1.4) and the implicit solve of Eq. (2.14) in FP32
                        (relative error of lambda ~1e-6) instead of FP64; faster
                        on GB300's 1/64-rate FP64 pipe, but outside the FP32
                        deviation form, which keeps them in FP64. INVALID_ARG
                        with FP64. */
  int wall_pressure; /* IFDLBM_WALLP_*: the pressure the wall rule (Sec. 4) puts in
                        the wall node's equilibrium. ZEROTH (default): that of the
                        inner neighbour. FIRST: 2 P_nb - P_nnb, extrapolated along
                        the grid line through the next node (a reading the paper
                        leaves open). FIRST runs on the staged kernels: kernel
                        AUTO selects STAGED, FUSED is INVALID_ARG. */
} ifdlbm_options;

/* Pressure of the wall rule (ifdlbm_options.wall_pressure). */
#define IFDLBM_WALLP_ZEROTH 0
#define IFDLBM_WALLP_FIRST 1

/* Time-step rules ("c = 1, CFL = 0.5", Sec. 5.1). */
#define IFDLBM_DT_GRID 0          /* dt = cfl * min(L/(nx-1), H/(ny-1)) / c; on a skewed
                                     grid the contravariant Courant numbers exceed cfl
                                     and the two-stage scheme relies on collisions to
                                     stay stable (it fails for lambda/dt >~ 1) */
#define IFDLBM_DT_CONTRAVARIANT 1 /* dt = cfl * min(dxi / max|c_xi|, deta / max|c_eta|),
                                     the Courant number of the contravariant speeds
                                     of Eq. (3.4) (default); equal to GRID at 90 deg */

/* Relaxation time of Step (2). The paper lags it (text after Eq. 2.14): the
 * strain rate of Eqs. (2.12)-(2.13) is taken with the previous step's lambda.
 * The implicit form solves lambda = K max(gamma-dot(lambda), gamma_min)^(n-1)
 * / c_s^2 at every node, gamma-dot(lambda) = a / (2 lambda + dt) with a from
 * sum_i c_i c_i (f-hat_i - f^eq_i) (Eq. 2.18 at the same lambda), by a
 * bracketed Newton iteration in FP64 (the root is unique: the residual
 * increases strictly with lambda; in FP32 with the power_fp32 opt-in). Both
 * forms share steady states. The adjoint needs the lagged form. */
#define IFDLBM_LAMBDA_LAGGED 0   /* default */
#define IFDLBM_LAMBDA_IMPLICIT 1

/* Cavity-to-CTA schedules of the fused kernel. Tasks are strips of columns x
 * segments of rows of every cavity of the batch. */
#define IFDLBM_SCHED_GRID 0    /* one CTA per task */
#define IFDLBM_SCHED_STATIC 1  /* persistent CTAs (SMs x resident CTAs); CTA b takes
                                  the positions b, b + grid, ... of the tasks
                                  sorted largest first */
#define IFDLBM_SCHED_DYNAMIC 2 /* persistent CTAs taking the next position of that
                                  order from an atomic counter */

/* Result of ifdlbm_autotune. */
typedef struct {
  int fused_threads;
  int fused_rows;
  int schedule;
  int ntasks;
  double ms_per_step; /* mean event time of the trial steps */
  int candidates;     /* configurations timed */
  int pad;
} ifdlbm_tuning;

/* One cavity of a batch (pattern "batching"). */
typedef struct {
  int nx;
  int ny;
  ifdlbm_geometry geom;
  double Re;    /* power-law Reynolds number of Eq. (2.15.1), > 0 */
  double n;     /* power-law index of Eq. (1.4), > 0 */
  double U_lid; /* lid speed U of Eq. (1.5), > 0 */
} ifdlbm_cavity;

/* One cavity on a general convex quadrilateral (the trapezoid map of
 * Eq. (3.8.1) generalised to the bilinear map of its corners; the metrics
 * of Eqs. (3.2)-(3.3) then vary along both grid directions and eta_x need
 * not vanish). corners = {x0, y0, x1, y1, x2, y2, x3, y3}: bottom-left,
 * bottom-right, top-left, top-right; xi runs along the bottom edge and the
 * lid, eta up the side walls. The lid is the top edge and moves along it at
 * speed U_lid; the other walls and the two top corner nodes are at rest.
 * H is the reference length of Eq. (2.15.1). */
typedef struct {
  int nx;
  int ny;
  double corners[8];
  double H;     /* > 0 */
  double Re;    /* > 0 */
  double n;     /* > 0 */
  double U_lid; /* > 0 */
} ifdlbm_quad_cavity;

/* Scalar facts about one cavity of a handle. */
typedef struct {
  int nx, ny;
  int precision;
  int kernel;
  double dt;        /* time step */
  double K;         /* consistency coefficient U^(2-n) H^n / Re, Eq. (2.15.1) */
  double gamma_min; /* clamp in use */
  double eta_b;
  double courant_max; /* max over nodes/directions of dt(|c_xi|/dxi + |c_eta|/deta) */
  int64_t steps;      /* time steps taken so far */
  int64_t device_bytes; /* device memory owned by the whole handle */
  int64_t h2d_bytes;    /* bytes the handle copied host -> device at creation */
  int fused_threads, fused_rows, schedule, ntasks; /* fused kernel layout in use */
} ifdlbm_info_t;

typedef struct ifdlbm_ctx *ifdlbm_handle;

/* Device allocator hooks: alloc returns a device pointer of at least
 * `bytes` bytes usable on `stream`, or NULL; free releases it. `ctx` is
 * passed back unchanged. Process-wide; affects handles created afterwards.
 * Passing NULL for both restores cudaMalloc/cudaFree. */
typedef void *(*ifdlbm_alloc_fn)(size_t bytes, void *stream, void *ctx);
typedef void (*ifdlbm_free_fn)(void *ptr, size_t bytes, void *stream, void *ctx);
int ifdlbm_set_allocator(ifdlbm_alloc_fn alloc, ifdlbm_free_fn free_fn, void *ctx);

/* Fills *opt with the defaults listed in ifdlbm_options. */
int ifdlbm_default_options(ifdlbm_options *opt);

/* Creates one lid-driven trapezoidal cavity at rest (Step (1), Sec. 4):
 * f-hat = f = f^eq(P = 0, u) with u = 0 inside and on the walls, u = (U, 0)
 * on the lid nodes (impulsive start; the two top corners are wall nodes),
 * and lambda_prev equal to Eq. (2.14) at zero shear.
 *  nx, ny   >= 5 nodes along xi and eta
 *  g        L > 0, H > 0, 0 < theta_deg <= 90
 *  Re, n, U_lid  > 0 (Eqs. 1.4, 1.5, 2.15.1)
 *  opt      NULL for the defaults
 *  stream   cudaStream_t on which every device operation of the handle is
 *           enqueued (NULL: the legacy default stream)
 *  out      receives the handle
 * Errors: INVALID_ARG for out-of-range arguments, OOM, CUDA. */
int ifdlbm_create(int nx, int ny, ifdlbm_geometry g, double Re, double n, double U_lid,
                  const ifdlbm_options *opt, void *stream, ifdlbm_handle *out);

/* Creates `ncav` independent cavities (each as ifdlbm_create) that every
 * ifdlbm_step advances together in the same launches. `cavs` is a host
 * array of ncav entries; 1 <= ncav <= 4096. */
int ifdlbm_create_batch(int ncav, const ifdlbm_cavity *cavs, const ifdlbm_options *opt,
                        void *stream, ifdlbm_handle *out);

/* Creates `ncav` cavities on general quadrilaterals (ifdlbm_quad_cavity,
 * host array). The staged kernels keep one FP64 plane per metric and node
 * (xi_x, xi_y, eta_x, eta_y, x_eta, y_eta, J: 56 bytes per node). The fused
 * kernel has a general-quadrilateral variant for precision FP32DEV with the
 * lagged relaxation time (it forms each node's metrics from the map's
 * separable derivatives): there kernel AUTO selects FUSED and FUSED is
 * accepted; for FP64 or the implicit relaxation time AUTO selects STAGED and
 * FUSED is INVALID_ARG. The default time step applies the Courant number to the
 * largest contravariant speeds over all nodes (dt_mode CONTRAVARIANT);
 * dt_mode GRID without an explicit dt is INVALID_ARG. Every other call
 * takes the handle as it takes a trapezoid handle, except the adjoint
 * calls (INVALID_ARG). ifdlbm_eddies locates the eddies in (xi, eta) by
 * the same rule and maps their centres through the corners.
 * Errors: INVALID_ARG also for non-finite corners, H <= 0, or corners whose
 * Jacobian is not positive at all four of them (not convex and
 * counter-clockwise). */
int ifdlbm_create_quad_batch(int ncav, const ifdlbm_quad_cavity *quads,
                             const ifdlbm_options *opt, void *stream, ifdlbm_handle *out);

/* Advances every cavity of the handle by `nsteps` >= 0 time steps, Steps
 * (2)-(7) of Sec. 4 (Eqs. 2.8-2.18, 3.6-3.7, non-equilibrium extrapolation
 * walls). On the last step it also forms, per cavity, the global relative
 * errors of Eq. (2.19) between that step's input and output fields, the
 * max-norm velocity residual and the kinetic energy of Eq. (5.1).
 * Asynchronous: returns once the work is enqueued. A divergence flagged on
 * the device is reported by the next synchronising call. */
int ifdlbm_step(ifdlbm_handle h, int nsteps);

/* Macroscopic fields of cavity 0 at the current time, into HOST arrays of
 * nx*ny doubles ([ny][nx]); any pointer may be NULL to skip that field.
 *  rho  equivalent density rho0 + P / c_s^2 (the model carries P, Eq. 2.11)
 *  u, v velocity, Eq. (2.10)
 *  psi  stream function: psi = 0 on the bottom wall, integrated along each
 *       xi = const line, d psi = (u y_eta - v x_eta) d eta, trapezoidal rule.
 * Synchronises. */
int ifdlbm_macros(ifdlbm_handle h, double *rho, double *u, double *v, double *psi);

/* As ifdlbm_macros for cavity `cavity` of a batch, into HOST arrays. */
int ifdlbm_batch_macros(ifdlbm_handle h, int cavity, double *rho, double *u, double *v,
                        double *psi);

/* As ifdlbm_batch_macros into DEVICE arrays; does not synchronise. */
int ifdlbm_macros_dev(ifdlbm_handle h, int cavity, double *rho, double *u, double *v,
                      double *psi);

/* Residuals of cavity 0 from the last step taken, into HOST out[4]:
 *  out[0] E(u), out[1] E(P) of Eq. (2.19),
 *  out[2] max_nodes |u^n - u^(n-1)| / max_nodes |u^n| (max-norm residual),
 *  out[3] kinetic energy 1/2 sum |u|^2 J dxi deta of Eq. (5.1)
 *         (composite trapezoidal rule; J the Jacobian of Eq. 3.3).
 * All zero before the first step. Synchronises; returns DIVERGED if a step
 * produced a non-finite velocity. */
int ifdlbm_residual(ifdlbm_handle h, double *out);

/* Residuals of every cavity, HOST out[4 * ncav] in the order above. */
int ifdlbm_batch_residual(ifdlbm_handle h, double *out);

/* The same read without waiting: enqueues on the handle's stream the copy of
 * the [ncav][4] residuals into HOST out and, if status is not NULL, of the
 * status word into HOST *status (bit 0 set: some step produced a
 * non-finite velocity; bit 1 set: a TMA row load of the fused kernel did not
 * complete within its bounded wait, which synchronising calls report as
 * IFDLBM_ERR_TIMEOUT), and returns at once. out and status should be
 * page-locked (cudaHostAlloc or equivalent) for the copy to be
 * asynchronous. They are valid once the stream has reached the copy (an
 * event recorded after this call, or any synchronising call), so a caller
 * can read step n's residuals while step n + 1 runs. */
int ifdlbm_batch_residual_async(ifdlbm_handle h, double *out, unsigned *status);

/* State of cavity `cavity` in the paper's variables: fhat[9][ny][nx]
 * (f-hat of Eq. 2.3, full value, not the FP32 deviation) and
 * lambda_prev[ny][nx] (the relaxation time the next step's Eq. (2.18)
 * will use). HOST arrays; either may be NULL. Synchronises. */
int ifdlbm_get_state(ifdlbm_handle h, int cavity, double *fhat, double *lambda_prev);

/* Replaces the state of cavity `cavity` (HOST arrays, layouts as
 * ifdlbm_get_state; both required). The residual of the next step
 * compares against these fields. Synchronises. */
int ifdlbm_set_state(ifdlbm_handle h, int cavity, const double *fhat, const double *lambda_prev);

/* Time series without synchronising (unsteady runs, Sec. 5.3: probe
 * velocities and the kinetic energy of Eq. 5.1 over time). Both enqueue on
 * the handle's stream and return at once; results are valid once the stream
 * reaches them.
 *  ifdlbm_residual_dev: copies the [ncav][4] array of ifdlbm_batch_residual
 *    (E(u), E(P), max-norm residual, kinetic energy of the last step that
 *    formed them) into the DEVICE array out.
 *  ifdlbm_probe_dev: for n >= 0 probes, DEVICE int array probes[n][3] =
 *    (cavity, i, j), writes the DEVICE double array out[n][3] = (u, v, P) of
 *    Eqs. 2.10-2.11 at node (i, j) of that cavity at the current state (P is
 *    the pressure of Eq. 2.11, rho = rho0 + P / c_s^2). A probe outside its
 *    cavity yields NaNs; the probe array is read on the device only. */
int ifdlbm_residual_dev(ifdlbm_handle h, double *out);
int ifdlbm_probe_dev(ifdlbm_handle h, int n, const int *probes, double *out);

/* Copies of the whole batch state between the handle and caller-owned
 * DEVICE memory of ifdlbm_state_bytes(h) bytes (opaque layout, valid only
 * for the same handle). Used for checkpoints. Do not synchronise. */
int64_t ifdlbm_state_bytes(ifdlbm_handle h);
int ifdlbm_save_state_dev(ifdlbm_handle h, void *dst);
int ifdlbm_load_state_dev(ifdlbm_handle h, const void *src);

/* Scalar facts about cavity `cavity` (see ifdlbm_info_t). */
int ifdlbm_info(ifdlbm_handle h, int cavity, ifdlbm_info_t *info);

/* Waits for the handle's stream; returns DIVERGED or CUDA errors seen. */
int ifdlbm_sync(ifdlbm_handle h);

/* Releases the handle and all device memory it owns. NULL is a no-op. */
int ifdlbm_destroy(ifdlbm_handle h);

/* Text of the last error on `h` (or of the last failed create when h is
 * NULL). Valid until the next call on the same handle. */
const char *ifdlbm_last_error(ifdlbm_handle h);

/* Kernel timing. While enabled, every step kernel launch of `h` is
 * bracketed by CUDA events on the handle's stream (steps then run without
 * graph replay). ifdlbm_profile_read synchronises and returns, for kernel
 * `kernel` (IFDLBM_KPROF_*), the summed event time in milliseconds and the
 * number of launches since profiling was (re)enabled. Disabling discards
 * the records. */
#define IFDLBM_KPROF_COLLIDE 0 /* staged: Steps (2)-(3) */
#define IFDLBM_KPROF_HALF 1    /* staged: Step (4) */
#define IFDLBM_KPROF_FULL 2    /* staged: Steps (5)-(6) + residual partials */
#define IFDLBM_KPROF_REDUCE 3  /* residual reduction (Step 8) */
#define IFDLBM_KPROF_FUSED 4   /* fused: Steps (2)-(6) in one launch */
#define IFDLBM_KPROF_COUNT 5
int ifdlbm_profile(ifdlbm_handle h, int enable);
int ifdlbm_profile_read(ifdlbm_handle h, int kernel, double *total_ms, int64_t *launches);

/* Residuals between two sets of macroscopic fields, for callers that may
 * not allocate device memory. The paper has no counterpart: this is a
 * service of the library, not a step of the method.
 *
 * Some callers cannot call cudaMalloc: code that runs inside another
 * framework's stream-ordered memory pool or a fixed device-memory budget
 * (a multi-tenant service, a real-time loop), where an allocation would
 * synchronise the device, fragment the pool or fail at the worst moment.
 * This entry point allocates nothing, directly or through any library
 * (PyTorch's allocator included). Its scratch, one partial sum per 256
 * nodes, is a fixed 512 KiB array in device memory that every GPU which
 * loads libifdlbm.so holds until the process exits.
 *
 *  nx, ny   field size; nx * ny <= IFDLBM_STATIC_MAX_NODES, larger fields
 *           are rejected with IFDLBM_ERR_INVALID_ARG and a message
 *  u1, v1, p1  DEVICE arrays of nx*ny doubles: u, v, P at step n
 *  u0, v0, p0  DEVICE arrays of nx*ny doubles: u, v, P at step n-1
 *  out      DEVICE array of 3 doubles, written with E(u), E(P) of Eq. (2.19)
 *           and max|u^n - u^(n-1)| / max|u^n| (the same three values
 *           ifdlbm_residual returns for a handle's last step)
 *  stream   cudaStream_t the two kernels are enqueued on; the call does not
 *           synchronise
 * It works on the calling thread's current device. The first call on each
 * device is its set-up: it looks up the scratch array's device address
 * (cudaGetSymbolAddress) and loads the entry point's two kernels. Under lazy
 * module loading (the CUDA default) that is when the driver sets up this
 * module on the device, the 512 KiB array included, so the first call may
 * take device memory and can fail when none is left. Make that first call at
 * set-up time, before any stream capture and before the memory budget is
 * spent; later calls take nothing. Every
 * call shares the one array, and each call writes every partial it reads
 * (nothing carries over between calls); calls that overlap on the GPU (on
 * different streams, or from different threads) race on it and must be
 * serialised by the caller. */
#define IFDLBM_STATIC_MAX_NODES 2097152
int ifdlbm_residual_fields_static(int nx, int ny, const double *u1, const double *v1,
                                  const double *p1, const double *u0, const double *v0,
                                  const double *p0, double *out, void *stream);

/* Autotuner of the batched fused step (pattern "batching"): times
 * `trial_steps` >= 1 steps of every combination of fused_threads {64, 128,
 * 256}, rows per task {16, 32, 64, 128, 256} and schedule {GRID,
 * STATIC, DYNAMIC} on the handle's own cavities, starting each trial from
 * the same saved state, and keeps the fastest. The state is restored
 * afterwards, so the call does not advance the simulation. Needs a handle
 * using IFDLBM_KERNEL_FUSED. Synchronises; *best receives the choice. */
int ifdlbm_autotune(ifdlbm_handle h, int trial_steps, ifdlbm_tuning *best);

/* Discrete adjoint (reverse mode) of the step, for gradients of a scalar
 * objective with respect to n, Re and theta (pattern "differentiation").
 * Needs a handle created with IFDLBM_FP64 and IFDLBM_KERNEL_STAGED (and the
 * lagged relaxation time and zeroth-order wall pressure it differentiates). States
 * and adjoints are DEVICE buffers of ifdlbm_state_bytes(h) bytes in the
 * layout of ifdlbm_save_state_dev (adjoint entry k is d J / d state entry k).
 * dparams is a DEVICE array [ncav][3] to which d J / d n, d J / d Re and
 * d J / d theta_deg (theta in degrees) are ADDED. Asynchronous on the
 * handle's stream; the first call allocates the adjoint scratch.
 *
 * ifdlbm_adjoint_seed_energy: J = the kinetic energy of Eq. (5.1) of every
 *   cavity at `state` (composite trapezoidal rule, J dxi deta area element);
 *   writes adj = dJ/dstate and adds the direct theta term (through the
 *   Jacobian of Eq. 3.3) to dparams.
 * ifdlbm_adjoint_step: with state_n the state before step n (Steps 2-7) and
 *   adj the adjoint of the state after it, recomputes step n (see
 *   ifdlbm_adjoint_step_saved for a sweep that keeps it) and replaces adj
 *   by the adjoint of state_n, adding the step's parameter terms (n and Re
 *   through K of Eq. 2.15.1 and the exponent of Eq. 1.4; theta through the
 *   contravariant velocities of Eq. 3.4) to dparams. */
int ifdlbm_adjoint_seed_energy(ifdlbm_handle h, const void *state, void *adj, double *dparams);
int ifdlbm_adjoint_step(ifdlbm_handle h, const void *state_n, void *adj, double *dparams);

/* Seed for J = sum over cavities k of psi_k(i_k, j_k), the stream function
 * (psi = 0 on the bottom wall, trapezoidal rule along xi = const lines) at
 * one node per cavity given in the HOST array nodes[2k] = i_k, nodes[2k+1] =
 * j_k (0 <= i_k < nx, 0 <= j_k < ny). With the node of the primary eddy
 * (ifdlbm_eddies(...)[0].i, .j) this is the gradient of psi_min, the
 * primary-vortex strength, wherever its minimising node does not change.
 * Writes adj = dJ/dstate and adds the direct theta term (through x_eta of
 * Eq. 3.8.2) to dparams. Asynchronous; INVALID_ARG for a node outside its
 * cavity. */
int ifdlbm_adjoint_seed_psi(ifdlbm_handle h, const void *state, const int *nodes, void *adj,
                            double *dparams);

/* Forward intermediates of a step, kept for the adjoint sweep so that it
 * need not recompute them (the same adjoint handles as above).
 *
 * ifdlbm_intermediate_bytes: bytes of one step's intermediates: f-bar^+
 *   (Eq. 2.16), f-hat^+ (Eq. 2.15) and f(t + dt/2) (Eq. 2.17), 27 planes of
 *   the handle's precision in its plane layout; -1 for a NULL handle.
 * ifdlbm_save_intermediates_dev: copies the intermediates of the handle's
 *   last ifdlbm_step into the DEVICE buffer dst (ifdlbm_intermediate_bytes
 *   bytes, owned by the caller), on the handle's stream. The last step must
 *   have been a single step of this handle (ifdlbm_step(h, 1)); any later
 *   step or adjoint call overwrites the source. INVALID_ARG for a NULL
 *   argument or a handle the adjoint does not take.
 * ifdlbm_adjoint_step_saved: ifdlbm_adjoint_step with the forward step
 *   given instead of recomputed: state_np1 is the state after step n
 *   (ifdlbm_save_state_dev after the step) and inter its intermediates
 *   (ifdlbm_save_intermediates_dev after the same step). The result is the
 *   same bit for bit (the same kernels formed the intermediates). All
 *   buffers are DEVICE buffers; the same errors as ifdlbm_adjoint_step. */
int64_t ifdlbm_intermediate_bytes(ifdlbm_handle h);
int ifdlbm_save_intermediates_dev(ifdlbm_handle h, void *dst);
int ifdlbm_adjoint_step_saved(ifdlbm_handle h, const void *state_n, const void *state_np1,
                              const void *inter, void *adj, double *dparams);

/* Self-test of the FP64 power the FP64 form uses for Eq. (1.4): for n
 * DEVICE doubles x (finite, > 0) writes fast[k] = the library's
 * table-driven x^m and ref[k] = CUDA's pow(x[k], m), on the handle's stream
 * (no sync). */
int ifdlbm_selftest_pow(ifdlbm_handle h, int n, const double *x, double m, double *fast,
                        double *ref);

/* Test hook of the fused kernel's failure path (no counterpart in the paper).
 * While `enable` is nonzero the fused kernel issues no TMA row loads, so that
 * every bounded wait for one runs out (after about a second per warp); the
 * kernel records that in the status word, which the next synchronising call
 * reports as IFDLBM_ERR_TIMEOUT. The state computed meanwhile is meaningless;
 * the device context stays usable. Synchronises; drops captured graphs.
 * Errors: INVALID_ARG for a NULL handle or one on the staged kernels. */
int ifdlbm_inject_tma_timeout(ifdlbm_handle h, int enable);

/* Self-test of the FP64 power the FP32-deviation form uses for Eq. (1.4)
 * (FP32 strain rate, FP64 result): for n DEVICE doubles x[k] whose float
 * roundings xf_k are normal and > 0, writes out[k] = C xf_k^m as the library
 * evaluates it for cavity `cavity` of the handle (m = (n - 1)/2, C = K/c_s^2,
 * the cavity's own table) and out[n + k] = C * CUDA's pow(double(xf_k), m).
 * `out` is a DEVICE array of 2n doubles; on the handle's stream (no sync).
 * Errors: INVALID_ARG for a bad handle, cavity or pointers. */
int ifdlbm_selftest_pow_tab(ifdlbm_handle h, int cavity, int n, const double *x, double *out);

/* Self-test of the FP32 power the FP32-power opt-in uses for Eq. (1.4):
 * for n DEVICE doubles x[k] (finite, > 0 after rounding to float) writes
 * out[k] = float(x[k])^float(m) as the library evaluates it, widened to
 * double, on the handle's stream (no sync). */
int ifdlbm_selftest_pow_f32(ifdlbm_handle h, int n, const double *x, double m, double *out);

/* Number of kernel launches the library has enqueued since the process
 * started (graph replays count every kernel node). */
int64_t ifdlbm_launch_count(void);

/* Eddy centres of a steady cavity flow, as tabulated in Tables 1-3 (Sec. 5.1):
 * the primary eddy and the two counter-rotating bottom-corner eddies.
 *
 *  - primary: the interior node (0 < i < nx-1, 0 < j < ny-1) of smallest psi
 *    (psi = 0 on the bottom wall and d psi = u dy - v dx, so the clockwise
 *    eddy of a lid moving in +x has psi < 0);
 *  - bottom-left / bottom-right: among interior nodes with eta <= 1/2 and
 *    xi < 1/2 (left) or xi >= 1/2 (right), the strict local maximum of psi
 *    (larger than its 8 neighbours) with the largest psi > 0.
 *
 * Each centre is refined below the grid spacing by the least-squares
 * quadratic psi ~ a + b s + c t + d s^2 + e s t + f t^2 over the 3 x 3 nodes
 * around the extremum node (s, t its offsets in nodes), taking the
 * stationary point when the quadratic has one there of the same kind within
 * one node, else the node itself. xi = (i + s)/(nx-1), eta = (j + t)/(ny-1)
 * are mapped to (x, y) by the map of Eq. (3.8.1) with the cavity's L, H and
 * theta. */
typedef struct {
  double x, y;     /* physical centre */
  double xi, eta;  /* computational coordinates of the centre */
  double psi;      /* fitted psi at the centre */
  int i, j;        /* extremum node */
  int found;       /* 1 if the eddy exists, else 0 and the rest is zero */
  int refined;     /* 1 if the quadratic fit moved the centre off the node */
} ifdlbm_eddy;

/* Host-only, no GPU: eddies of a HOST psi array [ny][nx] (nx, ny >= 3) of a
 * cavity with geometry g. out[0] primary, out[1] bottom-left, out[2]
 * bottom-right. */
int ifdlbm_find_eddies(int nx, int ny, ifdlbm_geometry g, const double *psi,
                       ifdlbm_eddy out[3]);

/* The same for cavity `cavity` of a handle at its current state (forms psi
 * as ifdlbm_batch_macros does; synchronises). */
int ifdlbm_eddies(ifdlbm_handle h, int cavity, ifdlbm_eddy out[3]);

#ifdef __cplusplus
}
#endif

#endif /* IFDLBM_H */
