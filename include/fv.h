/*
 * libfv: FP64 structured-grid Euler solver for GB300 (sm_103a), C ABI.
 *
 * The library advances the semi-discrete finite-volume form of the Euler
 * equations,   |Omega_k| dU/dt + R_h(U) = 0          (paper Eq. (4)),
 * with the spatial residual of Eq. (5) (source term S = 0),
 *              R_h = sum over the cell's faces of F.n ds,
 * face states from the MUSCL extrapolation of conserved variables, Eq. (6),
 * with the minmod limiter, and F the Roe approximate-Riemann flux with
 * Harten's entropy fix on the acoustic waves (the paper names neither flux nor
 * limiter; these are the pinned readings).  Time marching is the three-stage
 * SSP Runge-Kutta scheme (the paper: "an explicit Runge-Kutta time marching
 * method", Sec. 3.2) with a CFL time step.
 *
 * Data layout (struct of arrays, the SoA layout of Sec. 3.1): a state is
 * float64, contiguous, U[v][z][y][x] with x fastest; v = 0..nvar-1 indexes
 * (rho, rho*u, rho*v[, rho*w], rho*e_t); nvar = 4 in 2D and 5 in 3D.  Only
 * interior cells are stored: ghost cells are generated inside the kernels
 * from the boundary conditions.
 *
 * Pointers.  State and residual arrays may be device pointers (used in place,
 * stream-ordered on the context's stream, the call returns without waiting)
 * or host pointers (the call copies them to the device and back through a
 * staging buffer owned by the context and waits for the copies).  The caller
 * owns every array it passes; the context owns its workspaces.
 *
 * Errors.  Every call returns an fv_status.  Argument errors are detected on
 * the host before anything is launched.  Device-side conditions (a cell with
 * rho <= 0, p <= 0 or a NaN seen by the time-step kernel; a bounded wait that
 * ran out) set flags in device memory that are reported by the next call that
 * waits for the device (fv_sync, or any call given a host output pointer).
 * No call aborts the process or throws.
 */
#ifndef FV_H
#define FV_H

#ifdef __cplusplus
extern "C" {
#endif

typedef enum fv_status {
  FV_OK = 0,
  FV_EINVAL = 1,         /* an argument is out of range or inconsistent */
  FV_ENOMEM = 2,         /* device or host allocation failed */
  FV_ECUDA = 3,          /* a CUDA runtime or driver call failed */
  FV_ENONPHYSICAL = 4,   /* a cell had rho <= 0, p <= 0 or a NaN */
  FV_ETIMEOUT = 5,       /* a bounded device-side wait gave up */
  FV_EUNSUPPORTED = 6    /* valid request the library does not support */
} fv_status;

enum { FV_BC_PERIODIC = 0, FV_BC_TRANSMISSIVE = 1 };

/* A uniform Cartesian single-block grid: dim = 2 or 3, n = cells per axis
 * (n[2] = 1 in 2D), len = domain extent per axis (spacing len/n), bc = per
 * axis (low, high) FV_BC_PERIODIC (must be set on both sides) or
 * FV_BC_TRANSMISSIVE (zero-gradient ghost cells). */
typedef struct fv_grid {
  int dim;
  int n[3];
  double len[3];
  int bc[3][2];
} fv_grid;

enum { FV_LIM_MINMOD = 0, FV_LIM_VANLEER = 1, FV_LIM_NONE = 2 };
enum { FV_RECON_CONSERVED = 0, FV_RECON_PRIMITIVE = 1 };

/* gamma: ratio of specific heats (1.4).  cfl: CFL number (0.5).
 * eps, kappa: MUSCL parameters of Eq. (6); eps = 1 gives second order.
 * limiter: the Psi of Eq. (6) -- FV_LIM_MINMOD (Psi(r) = max(0, min(1, r)),
 * the default), FV_LIM_VANLEER (Psi(r) = (r + |r|)/(1 + |r|)) or FV_LIM_NONE
 * (Psi = 1: the unlimited kappa-scheme, kappa = -1 upwind, 0 Fromm, 1/3 third
 * order, 1 central).  With either limiter the two kappa-weighted limited
 * slopes are equal, so kappa matters only for FV_LIM_NONE.  Batched contexts
 * and the adjoint support FV_LIM_MINMOD only.
 * efix: Harten entropy-fix width as a fraction of the Roe sound speed (0.1),
 * 0 <= efix < 1 (the fix stays within one acoustic wave's sonic region); 0
 * disables the fix.
 * recon: the variables Eq. (6) extrapolates -- FV_RECON_CONSERVED (Sec. 3.1,
 * the default) or FV_RECON_PRIMITIVE (rho, velocity, p; the face states are
 * converted back to conserved variables for the flux).  Primitive
 * reconstruction is not supported by batched contexts, the adjoint or the
 * z-marching kernel (launch field march). */
typedef struct fv_scheme {
  double gamma, cfl, eps, kappa, efix;
  int limiter;
  int recon;
} fv_scheme;

enum { FV_LOADER_TMA = 0, FV_LOADER_PLAIN = 1 };

/* Launch parameters of one kernel: the tunables of the autotuner.
 * Tiled kernels (residual and RK stages): cells per CTA tile (tile[0] even,
 * 2..252 per axis, tile[2] = 1 in 2D), threads per CTA (a multiple of 32,
 * 32..256; 32..192 for 3D box tiles); grid must be 0 (one CTA per tile covers
 * the domain); loader
 * FV_LOADER_TMA stages tiles with TMA when the grid allows it (even nx, a
 * 16-byte aligned state, tile + halo no larger than the grid) and falls back
 * to plain loads otherwise, FV_LOADER_PLAIN always uses plain loads.
 * march (3D only): 0 = box tiles of tile[0] x tile[1] x tile[2] cells;
 * 1 = x-y tiles of tile[0] x tile[1] columns that march along z through
 * chunks of tile[2] planes (1..nz), computing every z-face once per chunk.
 * Time-step reduction: threads per CTA (32..1024) and grid = number of CTAs
 * (0 = 2048 / threads per SM, filling every SM); tile, loader and march are
 * ignored. */
typedef struct fv_kernel_cfg {
  int tile[3];
  int threads;
  int grid;
  int loader;
  int march;
} fv_kernel_cfg;

/* Kernel structure of a stage.
 * FV_FUSED (the default): one kernel per RK stage -- reconstruction, flux,
 *   residual and update together (launch fields stage[] and dt).
 * FV_SPLIT: the kernel structure of the paper's solver (Sec. 3.4): per axis a
 *   limiter kernel (the MUSCL face states of Eq. (6)) and a flux kernel (the
 *   Roe flux of every face), then a source kernel (-|Omega| S of Eq. (5), or
 *   0), a right-hand-side kernel (the flux differences of Eq. (5)) and an
 *   update kernel (the SSP-RK3 stage), with face states, fluxes and the
 *   residual held in device memory between them: 7 kernels per stage in 2D,
 *   9 in 3D.  Each is a grid-stride loop over its items (faces or cells, x
 *   fastest) launched with split[k].grid CTAs (the paper's gang count; 0 =
 *   one item per thread over the whole domain) of split[k].threads threads
 *   (its vector length; 32..512, a multiple of 32); the other fields of
 *   split[k] are ignored.  Slots: FV_SK_LIMITER + axis, FV_SK_FLUX + axis,
 *   FV_SK_SOURCE, FV_SK_RHS, FV_SK_UPDATE (the z slots are unused in 2D).
 *   The time-step reduction (dt) is the same as in FV_FUSED.  Batched
 *   contexts support FV_FUSED only; the face-state, flux and residual arrays
 *   (3 x nvar x faces per axis + nvar x cells doubles) are allocated on the
 *   first split launch and kept by the context. */
enum { FV_FUSED = 0, FV_SPLIT = 1 };
enum { FV_SK_LIMITER = 0, FV_SK_FLUX = 3, FV_SK_SOURCE = 6, FV_SK_RHS = 7, FV_SK_UPDATE = 8, FV_SK_COUNT = 9 };

/* stage[s]: RK stage s+1 (fv_residual uses stage[0]); dt: time-step
 * reduction; mode: FV_FUSED or FV_SPLIT; split[]: the FV_SPLIT kernels
 * (ignored, and may be zero, in FV_FUSED mode). */
typedef struct fv_launch {
  fv_kernel_cfg stage[3];
  fv_kernel_cfg dt;
  int mode;
  fv_kernel_cfg split[FV_SK_COUNT];
} fv_launch;

typedef struct fv_ctx fv_ctx;

/* Fill *l with the default launch configuration for grid g (one tile shape
 * and thread count for all stages): mode FV_FUSED; 2D 64x16 box tiles with
 * 192 threads (32x32 tiles with 256 threads in a batched context created
 * without a launch); 3D
 * 8x8x8 box tiles with 192 threads; time-step reduction 512 threads, four
 * CTAs per SM; split kernels 128 threads, grid 0 (one item per thread: the
 * analogue of a directive compiler's default vector length and gang count).
 * Returns FV_EINVAL for a bad grid. */
int fv_default_launch(const fv_grid *g, fv_launch *l);

/* Create a solver context for ngrids grids.  ngrids = 1: one grid, 2D or 3D.
 * ngrids > 1: a batch of independent 2D grids of any sizes (3D batches return
 * FV_EUNSUPPORTED), stored packed (see fv_layout) and advanced together by
 * fv_run / fv_rk_step in one persistent cooperative kernel launch per call,
 * each grid with its own CFL time step; the batch uses launch stage[0]'s tile
 * and threads for every stage.  fv_residual and fv_time_step need ngrids = 1.
 * Allocates the RK stage buffers and reduction scratch on the current CUDA
 * device.  stream: a cudaStream_t on which every later call
 * is ordered (NULL = the legacy default stream).  l = NULL selects
 * fv_default_launch.  On success *out owns the context (free with
 * fv_destroy). */
int fv_init(fv_ctx **out, const fv_grid *grids, int ngrids, const fv_scheme *s, const fv_launch *l,
            void *stream);

/* Layout of the packed state of a context: grid g's SoA block (nvar x cells
 * doubles, the layout above) starts at offsets[g] doubles; offsets[ngrids] is
 * the total.  offsets: host array of ngrids + 1 entries.  Blocks start on
 * 256-byte boundaries. */
int fv_layout(const fv_ctx *ctx, long long *offsets, int ngrids);

/* Replace / read the launch configuration (validated against the device).
 * fv_set_launch waits for the context's queued work and drops its captured
 * graphs. */
int fv_set_launch(fv_ctx *ctx, const fv_launch *l);
int fv_get_launch(const fv_ctx *ctx, fv_launch *l);

/* Cell-averaged source S_h of Eq. (5): S is a caller-owned DEVICE array of
 * nvar*ncells doubles in the layout of U (not copied: it must stay valid and
 * unchanged while the context uses it), or NULL for S = 0 (the default).
 * Every later residual, RK step and run includes it: R = sum F.n ds -
 * |Omega| S, dU/dt = -R/|Omega|.  Waits for the context's queued work and
 * drops its captured graphs when S changes.  FV_EINVAL for a host pointer,
 * FV_EUNSUPPORTED for a batched context.  The adjoint is unchanged (S does
 * not depend on U). */
int fv_set_source(fv_ctx *ctx, const double *S);

/* Spatial residual R_h of Eq. (5): R = sum over faces of F.n ds - |Omega| S
 * (S = 0 unless set with fv_set_source), face areas included (not divided by
 * |Omega|).  U, R: nvar*ncells doubles (R may not alias U).  rnorm2: NULL, or
 * nvar doubles (device or host) receiving sum over cells of R_v^2 per
 * conserved variable. */
int fv_residual(fv_ctx *ctx, const double *U, double *R, double *rnorm2);

/* CFL time step dt = cfl / max over cells of sum_d (|u_d| + c) / dx_d.
 * dt_out: a host pointer (the call waits) or a device pointer (written
 * stream-ordered).  Non-physical cells make the call return FV_ENONPHYSICAL
 * when dt_out is a host pointer. */
int fv_time_step(fv_ctx *ctx, const double *U, double *dt_out);

/* One SSP-RK3 step applied in place to U:
 *   U1 = U + dt L(U),  U2 = 3/4 U + 1/4 (U1 + dt L(U1)),
 *   U <- 1/3 U + 2/3 (U2 + dt L(U2)),   L(U) = -R_h(U) / |Omega|.
 * dt > 0 is used as given; dt <= 0 takes the CFL step of U.  dt_used: NULL or
 * a host pointer that receives the step taken (the call then waits). */
int fv_rk_step(fv_ctx *ctx, double *U, double dt, double *dt_used);

/* nsteps SSP-RK3 steps in place, replayed from CUDA graphs captured on the
 * first call for this U pointer and dt mode.  dt_fixed > 0 holds the step;
 * otherwise every step takes the CFL step of its starting state.  t_out:
 * NULL (asynchronous) or a host pointer receiving the simulated time -- one
 * double per grid (ngrids of them) -- (the call waits and reports device-side
 * flags).  Batched contexts: U is the packed state, and a grid barrier that
 * waits longer than 2 s ends the kernel with FV_ETIMEOUT.
 * A host state U (single-grid contexts, fused kernels, box-tiled stage 1)
 * gives the same bits as a device state, with the copies overlapped: the
 * first step's stage 1 computes its flux differences band by band as the
 * state arrives and forms U1 from them once the CFL step is known
 * (allocates, on first use, a device buffer of dim states for them, plus a
 * second stream; without that memory the state is copied in whole first,
 * with the same result), and on page-locked host memory mapped into the device's
 * address space the last stage writes the result to U directly (pageable
 * memory: copied back band by band). */
int fv_run(fv_ctx *ctx, double *U, int nsteps, double dt_fixed, double *t_out);

/* Discrete adjoint (vector-Jacobian products), FP64, single-grid contexts.
 * what = FV_VJP_RESIDUAL: out = (dR_h/dU)^T lambda, R_h of Eq. (5) with face
 *   areas as fv_residual returns it (dt ignored).
 * what = FV_VJP_RKSTEP: out = (dU^{n+1}/dU^n)^T lambda for one SSP-RK3 step
 *   of fv_rk_step with the step held fixed at dt > 0 (the CFL step's
 *   dependence on U is not differentiated).
 * U (the state the Jacobian is taken at), lambda and out: caller-owned device
 * arrays of nvar*ncells doubles; out must not alias U or lambda.
 * Non-differentiable points follow the forward-mode convention: |x|' =
 * sign(x) with sign(+0) = +1; the entropy fix and the limiter take the branch
 * the forward pass took; minmod(a, b) passes the derivative of the argument it
 * returns (b on ties) and none when a and b do not share one strict sign.
 * Stream-ordered; allocates two adjoint work states on first use. */
enum { FV_VJP_RESIDUAL = 0, FV_VJP_RKSTEP = 1 };
int fv_adjoint_vjp(fv_ctx *ctx, int what, const double *U, const double *lambda, double dt, double *out);

/* One SSP-RK3 step of fv_rk_step at the fixed step dt > 0, in place on the
 * device state U, that also writes its two stage states (Eq. (4)):
 *   U1 = U + dt L(U),  U2 = 3/4 U + 1/4 (U1 + dt L(U1))
 * into caller-owned device arrays U1, U2 of the state's size (distinct from
 * U and from each other).  U after the call is bit for bit fv_rk_step's.  For
 * the discrete adjoint of a run: with the stage states kept, the step's VJP
 * (fv_adjoint_vjp_stages) does not recompute them.  Single-grid contexts
 * (FV_EUNSUPPORTED otherwise); FV_EINVAL for dt <= 0, host pointers or
 * aliased arrays.  Stream-ordered; returns without waiting. */
int fv_rk_step_stages(fv_ctx *ctx, double *U, double dt, double *U1, double *U2);

/* The FV_VJP_RKSTEP product of fv_adjoint_vjp, out = (dU^{n+1}/dU^n)^T
 * lambda at the fixed step dt > 0, from the step's stage states U1, U2 as
 * fv_rk_step_stages wrote them for the same U and dt (not recomputed): the
 * same bits as fv_adjoint_vjp.  Device arrays of the state's size; out must
 * not alias any input.  Same support and errors as fv_adjoint_vjp. */
int fv_adjoint_vjp_stages(fv_ctx *ctx, const double *U, const double *U1, const double *U2, const double *lambda,
                          double dt, double *out);

/* Wait for all work of the context and report (then clear) device-side
 * flags: FV_ENONPHYSICAL, FV_ETIMEOUT, or FV_OK. */
int fv_sync(fv_ctx *ctx);

/* Free the context and its device memory (waits for its work first). */
void fv_destroy(fv_ctx *ctx);

/* Static description of a status code. */
const char *fv_strerror(int status);

/* ------------------------------------------------------------------------
 * Autotuning (paper Sec. 3.3-3.6): a fully connected network regresses the
 * run time of one SSP-RK3 step on the launch parameters of the kernels, is
 * trained on a random sample of the tuning space, and picks the
 * configuration to use.
 * ---------------------------------------------------------------------- */

/* Training hyperparameters (Table "para-setting"): L2 coefficient alpha
 * (1e-4), Adam beta1 (0.95), beta2 (0.90), learning rate (0.0009), numerical
 * stability eps (1e-9), tolerance tol (1e-6) with n_iter_no_change (10)
 * epochs, batch (200), max_epochs (200). */
typedef struct fv_mlp_hyper {
  double alpha, beta1, beta2, lr, eps, tol;
  int batch, max_epochs, n_iter_no_change;
} fv_mlp_hyper;

/* Train the surrogate network on the device, FP64.  nl weight layers with
 * widths sizes[0..nl] (sizes[0] = features, sizes[nl] = 1, each <= 1024,
 * nl <= 8): ReLU hidden layers, identity output.  params: device array packed
 * [W_0 (sizes[0] x sizes[1], row-major), b_0, W_1, b_1, ...], updated in
 * place.  X: device [n][sizes[0]]; y: device [n]; order: device int32
 * [epochs][n], the sample indices of each epoch, taken in minibatches of
 * h->batch.  Loss per minibatch: 1/2 mean (y_hat - y)^2 + alpha/(2B) sum W^2;
 * Adam with bias corrections; stops early once the epoch loss has not
 * improved by h->tol for more than h->n_iter_no_change epochs (0 = never).
 * loss_out: NULL or a host array [epochs] of mean epoch losses; *epochs_run:
 * epochs done.  Allocates its workspace, waits for completion. */
int fv_mlp_train(int nl, const int *sizes, double *params, const double *X, const double *y, long n,
                 const int *order, int epochs, const fv_mlp_hyper *h, double *loss_out, int *epochs_run,
                 void *stream);

/* out[i] = network output for row i of X (device [n][sizes[0]]), out device [n]. */
int fv_mlp_predict(int nl, const int *sizes, const double *params, const double *X, long n, double *out,
                   void *stream);

/* Tuning options; zero fields take the defaults in brackets. */
typedef struct fv_tune_opts {
  int samples;     /* random configurations timed, split 75% train / 25% test [1000] */
  int steps;       /* SSP-RK3 steps timed per measurement, after one warm-up step [2] */
  int repeats;     /* measurements per configuration, median taken [1] */
  int candidates;  /* random configurations scored by the network [200000] */
  int top;         /* best-predicted candidates re-measured [16] */
  int exhaustive;  /* 1: also time every configuration of the reduced space [0] */
  int final_repeats; /* repeats of the final default / tuned / exhaustive timings [5] */
  int rounds;      /* surrogate rounds: retrain on all measurements, re-measure the top predictions [3] */
  int refine;      /* coordinate-descent sweeps around the best measured configuration [2]; -1: none */
  unsigned long long seed; /* SplitMix64 seed [1] */
  int hidden[4];   /* hidden-layer widths, 0-terminated; all 0 = (128, 64, 32) */
  fv_mlp_hyper mlp;
} fv_tune_opts;

typedef struct fv_tune_report {
  double t_default;       /* s per SSP-RK3 step, default launch */
  double t_tuned;         /* s per step, the returned launch */
  double t_search;        /* s per step, the best launch the search itself found */
  double t_best_sampled;  /* s per step, best of the random sample */
  double t_exhaustive;    /* s per step, best of the reduced space (0 if not run) */
  double r2_train, r2_test; /* Eq. (7) on run times, training / held-out samples */
  double space_size;      /* points in the full tuning space */
  int n_params;           /* tuning parameters (fused: 14 in 2D, 20 in 3D; split: 14, 18) */
  int n_train, n_test, epochs, n_measured, n_exhaustive;
  int rounds, n_refined;  /* surrogate rounds run; measurements made by the refinement */
  int chosen;             /* the returned launch: 0 the search's, 1 the default, 2 the exhaustive best */
  fv_launch exhaustive_best;
  fv_launch search_best;  /* the best launch the search itself found (timed as t_search) */
} fv_tune_report;

/* Tune the launch configuration of ctx for the state U (device or host; not
 * modified: timing runs on a copy in the context's staging buffer), in the
 * kernel structure of its current launch (mode).
 * FV_SPLIT space, the paper's (Sec. 3.4, Table "tuning-parameters"): per
 * split kernel a gang count (grid) in {100, 200, ..., 1000} and a vector
 * length (threads) in {32, 64, ..., 384} -- 14 parameters over 10^7 x 12^7
 * points in 2D, 18 in 3D.
 * FV_FUSED space: per RK-stage kernel tile_x in {8,16,32,64,128}, tile_y in
 * {2,4,8,16,32} (3D: tile_x {8,16,32}, tile_y {4,8,16}, tile_z {2,4,8}, and
 * the kernel: box tiles or z-marching with chunks of 8 x tile_z planes),
 * threads in {64,96,...,256}, loader in {TMA, plain}; time-step kernel
 * threads in {128,256,512,1024} and grid in {1,2,4,8} x SMs.
 * Procedure: time the default launch (a training sample when it lies in the
 * space) and opts->samples random valid configurations; train the network
 * (features: log2 of the parameters, standardised; target: log time,
 * standardised); score opts->candidates random configurations; re-measure
 * the opts->top best predicted; repeat for opts->rounds rounds, each
 * retrained on everything measured so far (the held-out 25% of the random
 * sample excepted); then refine the best measured configuration by
 * coordinate descent (each parameter in turn over its value set).  With
 * opts->exhaustive an exhaustive search of a reduced space is timed:
 * FV_FUSED, every configuration with one shared (tile, threads) for the
 * three stages, box tiles, TMA loads and the default time-step kernel;
 * FV_SPLIT, one shared (gang, vector) for every kernel (120 points).
 * Finally the search's best, the default and (if run) the exhaustive best
 * are timed interleaved opts->final_repeats times; the fastest by median is
 * returned in *best and installed in ctx.  rep may be NULL.  Waits for
 * completion. */
int fv_tune(fv_ctx *ctx, const double *U, const fv_tune_opts *opts, fv_launch *best, fv_tune_report *rep);

/* The autotuner's search space for a dim-dimensional grid in kernel
 * structure mode (FV_FUSED or FV_SPLIT): *n_params tuning parameters and
 * *size points (the product of the value-set sizes listed at fv_tune; in 2D
 * FV_SPLIT is the paper's space, Sec. 3.4: 14 parameters over 10^7 x 12^7
 * points).  Host only: needs no GPU.  Returns FV_EINVAL unless dim is 2 or 3,
 * mode is valid and both pointers are non-NULL. */
int fv_tune_space(int dim, int mode, int *n_params, double *size);

/* The residual and, if rnorm2 != NULL, sum over cells of R_v^2 per variable,
 * without a context and without allocating anything: the values fv_residual
 * returns on a context created with the same grid and scheme and no source
 * set (S = 0).  The paper has no counterpart: this is a facility for callers
 * that cannot allocate device memory when they call -- services that fix
 * their device-memory budget at start-up, plug-ins running inside an
 * application that owns the device's memory, hosts that cannot afford the
 * device-wide synchronisation cudaFree implies.
 * U, R (nvar*ncells doubles, R not aliasing U) and rnorm2 (nvar doubles) are
 * caller-owned DEVICE pointers of the current GPU (or managed memory); host
 * pointers and memory of another GPU return FV_EINVAL.  The default launch
 * configuration is used, with plain tile loads.  Stream-ordered on `stream`
 * (a cudaStream_t, NULL = legacy default); returns without waiting.  Like
 * fv_residual it does not test the state: a non-physical U (rho <= 0, p <= 0,
 * NaN) gives a non-physical R, and nothing reports it (the time-step
 * reduction of a context is what flags such cells).
 * Scratch: a fixed array of 131072 + 32 doubles (1 MiB + 256 B) in the
 * library's device image -- every GPU that loads libfv holds it until the
 * process exits -- holding nvar partial sums per tile.  With rnorm2 != NULL
 * the grid may have at most 131072 / nvar default tiles (2D: 32768 tiles of
 * 64x16 cells, e.g. 5760 x 5760; 3D: 26214 tiles of 8x8x8 cells); larger
 * grids return FV_EINVAL before anything is launched.  The first call on each
 * device looks up the scratch array's device address (cudaGetSymbolAddress)
 * and sets kernel attributes: make that first call before any stream capture.
 * Every call reuses the same scratch (a flags word is cleared by each call,
 * the partials are rewritten), so calls that may overlap on the GPU -- on
 * different streams without ordering, or from several threads -- race and
 * must be serialised by the caller. */
int fv_residual_noalloc(const fv_grid *g, const fv_scheme *s, const double *U, double *R, double *rnorm2,
                        void *stream);

/* Diagnostic of the device arithmetic used by the kernels: for n inputs x
 * (device pointer), out_rsqrt[i] = 1/sqrt(x[i]) and out_rcp[i] = 1/x[i] as
 * computed inside the flux kernels (approximation refined to full double
 * precision).  Stream-ordered on `stream`. */
int fv_debug_math(const double *x, double *out_rsqrt, double *out_rcp, long n, void *stream);

/* Reference FP64 issue rate of the current device (not in the paper; for
 * reporting the ALU roofline): a kernel of 8 x SMs CTAs of 256 threads, each
 * thread running 8 independent chains of 4096 operations -- kind 0: DFMA,
 * kind 1: DADD, kind 2: the flux kernels' products on the integer pipe
 * (bit for bit the FP64 product), kind 3: 4 DFMA chains beside 4 integer-pipe
 * product chains -- timed with CUDA events on `stream` after a short
 * warm-up.  *lane_ops_per_s receives operations (lanes) per second.
 * Allocates and frees 256 doubles per CTA; synchronises `stream`.  FV_EINVAL
 * for a bad kind or a NULL output. */
int fv_debug_fp64_rate(int kind, double *lane_ops_per_s, void *stream);

/* The kernels' integer-pipe replacements of FP64 operations, applied to n
 * device doubles (for tests): out[i] = op(x[i], y[i]) with op 0: x/2 for
 * x >= 0 (half_nonneg), 1: x/4, 2: x/2, 3: 2x (exponent shifts), 4:
 * minmod(x, y), 5: |x|, 6: x * y (the product on 32-bit integer operations
 * the flux kernels use, with the FP64 multiplier for operands or results off
 * its path), 7: the same with signed zeros on the integer path.  Each must
 * equal its FP64 definition bit for bit.  y is read only by ops 4, 6 and 7.  Stream-ordered, no synchronisation.  FV_EINVAL
 * for a bad op or pointer. */
int fv_debug_bits(int op, const double *x, const double *y, double *out, long n, void *stream);

/* Failure-path check of the library's bounded device waits (not in the
 * paper; for tests): one CTA waits on something that never completes --
 * kind 0: an mbarrier no copy arrives on (the wait of every TMA tile load),
 * kind 1: a word nothing changes (the wait of the batched kernel's grid
 * barrier) -- gives up after limit_seconds (0 < limit <= 10), raises its
 * timeout flag and returns.  Synchronises `stream` and returns FV_ETIMEOUT
 * when the wait ran out as designed (the device stays usable), FV_OK if it
 * unexpectedly completed, FV_EINVAL for a bad kind or limit, FV_ECUDA or
 * FV_ENOMEM on a CUDA failure.  Allocates and frees 8 bytes of device
 * memory. */
int fv_debug_wait(int kind, double limit_seconds, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* FV_H */
