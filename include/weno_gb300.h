/*
 * weno_gb300.h -- C ABI of the GB300 (sm_103a) WENO5-JS residual library
 * for the compressible Euler equations.
 *
 * The library computes, on one GPU, the semi-discrete finite-difference
 * residual of Danis et al., "Tensor-Train WENO Scheme for Compressible
 * Flows":
 *   L(U) = -(F^_{i+1/2} - F^_{i-1/2})/dx - (G^...)/dy - (H^...)/dz
 * (Sec. 4.1, Eq. euler-system-for-loop) with the Euler fluxes of Sec. 2.1,
 * global Lax-Friedrichs splitting f(+/-) = (f(u) +/- alpha u)/2 (Sec. 2.2,
 * Eq. lax-friedrichs; alpha = max(|u| + a), Sec. 4.3), fifth-order WENO-JS
 * reconstruction of f(+) and of its mirror image f(-) (Sec. 2.2), three ghost
 * layers per side (Sec. 4.5), and the SSP-RK3 time step of Eq. (tt-ssprk3)
 * without rounding, with dt = lambda h / max(alpha) (Eq. cfl-other).
 *
 * Conventions shared by every call
 *   - Status: every call returns a weno_status (int).  On failure the handle's
 *     weno_last_error() text says why.  Nothing is ever computed on the host:
 *     a combination the GPU path does not implement returns
 *     WENO_ERR_UNSUPPORTED.
 *   - Memory: every array argument is caller-owned.  Unless a parameter says
 *     "host", it is a device pointer of the current CUDA device.  The library
 *     owns only the scratch it allocates in weno_init (stage states, residual
 *     accumulator, reduction partials, control block), freed by weno_destroy.
 *   - State layout: FP64 structure-of-arrays U[f][k][j][i], i (x) fastest,
 *     interior cells only, contiguous; nf = dim + 2 fields in the order
 *     rho, rho u, (rho v), (rho w), rho E.  Ghost cells are not stored; the
 *     kernels synthesise them from the boundary rule.
 *   - Streams: work is enqueued asynchronously on the handle's stream.
 *     Device-side conditions (non-physical state: non-finite values, rho <= 0,
 *     p <= 0) are latched in a device status word and reported by the next
 *     synchronising call (weno_sync, weno_get_time, weno_sums, weno_run,
 *     weno_run_host) as WENO_ERR_NONPHYSICAL.
 *   - Grid: cell-centred, x_i = lo + (i + 1/2) h, h = (hi - lo) / n.
 */
#ifndef WENO_GB300_H
#define WENO_GB300_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct weno_ctx *weno_handle;

typedef enum {
    WENO_OK = 0,
    WENO_ERR_ARG = 1,          /* invalid argument (null pointer, size, enum) */
    WENO_ERR_CUDA = 2,         /* a CUDA runtime call failed */
    WENO_ERR_NONPHYSICAL = 3,  /* device saw NaN/Inf, rho <= 0 or p <= 0 */
    WENO_ERR_TIMEOUT = 4,      /* a bounded device wait gave up */
    WENO_ERR_UNSUPPORTED = 5   /* combination not implemented on the GPU */
} weno_status;

/* Boundary rules (Sec. 4.5).  PERIODIC: ghosts copy the opposite interior
 * end.  TRANSMISSIVE: ghosts copy the nearest interior cell (zero-order
 * extrapolation; not defined in the paper).  REFLECTIVE: symmetry plane,
 * q(-2+l) = q(3-l) for l = 0,1,2 with the normal momentum negated.  INFLOW:
 * all three ghost layers hold a given conserved state (weno_params.bc_state;
 * the full-grid counterpart of the TT inflow rule, which zeroes the ghost rows
 * and adds a rank-1 TT of the inflow state); not available for TT cores. */
typedef enum { WENO_BC_PERIODIC = 0, WENO_BC_TRANSMISSIVE = 1, WENO_BC_REFLECTIVE = 2, WENO_BC_INFLOW = 3 } weno_bc;

/* WENO_FP64: every operation in FP64.  WENO_FP32_BULK: point fluxes, splitting
 * and reconstruction in FP32 on stencil differences formed before rounding to
 * FP32 (2D, and the z direction of 3D: differences of neighbouring points from
 * their FP32 hi/lo splits; 1D and the x and y directions of 3D: values relative
 * to a reference state of each tile); the SSP-RK3 stages run on FP32
 * increments of the FP64 state (U^{n+1} = U^n + Delta_3 in FP64); the state,
 * the maximum behind alpha, dt and the conservation sums stay FP64 (the
 * per-cell wavespeeds are FP32). */
typedef enum { WENO_FP64 = 0, WENO_FP32_BULK = 1 } weno_precision;

/* Lax-Friedrichs constant.  WENO_ALPHA_GLOBAL_NORM: one global alpha = max
 * over cells of |u| + a, used by every direction (Sec. 4.3, Eq. cfl-other).
 * WENO_ALPHA_PER_DIR: direction d splits with alpha_d = max over cells of
 * |u_d| + a (Eq. lax-friedrichs, alpha = max |f'(u)| read per direction).
 * Either way both are recomputed from every stage's state, and dt uses the
 * global max(|u| + a). */
typedef enum { WENO_ALPHA_GLOBAL_NORM = 0, WENO_ALPHA_PER_DIR = 1 } weno_alpha_mode;

/* Conservation law.  WENO_MODEL_EULER: the compressible Euler equations (nf =
 * dim + 2 fields, Sec. 2.1).  WENO_MODEL_ADVECT: one scalar field under
 * u_t + sum_d u_{x_d} = 0 (unit velocity in every direction, Sec. 5.1).
 * WENO_MODEL_BURGERS: one scalar field under u_t + sum_d (u^2/2)_{x_d} = 0
 * (Sec. 5.2).  The scalar laws split with alpha = max |f'(u)| (1, resp.
 * max |u|) in every direction (weno_params.alpha_mode is ignored), run in
 * WENO_FP64 only (WENO_FP32_BULK gives WENO_ERR_UNSUPPORTED), and treat a
 * reflective side as a plain mirror (no component is negated). */
typedef enum { WENO_MODEL_EULER = 0, WENO_MODEL_ADVECT = 1, WENO_MODEL_BURGERS = 2 } weno_model;

typedef struct {
    int32_t dim;     /* 1, 2 or 3 */
    int32_t reserved;
    int64_t n[3];    /* interior cells per direction; n[d] = 1 for d >= dim */
    double lo[3];    /* domain [lo, hi) per direction */
    double hi[3];
} weno_grid;

typedef struct {
    double gamma;        /* ratio of specific heats (1.4 for air) */
    double eps_weno;     /* WENO epsilon in alpha_r = d_r / (beta_r + eps)^2 */
    double cfl;          /* lambda in dt = lambda h / max(alpha); h = min_d h_d */
    int32_t bc[3][2];    /* weno_bc per direction, [low side, high side] */
    int32_t precision;   /* weno_precision */
    int32_t alpha_mode;  /* weno_alpha_mode */
    double bc_state[3][2][5];  /* conserved state (rho, rho u, .., rho E; first nf
                                * entries) of each WENO_BC_INFLOW side */
    int32_t model;       /* weno_model */
    int32_t reserved;
} weno_params;

/* Creates a handle for one grid and parameter set, allocates its scratch
 * (three FP64 state-sized buffers and one residual accumulator) and binds
 * cuda_stream (a cudaStream_t; NULL = the legacy default stream).  grid may be
 * NULL for a handle used only by weno_cross_eval.  Errors: WENO_ERR_ARG for a
 * bad grid/parameter, WENO_ERR_CUDA if allocation fails (nothing is leaked). */
int weno_init(weno_handle *out, const weno_grid *grid, const weno_params *params, void *cuda_stream);

/* Frees the handle and its scratch (synchronises its stream first). */
int weno_destroy(weno_handle h);

/* Rebinds the stream used by later calls.  Synchronises the old stream, then
 * drops every captured CUDA graph of the handle (the step graph of weno_run and
 * the replay graphs of weno_cross_eval); later calls capture them again. */
int weno_set_stream(weno_handle h, void *cuda_stream);

/* alpha_dev[0] = max over interior cells of |u| + sqrt(gamma p / rho) of U
 * (Sec. 4.3), computed in the handle's precision.  alpha_dev: device double.
 * (In WENO_ALPHA_PER_DIR mode the splitting constants are per direction; this
 * call still returns the global maximum, the one dt uses.) */
int weno_alpha(weno_handle h, const double *U, double *alpha_dev);

/* R = L(U) (Sec. 4.1, Eq. euler-system-for-loop), with alpha recomputed from U.
 * U, R: device FP64 [nf][nz][ny][nx]; R must not alias U.  alpha_dev (device
 * double, may be NULL) receives the alpha used. */
int weno_rhs(weno_handle h, const double *U, double *R, double *alpha_dev);

/* Sets / reads the handle's simulation time (a device scalar, so that captured
 * graphs need no host round trip).  weno_get_time synchronises the stream and
 * also returns the number of steps taken since the last weno_set_time; it
 * returns WENO_ERR_NONPHYSICAL if the device latched a non-physical state. */
int weno_set_time(weno_handle h, double t);
int weno_get_time(weno_handle h, double *t, int64_t *steps);

/* Advances U in place by one SSP-RK3 step (Eq. tt-ssprk3 without rounding):
 *   U1 = U + dt L(U); U2 = 3/4 U + 1/4 (U1 + dt L(U1)); U' = 1/3 U + 2/3 (U2 + dt L(U2)),
 * alpha recomputed from every stage's state.  dt > 0: that step size;
 * dt <= 0: dt = cfl h / alpha(U) (Eq. cfl-other).  Either way the step is
 * shortened so that the handle's time does not pass t_end, and it is a no-op
 * once the time has reached t_end.  The time and step count advance on the
 * device.  U: device FP64, overwritten. */
int weno_ssprk3_step(weno_handle h, double *U, double t_end, double dt);

/* Up to max_steps SSP-RK3 steps (as weno_ssprk3_step) until the handle's time
 * reaches t_end.  Steps are launched as CUDA graphs of graph_steps steps
 * (graph_steps <= 0: plain launches); the graph is captured on first use for a
 * given U and reused.  alpha is carried from the last stage of one step to the
 * next.  Synchronises; *steps_out (host, may be NULL) receives the number of
 * steps taken by this call. */
int weno_run(weno_handle h, double *U, double t_end, double dt, int64_t max_steps, int32_t graph_steps,
             int64_t *steps_out);

/* As weno_run, for a state held in HOST memory (pinned memory is fastest):
 * copies U_host to the device, runs, and copies the result back into U_host. */
int weno_run_host(weno_handle h, double *U_host, double t_end, double dt, int64_t max_steps,
                  int32_t graph_steps, int64_t *steps_out);

/* Conservation sums: sums_host[f] = sum over interior cells of U[f], FP64, in a
 * fixed order (bitwise reproducible).  Synchronises.  sums_host: host, nf. */
int weno_sums(weno_handle h, const double *U, double *sums_host);

/* Synchronises the handle's stream; returns the latched device status. */
int weno_sync(weno_handle h);

/* Kernel timing.  While enabled, calls that launch kernels without a CUDA graph
 * (weno_rhs, weno_ssprk3_step, weno_run with graph_steps <= 0) record a CUDA
 * event pair around every kernel on the handle's stream; weno_profile_read
 * (synchronises) adds the elapsed times up per kernel kind:
 *   kind 2: fused x+y kernel of a 3D grid (stores to the accumulator),
 *   kind 3: 1D sweep, kind 4: fused x+y kernel of a 2D grid, kind 5: z sweep
 *           of a 3D grid (3..5 end a residual: stage combination or L(U)),
 *   kind 6: wavespeed max, kind 7: step control and other small kernels,
 *   kind 0: QR factor/apply (weno_tt_round, weno_tt_cross), kind 1: SVD and
 *   contractions of weno_tt_round, maxvol, the TT-cross bookkeeping kernels;
 *   weno_cross_eval's kernels count as kind 7.
 * ms and launches (host arrays of WENO_PROFILE_KINDS) receive the totals since
 * the last enable; *total_launches counts every kernel this handle launched
 * (graphs included) since the last enable. */
enum { WENO_PROFILE_KINDS = 8 };
int weno_profile_enable(weno_handle h, int32_t enable);
int weno_profile_read(weno_handle h, double *ms, int64_t *launches, int64_t *total_launches);

/* Conservation sums for callers that cannot allocate device memory -- for
 * example a host application or framework that owns all device memory through
 * its own pool and forbids other allocations, a latency-critical loop in which
 * cudaMalloc / cudaFree would synchronise the device, or a process that has
 * already committed its device memory and cannot risk an allocation failing
 * mid-run.  The paper has no counterpart; it is a deployment convenience.
 *
 * Same result as weno_sums (the same fixed-order two-level reduction, so the
 * same bits), without a handle and without allocating: the per-block partial
 * sums live in a 40 KiB device array inside the library (1024 blocks x 5
 * fields), which every device that loads the library keeps until the process
 * exits.
 *   U         device FP64 [nf][ncells], caller-owned
 *   nf        1..5 fields; ncells 1..2^40 cells (anything else: WENO_ERR_ARG)
 *   sums_dev  device FP64 [nf], caller-owned, written asynchronously
 *   stream    cudaStream_t to enqueue on (NULL: legacy default stream)
 * The first call on each device looks up the device address of the scratch
 * array (with that device current) and keeps it for the life of the process;
 * make that first call before any stream capture.  The kept address does not
 * survive cudaDeviceReset or a teardown of the device's primary context: do
 * not call this entry point after either.  All calls share the one scratch array and it keeps the last
 * call's contents, so calls that overlap on the GPU (different streams, no
 * ordering between them) race and must not be issued.  Errors are returned as
 * a status; weno_last_error(NULL) then gives the reason. */
int weno_sums_noalloc(const double *U, int32_t nf, int64_t ncells, double *sums_dev, void *cuda_stream);

/* Text of the last error on this handle (never NULL; static storage of the
 * handle, valid until the next call on it).  h may be NULL: then it describes
 * the last failure of this thread in weno_init or weno_sums_noalloc. */
const char *weno_last_error(weno_handle h);

/* ------------------------------------------------------------------------
 * Pointwise evaluation at TT-cross sample points (Sec. 4.2-4.3, Algorithms 1
 * and 2): for each sample of a cross sweep, the 7-point stencil along the flux
 * direction is contracted out of the TT cores (Eq. TT_def), and the
 * Lax-Friedrichs split, WENO5 reconstruction and flux difference give the
 * direction's residual contribution -(F^_{i+1/2} - F^_{i-1/2}) / h.
 * ------------------------------------------------------------------------ */

/* One 3D Euler state in TT format.  core[f][m] is the device FP32 core of mode
 * m of field f, shaped [n_m][r_{m-1}][r_m] (r_0 = r_3 = 1), so that
 * U_f(i,j,k) = sum_{a,b} core[f][0][i][0][a] core[f][1][j][a][b] core[f][2][k][b][0].
 * Ghost rows (Sec. 4.5, core-level periodic / symmetry fill) are not stored:
 * row indices outside [0, n_m) are mapped by bc[m]. */
typedef struct {
    int32_t n[3];
    int32_t r[2];
    int32_t reserved;
    const float *core[5][3];
    double h[3];       /* spacing per mode */
    double alpha;      /* LF constant (the paper estimates it with tt_max_abs) */
    int32_t bc[3][2];  /* weno_bc per mode, [low, high] */
} weno_tt_instance;

/* The samples of one cross sweep of one instance over `mode`: every
 * (left l, index i of mode, right r), left/right being the rank index sets of
 * TT-cross.  left: device int32 [n_left][mode] (multi-indices over modes <
 * mode; n_left = 1 and NULL when mode = 0); right: device int32
 * [n_right][2 - mode] (over modes > mode; n_right = 1 and NULL when mode = 2).
 * out: device [5][n_left][n_mode][n_right], FP32 (FP64 with
 * WENO_CROSS_FP64_CHECK). */
typedef struct {
    int32_t instance;
    int32_t mode;
    int32_t flux_dir;
    int32_t reserved;
    int64_t n_left;
    int64_t n_right;
    const int32_t *left;
    const int32_t *right;
    void *out;
} weno_fiber_set;

/* WENO_CROSS_FP64_CHECK: evaluate in FP64 and write FP64 outputs.
 * WENO_CROSS_GRAPH: run the evaluation as a CUDA graph captured for these
 * exact descriptors (instance and fiber-set fields, pointers included) and
 * replay it on later calls with the same descriptors -- the device arrays they
 * point to (index sets, cores, outputs) may hold new contents.  The handle
 * keeps up to 16 such graphs, each with its own scratch; the first call of a
 * descriptor set synchronises the stream once. */
enum { WENO_CROSS_FP64_CHECK = 1, WENO_CROSS_GRAPH = 2 };

/* Evaluates every fiber set on the handle's stream: one launch contracts the
 * left and right TT vectors of every set, one persistent launch evaluates all
 * samples of all sets.  inst, sets: HOST arrays (copied into the handle's
 * scratch; the device arrays they point to must stay valid until the work
 * completes).  Uses the handle's gamma and eps_weno.  flags:
 * WENO_CROSS_FP64_CHECK evaluates in FP64 and writes FP64 outputs.  Errors:
 * WENO_ERR_ARG for inconsistent sizes or ranks above 32; an index set holding
 * an index outside its mode is found on the device, its set is skipped, and
 * the next synchronising call returns WENO_ERR_ARG. */
int weno_cross_eval(weno_handle h, const weno_tt_instance *inst, int32_t n_inst, const weno_fiber_set *sets,
                    int32_t n_sets, int32_t flags);

/* Autotuner of the evaluation kernel: times every compiled variant of it
 * (threads per CTA x samples per shared-memory chunk) with every persistent
 * grid of 1..4 CTAs per SM on this workload, reps timed runs each after a
 * warm-up (the outputs are written), and keeps the fastest for the workload's
 * class (precision, rank bucket 8/16/32, samples per call to a factor of 4);
 * later weno_cross_eval calls of that class use it.  choice (host int[3], may
 * be NULL): threads per CTA, samples per chunk, CTAs per SM; ms (host, may be
 * NULL): its time per evaluation.  Synchronises.  Errors: those of
 * weno_cross_eval, WENO_ERR_ARG for reps < 1. */
int weno_cross_autotune(weno_handle h, const weno_tt_instance *inst, int32_t n_inst, const weno_fiber_set *sets,
                        int32_t n_sets, int32_t flags, int32_t reps, int32_t *choice, double *ms);

/* Tuning cache file.  weno_tune_save writes the handle's choices (a first line
 * naming the GPU model and SM count, then one line per workload class);
 * weno_tune_load reads a file written on the same GPU model (a file from
 * another model loads nothing) and reports the entries taken in *n_loaded.
 * Errors: WENO_ERR_ARG for a null path or a file that cannot be opened. */
int weno_tune_save(weno_handle h, const char *path);
int weno_tune_load(weno_handle h, const char *path, int32_t *n_loaded);

/* ------------------------------------------------------------------------
 * TT-rounding (Sec. 3, "TT-rounding": Oseledets' two-pass algorithm) of sums
 * of 3D tensor trains, the operation that closes every stage of the TT time
 * step, Eq. (tt-forward-euler) and Eq. (tt-ssprk3):
 *   F = round(U^k + dt L(U^k)),   U' = round(a U^n + b F).
 * ------------------------------------------------------------------------ */

enum { WENO_TT_MAX_TERMS = 4, WENO_TT_MAX_RANK = 96 };

/* One 3D TT in FP64 device memory: core[m] is shaped [n_m][r_{m-1}][r_m] with
 * r_0 = r_3 = 1, X(i,j,k) = sum_{a,b} core[0][i][0][a] core[1][j][a][b] core[2][k][b][0]. */
typedef struct {
    int32_t n[3];
    int32_t r[2];
    double *core[3];
} weno_tt3;

/* out = round(sum_t coef[t] term[t], eps_tt) with ||sum - out||_F <= eps_tt ||sum||_F.
 * Terms share n; their cores are read only.  out.core[m] are caller device
 * buffers of cap[m] doubles; the call writes out.n, out.r (the ranks it chose)
 * and norm (= ||sum||_F).  Sufficient capacities: with k3 = min(n3, R2),
 * k2 = min(n2 k3, R1), kc = min(n1, k2), ke = min(kc n2, k3) (R1, R2 the summed
 * ranks): cap = {n1 kc, n2 kc ke, n3 ke}. */
typedef struct {
    int32_t n_terms;
    int32_t reserved;
    double coef[WENO_TT_MAX_TERMS];
    weno_tt3 term[WENO_TT_MAX_TERMS];
    weno_tt3 out;
    int64_t cap[3];
    double norm;
} weno_tt_round_problem;

/* Rounds every problem of the batch (probs: HOST array; the ranks and norms
 * are written back into it).  Right-to-left orthogonalisation by Householder
 * QR of the core unfoldings, then left-to-right truncated SVDs (one-sided
 * Jacobi of the triangular factors) with threshold eps_tt / sqrt(2) ||sum||_F,
 * all in FP64 on the handle's stream.  The call synchronises the stream twice
 * (to read the ranks it chose); the output cores are complete when the stream
 * next synchronises.  Kernel timing kinds: 0 (QR factor/apply), 1 (SVD and
 * contractions).  Errors: WENO_ERR_ARG for 0 or more than 4 terms, unequal
 * mode sizes, null cores, ranks < 1, eps_tt < 0, or too small a capacity
 * (nothing is written); WENO_ERR_UNSUPPORTED when the summed ranks R1 or R2
 * exceed WENO_TT_MAX_RANK. */
int weno_tt_round(weno_handle h, weno_tt_round_problem *probs, int32_t n_probs, double eps_tt);

/* ------------------------------------------------------------------------
 * Cross-index selection (Sec. 3, "TT-cross Interpolation": the rows and
 * columns of the skeleton decompositions are chosen by the maximum-volume
 * principle, Goreinov et al. 2010).
 * ------------------------------------------------------------------------ */

typedef struct {
    int32_t n, r;       /* n >= r, 1 <= r <= 64 */
    const double *A;    /* device, n x r row-major */
    double *B;          /* device, n x r: receives A A[I]^{-1} (identity on the rows I) */
    int32_t *idx;       /* device, r: receives the selected rows I */
} weno_maxvol_problem;

/* Batched maxvol (Sec. 3, "TT-cross Interpolation"), FP64, one thread-block
 * cluster per matrix: the r pivot rows I of Gaussian elimination with partial
 * pivoting (ties to the smaller row), B = A A[I]^{-1} formed from the
 * elimination's multipliers L as L L[I]^{-1} (rows I exactly the unit
 * vectors), then row swaps while some |B[i][j]| > 1 + delta (each swap
 * multiplies |det A[I]| by |B[i][j]|; ties go to the first entry in row-major
 * order) or max_iters swaps are done.  probs: HOST array, at most 65535
 * matrices; synchronises the stream; swaps (host, may be NULL) receives the
 * swaps per matrix.  Errors: WENO_ERR_ARG for bad sizes, null pointers, or a
 * matrix whose elimination meets a zero pivot column (rank < r). */
int weno_maxvol(weno_handle h, const weno_maxvol_problem *probs, int32_t n_probs, double delta, int32_t max_iters,
                int32_t *swaps);

/* One fixed-rank TT-cross of A(i, j, k, f) = the flux_dir residual contribution
 * -(F^_{i+1/2} - F^_{i-1/2}) / h of Euler component f at cell (i, j, k) of one
 * weno_tt_instance (the values weno_cross_eval computes).  The components sit
 * in the last core, as in the LF-cross layout of Sec. 4.2. */
typedef struct {
    int32_t r[2];       /* cross ranks: 1 <= r1 <= min(n1, n2 r2, 64), 1 <= r2 <= min(r1 n2, 5 n3, 64) */
    int32_t *J1;        /* device [r1][3] (j, k, f): initial right index set in, final one out */
    int32_t *J2;        /* device [r2][2] (k, f): in/out */
    int32_t *I1;        /* device [r1]: left index set out */
    int32_t *I2;        /* device [r2][2] (i, j): out */
    double *core[3];    /* device out: [n1][1][r1], [n2][r1][r2], [n3][r2][5] */
} weno_tt_cross_problem;

/* Alternating TT-cross with maxvol index selection (Sec. 3, "TT-cross
 * Interpolation"; AMEn's rank adaptation is not part of it).  For every
 * instance i (problem i): a left-to-right pass evaluates A(:, J1), A(I1, :, J2),
 * A(I2, :, :) as fiber sets and takes maxvol's rows of each unfolding C to
 * form I1, I2 and the interpolation cores C C[I]^{-1} (no orthogonalisation
 * first: maxvol's pivots and C C[I]^{-1} depend only on C's column space, so
 * they equal those of C's Householder Q);
 * `sweeps` times a right-to-left pass updates J2 and J1 the same way before the
 * next left-to-right pass.  The resulting TT interpolates A on the final index
 * sets.  Fibers are evaluated in FP32 (FP64 with WENO_CROSS_FP64_CHECK in
 * flags); the selection and the cores are FP64.  inst, probs: HOST arrays;
 * synchronises once at the end.  Uses the handle's gamma and eps_weno.
 * Errors: WENO_ERR_ARG for bad ranks, null pointers or a fiber matrix of rank
 * below the cross rank; those of weno_cross_eval. */
int weno_tt_cross(weno_handle h, const weno_tt_instance *inst, int32_t n_inst, int32_t flux_dir,
                  weno_tt_cross_problem *probs, int32_t sweeps, double delta, int32_t flags);

#ifdef __cplusplus
}
#endif

#endif /* WENO_GB300_H */
