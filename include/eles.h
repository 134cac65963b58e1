/*
 * eles.h -- C ABI of the GB300 (sm_103a) explicit-filter library.
 *
 * The library computes, for channel-flow velocity snapshots, the explicitly
 * filtered velocity and the exact subfilter stress of Bae & Lozano-Duran,
 * "DNS-aided explicitly filtered LES of channel flow" (arXiv 1902.02508):
 *
 *   bar(phi)(x) = integral G(x - x') phi(x') dx'                     (Eq. 2)
 *   T_ij = bar(u_i u_j) - ~bar(u_i) ~bar(u_j)                         (Eq. 6)
 *
 * following the four steps of Sec. 2.1 (form u_i u_j, filter it, form the
 * product of the filtered velocities, subtract), with the wall-normal line
 * extended across both walls by Eq. 7 (u1, u3 even, u2 odd) so that the
 * filter keeps a constant width up to the wall, and with the filtered field
 * sampled on the LES grid by linear interpolation (the discretization
 * operator of Sec. 3).  The kernel is a Gaussian of width Delta per direction
 * (transfer function exp(-k^2 Delta^2 / 24)), cut at |s| <= 2.5 Delta, with
 * trapezoid weights on the extended node set and every row normalised.
 *
 * Conventions shared by every call:
 *  - Fields are device pointers, row-major [component][y][z][x], x fastest.
 *    Velocity input u: [3][ny][nz][nx]; filtered velocity ubar:
 *    [3][nly][nlz][nlx]; stress tau: [6][nly][nlz][nlx] in the order
 *    11, 12, 13, 22, 23, 33.  Element type: double for EF_PREC_FP64, float
 *    for every other precision.  Velocities in units of u_tau.
 *  - The caller owns every field buffer.  The library owns plans: their
 *    filter weights and their scratch memory live on the device of the plan
 *    and are allocated by ef_filter_setup only; hot calls allocate nothing
 *    and never synchronise the host.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *    stream).  Calls are asynchronous on it.  Calls that share a plan must
 *    not overlap in time (they share its scratch): issue them on one stream.
 *  - Host threads: plans are independent, but the first launch of each
 *    kernel configuration raises that kernel's shared-memory limit through
 *    an unlocked process-wide cache.  Make the first hot call of plans that
 *    need different limits from one thread (later calls may come from any
 *    thread).
 *  - Every call returns an ef_status.  On failure ef_last_error() returns a
 *    thread-local message.  Device-side problems (non-finite input, a wait
 *    that ran out) are recorded in the plan's error word and read back by
 *    ef_check_device_error().
 */
#ifndef ELES_H
#define ELES_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Status codes. */
typedef enum {
    EF_OK = 0,
    EF_ERR_ARG = 1,          /* invalid argument (NULL, non-positive size, Delta <= 0 ...) */
    EF_ERR_SHAPE = 2,        /* grid shapes the library does not accept */
    EF_ERR_CUDA = 3,         /* a CUDA runtime call failed */
    EF_ERR_NAN = 4,          /* non-finite values seen on the device */
    EF_ERR_TIMEOUT = 5,      /* a bounded device wait ran out */
    EF_ERR_OOM = 6,          /* device allocation failed in a setup call */
    EF_ERR_UNSUPPORTED = 7,  /* valid request the library does not implement */
    EF_ERR_RANGE = 8         /* a global index failed its range check (range-checked build only) */
} ef_status;

/* Filter kernels.  The Gaussian, with the y integral of Eq. 2 on the
 * stretched, wall-extended line evaluated either by the trapezoid rule on
 * the extended nodes (EF_KERNEL_GAUSSIAN) or exactly against the
 * piecewise-linear interpolant of the extended field (EF_KERNEL_GAUSSIAN_HAT:
 * the quadrature alternative Sec. 3 names for the commutation error; it
 * reproduces linear profiles exactly away from the walls).  x and z use the
 * trapezoid rule in both.
 * EF_KERNEL_DIFFERENTIAL is the filter of the paper's simulations (Sec. 3):
 * the Green's function of (1 - a^2 lap), i.e. ubar solves
 * (1 - a^2 lap) ubar = u on the extended domain, with the second-order
 * finite-difference Laplacian on the DNS nodes (three-point periodic in x
 * and z, three-point non-uniform in y with mirror ghosts of each field's
 * parity at both walls) and a^2 = Delta_f^2 / 40 (`delta` is Delta_f).
 * EF_PREC_FP64 filters u and u u directly.  EF_PREC_FP32 transforms the
 * fluctuations about the FP64 plane-mean profile (u', u'u' and U u') in FP32
 * and solves the profile terms and forms ubar and T in FP64.  It needs one
 * of these precisions, an extension (Eq. 7 or Eq. 9), nx and nz of the form
 * 2^p 3^q (at most 1024), and LES nodes that are DNS nodes (nx, nz
 * multiples of nlx, nlz; LES y nodes among the DNS y nodes); otherwise
 * ef_filter_setup returns EF_ERR_SHAPE / EF_ERR_ARG / EF_ERR_UNSUPPORTED.
 * The fields of a snapshot are transformed and solved in groups (3 in FP64,
 * 6 in FP32), so the plan holds the spectra of one group (16 or 8 bytes per
 * mode, ny nz (nx/2 + 1) modes per field: about 1.2 GB at 512x257x384)
 * and the Thomas factors of both parities (2 ny nz (nx/2 + 1) pairs). */
enum { EF_KERNEL_GAUSSIAN = 0, EF_KERNEL_GAUSSIAN_HAT = 1, EF_KERNEL_DIFFERENTIAL = 2 };

/* Wall treatment. */
enum {
    EF_EXT_EVEN_ODD = 0,     /* Eq. 7: u1, u3 even, u2 odd about each wall */
    EF_EXT_ODD_EVEN = 1,     /* Eq. 9: u1, u3 odd, u2 even (divergence-preserving, not NS-compatible) */
    EF_EXT_NONE = 2          /* no extension: support cut at the walls (does not commute, Sec. 2.2) */
};

/* Arithmetic of the filter contractions.
 * The split-precision forms (float in/out) contract the fluctuations about a
 * reference profile U(y) (the mean of each plane's z-row 0; exact algebra of
 * Eq. 6) on the tensor cores with FP32 accumulation, and form ~bar(u) and T
 * from FP64 profile terms:
 *   EF_PREC_BF16X3  the velocity fluctuations u'_a and the weights split
 *                   into two BF16 parts, three products (A_hi B_hi + A_lo
 *                   B_hi + A_hi B_lo), in x and in z;
 *   EF_PREC_TF32X2  x: the velocity fluctuations and the weights split into
 *                   two TF32 parts (three products); z as BF16X3;
 *   both: the six product fields u'_a u'_b are rounded once to an 11-bit
 *   significand (FP16, TF32's precision) before x and again before z, each
 *   time against weights split into two FP16 parts (two products); the y
 *   contraction is split BF16 (three products) for every field.  Measured
 *   on the 512 x 257 x 384 channel at Delta = Lx/64: max |T - FP64| per
 *   component 1.4e-5 u_tau^2 or less.
 * A plan of either form runs the x-z contraction on the tensor cores or is
 * refused with EF_ERR_UNSUPPORTED: the warp-specialised kernel needs LES x
 * and z nodes at
 * every r-th DNS node (x stride 4, 8 or 16), nz in {64, 128, 192, 256, 384},
 * nlz a multiple of 16, nlx a multiple of 16 / (x stride), and a filter that
 * fits its window (2.5 Delta at most about 13 x strides; wider x filters are
 * split into 2 or 4 output phases, each a CTA that re-reads the plane);
 * BF16X3 plans outside it may still run the earlier tensor-core kernel
 * (x stride 8 with at most 7 outputs per input; it splits every field in x
 * and z into BF16 parts).  ef_plan_info index 10 tells which kernel runs. */
enum {
    EF_PREC_FP64 = 0,        /* double in, double out, FP64 throughout */
    EF_PREC_FP32 = 1,        /* float in/out, FP32 contractions on CUDA cores, FP64 recovery */
    EF_PREC_TF32X2 = 2,      /* float in/out, split TF32 x-contraction on tensor cores (above) */
    EF_PREC_BF16X3 = 3       /* float in/out, split BF16 x-contraction on tensor cores (above) */
};

/*
 * A channel grid: nx x ny x nz nodes, periodic in x (length Lx) and z (Lz),
 * wall-normal nodes y[0..ny-1] on the host, strictly ascending with
 * y[0] = -1 and y[ny-1] = +1 (both walls are nodes).  x_i = i Lx / nx,
 * z_k = k Lz / nz.
 */
typedef struct {
    int nx, ny, nz;
    double Lx, Lz;
    const double *y;
} ef_grid;

typedef struct ef_plan ef_plan;

/*
 * ef_filter_setup -- build a filter plan on the current CUDA device.
 * Cite: Eq. 2 (filter), Eq. 7 / Eq. 9 (extension), Sec. 3 (linear
 * interpolation to the LES grid), constant filter width Delta (Sec. 2.2).
 *  dns, les   grids (host structs; y arrays are copied).  les must span the
 *             same box: les->Lx == dns->Lx, les->Lz == dns->Lz, les->y within
 *             [-1, 1] ascending with les->y[0] = -1 and les->y[nly-1] = +1.
 *  delta      filter width, > 0; for the Gaussian kernels 2.5 delta must be
 *             < Lx/2, Lz/2 and < 2.
 *  kernel     EF_KERNEL_GAUSSIAN, EF_KERNEL_GAUSSIAN_HAT or
 *             EF_KERNEL_DIFFERENTIAL.
 *  extension  EF_EXT_*.
 *  precision  EF_PREC_*.
 *  out        receives the plan (owned by the caller, free with
 *             ef_plan_destroy).
 * The operator weights are computed on the device in FP64 (one thread per
 * operator row) and kept there; the plan also allocates the scratch memory
 * its hot calls use.  Synchronises the device.  Errors: EF_ERR_ARG,
 * EF_ERR_SHAPE, EF_ERR_OOM, EF_ERR_CUDA, EF_ERR_UNSUPPORTED.
 */
int ef_filter_setup(const ef_grid *dns, const ef_grid *les, double delta, int kernel,
                    int extension, int precision, ef_plan **out);

/* Release a plan and its device memory (NULL is ignored). */
void ef_plan_destroy(ef_plan *plan);

/*
 * ef_filter_fields -- ~bar(u_i) only (steps 2-3 of Sec. 2.1 for the
 * velocities; the initial condition of Sec. 3 is exactly this call).
 *  u     device [3][ny][nz][nx]
 *  ubar  device [3][nly][nlz][nlx]
 * Errors: EF_ERR_ARG (NULL plan or pointer), EF_ERR_CUDA (launch failure).
 */
int ef_filter_fields(ef_plan *plan, const void *u, void *ubar, void *stream);

/*
 * ef_subfilter_stress -- ~bar(u_i) and T_ij on the LES grid (Eq. 6, the
 * four steps of Sec. 2.1).
 *  u           device [3][ny][nz][nx]
 *  ubar        device [3][nly][nlz][nlx]
 *  tau         device [6][nly][nlz][nlx], order 11, 12, 13, 22, 23, 33
 *  plane_mean  device double [3][ny]: the x-z plane means <u_i>(y_j)
 *              (Sec. 4.1's averaging in the homogeneous directions), or NULL.
 * Internally the products are formed about a reference profile U(y) (the
 * mean of one z-row per plane); the decomposition is exact algebra because
 * the x and z operators preserve functions of y, and the cancelling
 * subtractions run in FP64.
 * Errors: EF_ERR_ARG, EF_ERR_CUDA.
 */
int ef_subfilter_stress(ef_plan *plan, const void *u, void *ubar, void *tau,
                        double *plane_mean, void *stream);

/*
 * ef_subfilter_stress_batch -- the same for nsnap snapshots that share the
 * plan's grids and filter, stored back to back: u [nsnap][3][ny][nz][nx],
 * ubar [nsnap][3][..], tau [nsnap][6][..], plane_mean [nsnap][3][ny] or NULL.
 * Snapshots are independent; up to the plan's reserved count (see
 * ef_plan_reserve) run in one launch per phase, larger batches in groups.
 * Errors: EF_ERR_ARG, EF_ERR_CUDA.
 */
int ef_subfilter_stress_batch(ef_plan *plan, int nsnap, const void *u, void *ubar, void *tau,
                              double *plane_mean, void *stream);

/*
 * ef_plan_reserve -- size the plan's scratch for batches of up to
 * max_snapshots snapshots per launch (setup-time call: it allocates, and
 * synchronises the device; never call it while the plan is in use).  A new
 * plan reserves 1.  Errors: EF_ERR_ARG, EF_ERR_OOM.
 */
int ef_plan_reserve(ef_plan *plan, int max_snapshots);

/*
 * ef_check_device_error -- read (and clear) the plan's device error word.
 * Synchronises `stream`.  Returns EF_OK, or the ef_status a kernel recorded.
 */
int ef_check_device_error(ef_plan *plan, void *stream);

/*
 * ef_selftest_wait -- failure-detection self-test.  A one-thread kernel waits
 * on an mbarrier with the bounded wait every kernel of the library uses
 * (their limit is about 2 s of SM clocks).  complete = 0: nothing arrives,
 * the wait gives up after limit_cycles SM clocks and records EF_ERR_TIMEOUT
 * in the plan's error word (read it with ef_check_device_error); the
 * context stays usable.  complete = 1: the barrier phase completes first and
 * nothing is recorded.  Errors: EF_ERR_ARG (NULL plan, limit outside
 * 1 .. 4e9), EF_ERR_CUDA.
 */
int ef_selftest_wait(ef_plan *plan, long long limit_cycles, int complete, void *stream);

/*
 * ef_plan_set_wait_limit -- bound, in SM clocks, of every wait inside the
 * warp-specialised x-z kernel (its TMA stages and the hand-over between its
 * roles); 0 restores the default (about 2 s at the SM clock).  A wait that
 * runs out records EF_ERR_TIMEOUT in the plan's error word (read by
 * ef_check_device_error) and the kernel's roles stop at once, after the
 * bulk copies already issued have landed; the outputs of that call are then
 * undefined, and the plan and the context stay usable.  For tests of the
 * timeout path (a limit of 1 makes the first wait that is not already
 * complete run out).  Batch graphs holding the plan re-capture.
 * Errors: EF_ERR_ARG.
 */
int ef_plan_set_wait_limit(ef_plan *plan, long long cycles);

/* Plan facts for callers and tests.  ints: 0 nx, 1 ny, 2 nz, 3 nlx, 4 nly,
 * 5 nlz, 6 precision, 7 x-taps per row, 8 z-taps per row, 9 max y-taps per
 * row, 10 x-contraction variant (0 generic, 1 banded ring on CUDA cores,
 * 2 tensor cores, 3 tensor cores with warp-specialised producer, x and z
 * roles), 11 x and z fused in one kernel (0/1), 12 reserved snapshots,
 * 13 y-contraction variant (0 CUDA cores, 1 tensor cores; split-precision
 * plans), 14 differential-filter plan (0/1), 15 output phases of the
 * warp-specialised x-z kernel (CTAs per y-plane; 0 when it does not run).
 * Returns EF_ERR_ARG for an unknown index. */
int ef_plan_info(const ef_plan *plan, int what, long *value);

/*
 * ef_plan_weights -- copy one operator of the plan to the host as a dense
 * row-major FP64 matrix (for tests).  which: 0 A_x [nlx][nx], 1 A_z
 * [nlz][nz], 2 A_y even [nly][ny], 3 A_y odd [nly][ny].  dst must hold the
 * whole matrix.  Synchronises the device.
 */
int ef_plan_weights(const ef_plan *plan, int which, double *dst);

/*
 * Phase timing for benchmarks.  ef_profile_enable(plan, 1) clears the
 * accumulators and makes every later hot call record CUDA events on its own
 * stream before and after each phase; ef_profile_enable(plan, 0) stops it.
 * ef_profile_read waits for the recorded events and returns the summed
 * milliseconds per phase (ms[0] reference profile with the x- and
 * z-contractions, ms[1] reserved (0), ms[2] y-contraction and recovery,
 * ms[3] reserved (0)) and the number of calls timed.  A batch larger than
 * the reserved count is timed over its last group only.
 * Errors: EF_ERR_ARG, EF_ERR_CUDA.
 */
int ef_profile_enable(ef_plan *plan, int on);
int ef_profile_read(ef_plan *plan, double *ms, long *calls);

/* ------------------------------------------------------------------------
 * Error measures of Sec. 4 (Eq. 13-15), as device reductions.  Velocities are
 * divided by each run's friction velocity u_tau before comparison.
 * Quadrature (the paper states none): x and z periodic and uniform (node
 * sums), trapezoid rule on the y nodes; the wall-to-centre integral of
 * Eq. 14 and 15 is that of the piecewise-linear interpolant over y in
 * [-1, 0].  All sums are FP64 and in a fixed order (repeat calls agree bit
 * for bit).
 *
 * ef_stats_create -- set-up call for fields on `grid` (x, z uniform, y the
 * given ascending nodes) in the dtype of `precision` (FP64 for
 * EF_PREC_FP64, FP32 otherwise): uploads the weights and allocates the
 * partial-sum scratch.  Errors: EF_ERR_ARG, EF_ERR_CUDA.
 *
 * ef_plane_stats -- u [3][ny][nz][nx] (device): the plane means <u_c>(y_j)
 * and intensities u_c,rms(y_j) = sqrt(<(u_c - <u_c>)^2>) over x and z, into
 * mean, rms (device double [3][ny]).
 *
 * ef_error_field -- Eq. 13 for velocity component `component` (0, 1, 2; the
 * paper uses u_1) of two fields a, b [3][ny][nz][nx] (device) on the grid:
 * writes ||a/utau_a - b/utau_b||_V / ||b/utau_b||_V to *err (device double).
 *
 * ef_error_profile -- Eq. 14 (mean profiles) or Eq. 15 (rms profiles):
 * pa, pb device double [ny] on the grid's y nodes; writes the wall-to-centre
 * relative L2 error to *err (device double).
 *
 * All three are asynchronous on `stream`; calls on one ef_stats share its
 * scratch, so run them on one stream.  Errors: EF_ERR_ARG, EF_ERR_CUDA.
 * ---------------------------------------------------------------------- */
typedef struct ef_stats ef_stats;
int ef_stats_create(const ef_grid *grid, int precision, ef_stats **out);
void ef_stats_destroy(ef_stats *st);
int ef_plane_stats(ef_stats *st, const void *u, double *mean, double *rms, void *stream);
int ef_error_field(ef_stats *st, const void *a, const void *b, int component, double utau_a, double utau_b,
                   double *err, void *stream);
int ef_error_profile(ef_stats *st, const double *pa, const double *pb, double utau_a, double utau_b, double *err,
                     void *stream);

/*
 * ef_differential_unfilter -- the inverse of the differential filter
 * (EF_KERNEL_DIFFERENTIAL) on one grid: out = (1 - a^2 lap) in, a^2 =
 * delta^2 / 40, with the same second-order stencils (three-point periodic in
 * x and z, three-point non-uniform in y with mirror ghosts of each
 * component's parity at the walls).  Sec. 4 compares LES and DNS velocities
 * after reversing the filter on the LES field; with grid = the LES grid this
 * is that reversal, with grid = the DNS grid it undoes ef_filter_fields of a
 * differential plan whose LES grid is the DNS grid.
 *  grid       host struct (y copied, stream-ordered temporary)
 *  extension  EF_EXT_EVEN_ODD or EF_EXT_ODD_EVEN (component parities)
 *  in, out    device double [3][ny][nz][nx]; distinct buffers.  An odd
 *             component's wall rows are copied (its filtered values there
 *             are zero).
 * Errors: EF_ERR_ARG (NULL, in == out, no extension, delta <= 0),
 * EF_ERR_SHAPE (grid), EF_ERR_CUDA.
 */
int ef_differential_unfilter(const ef_grid *grid, double delta, int extension, const double *in, double *out,
                             void *stream);

/* ------------------------------------------------------------------------
 * Host buffers.  The same computation as ef_subfilter_stress_batch (Eq. 6
 * evaluated by the steps of Sec. 2.1 on the Eq. 7 extension) with the
 * snapshots and results in host memory: the copy of one group of `chunk`
 * snapshots in and of another group's results out overlap the compute of a
 * third (two device slots, a copy-in and a copy-out stream).
 *
 * ef_io_create -- set-up call: reserves the plan for `chunk` snapshots and
 * allocates two device slots of `chunk` snapshots (inputs and outputs) plus
 * two streams and events.  The pipeline uses the plan's scratch: one
 * pipeline per plan, and no other call on the plan while a host call runs.
 * Errors: EF_ERR_ARG, EF_ERR_OOM/EF_ERR_CUDA.
 *
 * ef_subfilter_stress_host -- u_host [nsnap][3][ny][nz][nx], ubar_host
 * [nsnap][3][..], tau_host [nsnap][6][..], plane_mean_host [nsnap][3][ny]
 * (double) or NULL, all in host memory, the plan's precision.  The copies
 * overlap only when the host buffers are page-locked (cudaHostAlloc, or
 * torch pin_memory); pageable buffers give the same results, serialised.
 * Asynchronous on `stream`: the results are in the host buffers once
 * `stream` is synchronised (the call ends with `stream` waiting on the last
 * copy out).  Errors: EF_ERR_ARG, EF_ERR_CUDA.
 * ---------------------------------------------------------------------- */
typedef struct ef_io ef_io;
int ef_io_create(ef_plan *plan, int chunk, ef_io **out);
void ef_io_destroy(ef_io *io);
int ef_subfilter_stress_host(ef_io *io, int nsnap, const void *u_host, void *ubar_host, void *tau_host,
                             double *plane_mean_host, void *stream);

/* ------------------------------------------------------------------------
 * Batches over several plans (different DNS grids, LES grids and filter
 * widths): item i runs nsnap[i] snapshots of plans[i].  ef_batch_run replays
 * every item's kernels as one CUDA graph on `stream` (captured on the first
 * run and again whenever a field pointer changes).  A plan may appear in one
 * batch only once (plans own their scratch); ef_batch_create reserves each
 * plan's scratch for its item (allocates).  Fields as in
 * ef_subfilter_stress_batch, one pointer per item.
 * ---------------------------------------------------------------------- */
typedef struct ef_batch ef_batch;
int ef_batch_create(ef_plan *const *plans, const int *nsnap, int n, ef_batch **out);
int ef_batch_run(ef_batch *batch, const void *const *u, void *const *ubar, void *const *tau, void *stream);
void ef_batch_destroy(ef_batch *batch);
/* Number of times the batch has captured its graph (a run re-captures when a
 * field pointer changed or a plan's scratch or kernel choice changed since the
 * last capture: ef_plan_reserve growing it, ef_io_create, a larger
 * ef_batch_create, ef_plan_set_variant, ef_plan_autotune). */
long ef_batch_captures(const ef_batch *batch);

/*
 * ef_plan_autotune -- time the x-z kernel variants the plan supports (the
 * unfused kernels; the fused kernel on CUDA cores or, for EF_PREC_BF16X3, on
 * the tensor cores; 2, 4 or 8 columns per z phase; for the split precisions
 * the warp-specialised tensor-core kernel) on one sample snapshot u (device,
 * plan precision; ubar, tau are scratch outputs of one snapshot), keep the
 * fastest, and report it as *choice = variant * 16 + columns (variant 0
 * unfused, 1 fused CUDA cores, 2 fused tensor cores, 3 fused tensor cores
 * warp-specialised, which ignores the column count) and its time.
 * Synchronises the device.
 * ef_plan_set_variant applies a stored choice (EF_ERR_UNSUPPORTED if the
 * plan cannot run that variant).  For split-precision plans the flag
 * EF_VARIANT_CUDA_CORE_Y may be or-ed into the choice: the y contraction then
 * runs on the CUDA cores (the pass such a plan takes when the banded
 * tensor-core tiling does not fit its geometry) after the tensor-core x-z
 * kernel; without the flag the tensor-core y pass is used where it fits.
 * Either call invalidates batch graphs that hold the plan (they re-capture
 * on their next run).
 */
#define EF_VARIANT_CUDA_CORE_Y 256
int ef_plan_autotune(ef_plan *plan, const void *u, void *ubar, void *tau, int reps, int *choice, float *best_ms);
int ef_plan_set_variant(ef_plan *plan, int choice);

/* ------------------------------------------------------------------------
 * Learned closure.  The paper proposes using the exact stress computed from
 * DNS to inform subgrid models, e.g. by machine learning (Sec. 2.1 and the
 * summary, Sec. 5).  The library provides one such model: an MLP
 * 10 -> 128 -> 128 -> 128 -> 6 with SiLU activations mapping the nine
 * filtered velocity gradients d~bar(u_i)/dx_j and the wall distance
 * y+ = (1 - |y|) Re_tau to T_11, T_12, T_13, T_22, T_23, T_33, trained with
 * Adam (mean-squared error on standardised inputs and targets) on the exact
 * T_ij of ef_subfilter_stress.  FP32 master weights, BF16 working weights,
 * FP32 accumulation; fixed-order reductions (reproducible bit for bit).
 * ---------------------------------------------------------------------- */
typedef struct {
    int hidden;               /* must be 128 */
    int batch;                /* training mini-batch size */
    float lr;                 /* Adam learning rate */
    float guard_sigma;        /* inference guard: a standardised input beyond this uses the exact stress */
    unsigned long long seed;  /* initialisation and batch order */
} ef_closure_cfg;

typedef struct ef_closure ef_closure;

/* Create a closure on the current device (allocates; synchronises). */
int ef_closure_create(const ef_closure_cfg *cfg, ef_closure **out);
void ef_closure_destroy(ef_closure *closure);

/*
 * ef_closure_features -- the ten inputs at every LES node.
 *  les     LES grid (host; y nodes as in ef_filter_setup)
 *  ubar    device float [3][nly][nlz][nlx] (e.g. from ef_subfilter_stress)
 *  re_tau  friction Reynolds number for y+
 *  extension  EF_EXT_* (wall parities of the mirror ghosts in y)
 *  feats   device float [N][10], N = nly nlz nlx, point order (J, Z, X):
 *          d~bar(u_i)/dx_j at 3i + j (j = x, y, z), then y+.
 * Second-order central differences; periodic in x and z; three-point
 * non-uniform stencil in y with mirror ghosts at the walls (Eq. 8).
 * Allocates a small temporary for the y nodes (stream-ordered).
 */
int ef_closure_features(const ef_grid *les, const float *ubar, double re_tau, int extension, float *feats,
                        void *stream);

/*
 * ef_closure_features_static -- the same features as ef_closure_features
 * without allocating anything (no cudaMalloc, cudaMallocAsync or cudaFree),
 * for callers that are not allowed to allocate device memory.  The paper has
 * no counterpart; this is a deployment variant.  The LES y nodes go to a
 * fixed device array of 4096 doubles (32 KB) that every device loading the
 * library holds until exit; les->ny above 4096 is rejected with EF_ERR_ARG.
 * The first call on a device looks up that array's address (make it before
 * any stream capture).  Every call copies les->y from the caller's host
 * memory into the array with cudaMemcpyAsync on `stream`, so the host array
 * must stay valid until that copy has run.  All calls share the array: calls
 * that overlap on the GPU race, so issue them on one stream.  Other
 * arguments and errors as ef_closure_features.
 */
int ef_closure_features_static(const ef_grid *les, const float *ubar, double re_tau, int extension, float *feats,
                               void *stream);

/* Standardisation statistics from training data: feats device [N][10],
 * tau device [6][N] (component-major, the layout of ef_subfilter_stress). */
int ef_closure_fit_norm(ef_closure *closure, const float *feats, const float *tau, long n, void *stream);

/* Train for `epochs` passes over n points (fits the statistics first if not
 * yet done): mini-batches of cfg.batch points in a seeded order per epoch,
 * MSE on the standardised outputs, Adam (Sec. 5's learned closure; the
 * paper leaves the model open).  The call allocates its scratch (the epoch's
 * permutation, Adam's per-step factors) and captures one full-batch step as
 * a CUDA graph on a private stream, replayed for every full batch; all of it
 * is released before it returns.  Results do not depend on the capture
 * (bit-identical to launching each step).  Synchronises the stream;
 * *loss_out = mean loss of the last epoch (standardised units).  Errors:
 * EF_ERR_ARG, EF_ERR_OOM, EF_ERR_CUDA. */
int ef_closure_train(ef_closure *closure, const float *feats, const float *tau, long n, int epochs,
                     void *stream, float *loss_out);

/*
 * ef_closure_infer -- tau_out device [6][N] from feats device [N][10].  Where
 * a standardised input exceeds the guard the model is outside its training
 * range: if exact_tau (device [6][N]) is given that exact stress is used
 * there, and *n_fallback (if not NULL) receives the count (synchronises).
 * One tensor-core kernel over all N points (tcgen05, accumulators in TMEM):
 * BF16 working weights, activations split into two BF16 parts, FP32
 * accumulation; standardisation, guard, SiLU and the fallback are fused.
 * A wait inside the kernel that ran out is recorded in the closure's error
 * word: returned here when n_fallback is requested, else read by
 * ef_closure_check_device_error.  Calls on one closure share its packed
 * weight image and counters: issue them on one stream (they must not
 * overlap on the GPU).  n may be any count >= 1 (persistent grid).
 */
int ef_closure_infer(ef_closure *closure, const float *feats, float *tau_out, long n, const float *exact_tau,
                     long *n_fallback, void *stream);

/*
 * ef_closure_infer_exact -- inference with the exact filter as the fallback.
 * As ef_closure_infer, but where a standardised input exceeds the guard the
 * output is the exact subfilter stress of Eq. 6 at that point, evaluated from
 * the DNS snapshot through the plan's operators (Eq. 2 with the wall
 * extension of Eq. 7 or Eq. 9 folded in, linear interpolation to the LES
 * node) by direct summation in FP64; the exact stress is computed only at
 * the guarded points.
 *  plan  a Gaussian-kernel plan (EF_KERNEL_GAUSSIAN or _HAT) of the LES grid
 *        the features were taken on: n must be nly nlz nlx and point
 *        p = (J nlz + Z) nlx + X (the order of ef_closure_features)
 *  u     device [3][ny][nz][nx], the plan's element type (double for
 *        EF_PREC_FP64 plans, float otherwise): the snapshot of the features
 * *n_fallback (if not NULL) receives the number of guarded points
 * (synchronises).  The plan is only read; calls on one closure must not
 * overlap on the GPU.  Errors: EF_ERR_ARG, EF_ERR_SHAPE (n),
 * EF_ERR_UNSUPPORTED (a differential-filter plan), EF_ERR_CUDA,
 * EF_ERR_TIMEOUT (as ef_closure_infer).
 */
int ef_closure_infer_exact(ef_closure *closure, const float *feats, float *tau_out, long n, ef_plan *plan,
                           const void *u, long *n_fallback, void *stream);

/* Read (and clear) the closure's device error word; synchronises `stream`.
 * Returns EF_OK or the recorded ef_status (EF_ERR_TIMEOUT). */
int ef_closure_check_device_error(ef_closure *closure, void *stream);

/* One forward and backward pass over n <= batch points without an update:
 * host grad_out[param count] (layout of ef_closure_get_params), *loss_out. */
int ef_closure_gradients(ef_closure *closure, const float *feats, const float *tau, long n, float *grad_out,
                         float *loss_out, void *stream);

/* Parameter count; parameters are stored per layer as W [out][in] then b [out]. */
long ef_closure_param_count(const ef_closure *closure);
/* Copy the FP32 master parameters (host [count]) and the 32 statistics
 * (fmu[10], fsd[10], tmu[6], tsd[6]) out or in (either pointer may be NULL). */
int ef_closure_get_params(const ef_closure *closure, float *params, double *norm_stats);
int ef_closure_set_params(ef_closure *closure, const float *params, const double *norm_stats);

/* Checkpoint to / from a flat little-endian file with a CRC-32 (weights,
 * Adam moments, step count, statistics); resuming training from a checkpoint
 * reproduces an uninterrupted run bit for bit. */
int ef_closure_save(const ef_closure *closure, const char *path);
int ef_closure_load(ef_closure *closure, const char *path);

/* ------------------------------------------------------------------------
 * The loop of Sec. 3 and Fig. 2: at every time step the DNS field is
 * filtered, T_ij (Eq. 6) is formed from it, and the explicitly filtered LES
 * equations (Eq. 6: Eq. 5 with bar(u_i u_j) = ubar_i ubar_j + T_ij) are
 * advanced one step with that T_ij.  The LES here is a minimal collocated
 * solver on the LES nodes of the filter, FP64 throughout:
 *   - second-order central differences (periodic in x and z, non-uniform in
 *     y), the three-point Laplacian;
 *   - R_i = -d_j (ubar_i ubar_j + T_ij) + nu lap ubar_i + forcing [i = 1] at
 *     the interior nodes, `forcing` the imposed mean pressure gradient (Sec. 3
 *     drives the channel with a constant one; 1 in units u_tau^2 / delta);
 *   - wall rows by Eq. 10 and Eq. 11: ubar_2 = 0, ubar_1 and ubar_3 the
 *     filter-consistent wall value F(u_i), taken from a filtered DNS field
 *     of the step (no slip when none is given);
 *   - third-order low-storage Runge-Kutta (the scheme family of Sec. 3) or
 *     forward Euler, each substep followed by the projection below, with
 *     T_ij and the wall values held over the step;
 *   - projection (the pressure step of the fractional-step method): the
 *     orthogonal projection, in the inner product weighted by
 *     (y[j+1] - y[j-1]) / 2, onto velocities of zero discrete divergence at
 *     every interior node, the wall values held; computed by discrete
 *     Fourier transforms in x and z (mixed-radix FFTs for lines of at most
 *     1024 points with prime factors 2, 3, 5, 7; plain sums otherwise) and
 *     two tridiagonal solves in y per mode.
 * Fields are device [3][ny][nz][nx] FP64 with x fastest; tau is the
 * [6][ny][nz][nx] output of ef_subfilter_stress in the precision of its
 * plan (double for EF_PREC_FP64, float otherwise), as is the wall-value
 * field ubar_bc.  The solver owns its scratch (about 13 doubles per node,
 * allocated by ef_les_create); calls on one solver must not overlap on the
 * GPU.  The other calls are asynchronous on `stream` and allocate nothing;
 * they return EF_ERR_ARG for a NULL pointer, a non-positive dt, an unknown
 * precision or a current device other than the solver's, and EF_ERR_CUDA if
 * a launch fails.
 */
enum { EF_LES_RK3 = 0, EF_LES_EULER = 1 };
typedef struct {
    double nu;          /* kinematic viscosity (1 / Re_tau in wall units), >= 0 */
    double forcing;     /* mean pressure gradient driving u_1 */
    int scheme;         /* EF_LES_RK3 or EF_LES_EULER */
} ef_les_cfg;
typedef struct ef_les ef_les;

/* Set-up on the current device for the LES grid `les` (3 to 4096 nodes per
 * direction, at most 2^28 in all).  Errors: EF_ERR_ARG, EF_ERR_SHAPE,
 * EF_ERR_OOM, EF_ERR_CUDA. */
int ef_les_create(const ef_grid *les, const ef_les_cfg *cfg, ef_les **out);
void ef_les_destroy(ef_les *les);

/* One time step of length dt, in place on ubar (device [3][ny][nz][nx]
 * double).  tau (may be NULL: no subfilter term) and ubar_bc (may be NULL:
 * no slip) in `precision` as above.  Its wall rows are set first. */
int ef_les_step(ef_les *les, double *ubar, const void *tau, const void *ubar_bc, int precision, double dt,
                void *stream);

/* The projection alone: u = P ustar (u may equal ustar; wall rows copied). */
int ef_les_project(ef_les *les, const double *ustar, double *u, void *stream);

/* The discrete divergence of u at every node (zero on the wall rows). */
int ef_les_divergence(ef_les *les, const double *u, double *div, void *stream);

/* The right-hand side R (device [3][ny][nz][nx], zero on the wall rows) of
 * u as given (its wall rows are used as they are). */
int ef_les_rhs(ef_les *les, const double *u, const void *tau, int precision, double *rhs, void *stream);

/*
 * ef_apost_step -- one step of the loop of Fig. 2: ef_subfilter_stress of
 * the DNS snapshot u_dns into ubar_dns and tau (device, the plan's LES grid
 * and precision; the caller's scratch), then ef_les_step of ubar_les with
 * that tau and the wall values of ubar_dns.  The plan's LES grid must be the
 * solver's: the call compares the node counts and box lengths (EF_ERR_SHAPE
 * if they differ); the y nodes are the caller's to keep equal (both set-up
 * calls take them).  ubar_les must be a buffer of its own
 * (EF_ERR_ARG if it is ubar_dns or tau).  Other errors as the two calls.
 */
int ef_apost_step(ef_plan *plan, ef_les *les, const void *u_dns, void *ubar_dns, void *tau, double *ubar_les,
                  double dt, void *stream);

/*
 * ef_debug_fail_alloc -- test hook: the n-th device allocation the library
 * makes from now on (n = 0: the next one) fails as if the device were out of
 * memory, so that the set-up calls' EF_ERR_OOM paths (and the release of
 * what they had allocated) can be tested without exhausting the GPU; n = -1
 * disables the hook.  Process-wide.  Errors: EF_ERR_ARG (n < -1).
 */
int ef_debug_fail_alloc(int n);

/* Thread-local message of the last failed call on this thread ("" if none). */
const char *ef_last_error(void);

/* Library version string. */
const char *ef_version(void);

#ifdef __cplusplus
}
#endif

#endif /* ELES_H */
