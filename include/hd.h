/*
 * hd.h -- C ABI of the GB300 library for massively parallel local Monte Carlo
 * (MPMC) of hard disks: Engel, Anderson, Glotzer, Isobe, Bernard, Krauth,
 * "Hard-disk equation of state", arXiv:1211.1645.
 *
 * The library owns all device state.  Callers pass plain host pointers and
 * sizes; no call takes or returns a framework type.  Every call returns an
 * hd_status and never aborts the process.  Output-returning calls synchronise
 * the context's stream.  A CUDA failure or a device-side error flag leaves the
 * context in a sticky error state: every later call except hd_destroy returns
 * HD_ERR_STATE.  After HD_ERR_TIMEOUT in particular, a bulk copy that gave up
 * waiting may still have been in flight: destroy the context and treat what it
 * held on the device as lost.
 *
 * Units: sigma is the disk radius.  Positions are in [0, L) x [0, L) with
 * periodic boundaries; L = sqrt(N pi sigma^2 / eta) (Sec. II.A).
 *
 * A context holds R >= 1 independent chains ("replicas").  hd_init makes
 * R = 1; hd_batch_init makes R chains of different N and eta that advance
 * together in the same kernel launches.  Arrays documented as [R] or
 * [sum N_r] hold one entry per replica / per disk of every replica,
 * replica-major, disks in id order.
 */
#ifndef HD_H
#define HD_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct hd_ctx hd_ctx;

typedef enum hd_status {
    HD_OK = 0,
    HD_ERR_ARG = 1,      /* invalid argument; the context is unchanged           */
    HD_ERR_CUDA = 2,     /* a CUDA runtime call failed; the context is poisoned  */
    HD_ERR_OVERFLOW = 3, /* a cell held more disks than its capacity (device)   */
    HD_ERR_TIMEOUT = 4,  /* a bounded device-side wait gave up                  */
    HD_ERR_REACH = 5,    /* a measurement stencil would wrap around the box      */
    HD_ERR_STATE = 6     /* the context is in a sticky error state               */
} hd_status;

typedef enum hd_precision {
    HD_FP64 = 0,   /* plain IEEE double, no FMA contraction                     */
    HD_FIXED32 = 1 /* cell-relative int32 in units of 2^-24 sigma, int64 test  */
} hd_precision;

typedef enum hd_lattice {
    HD_LATTICE_SQUARE = 0,    /* n = ceil(sqrt N) columns of spacing L/n          */
    HD_LATTICE_TRIANGULAR = 1 /* same, odd rows shifted by half a spacing        */
} hd_lattice;

/* Options shared by all replicas of a context.  A zero field takes the
 * default given in brackets; so does a negative hist_bins, hist_dr, cell_min,
 * block_threads or threads_per_cell, while any other negative field is
 * HD_ERR_ARG. */
typedef struct hd_opts {
    int32_t precision;       /* hd_precision [HD_FP64]                              */
    int32_t lattice;         /* hd_lattice [HD_LATTICE_SQUARE]                      */
    int32_t trials_per_cell; /* n_t, trial moves per occupied active cell and pass;
                                Sec. II.B fixes it independent of occupancy
                                [ceil(N / m^2), per replica]                        */
    int32_t hist_bins;       /* K, contact-histogram bins, 5..512 (the quartic fit
                                needs five) [50]                                    */
    double hist_dr;          /* bin width in sigma [1e-3]; Sec. II.C.1              */
    double cell_min;         /* minimum cell side in sigma, >= 2 [2]; Sec. II.B     */
    int32_t block_threads;   /* threads per block of the split sweep kernels [128]  */
    int32_t sweep_kernel;    /* HD_SWEEP_SPLIT: a rebuild launch and four colour-pass
                                launches per sweep, each pass thread copying its
                                neighbours with cp.async [default]; HD_SWEEP_TMA:
                                the same launches, each pass block staging its
                                neighbourhood (six row segments of the colour
                                planes) with bulk copies (TMA); HD_SWEEP_FUSED: one
                                launch per sweep, tiles staged in shared memory;
                                HD_SWEEP_PERSISTENT: one launch for up to 256
                                sweeps, its blocks taking rebuild and colour-pass
                                work items of two-cell-row bands in order, each
                                item starting once the previous phase is done in
                                its band and the two next to it (a wavefront, no
                                launch boundary between phases).  All give
                                bit-identical chains.  A bulk-copy pass that
                                cannot stage its segments, or a persistent sweep
                                whose bounded dependency wait gives up, sets
                                HD_ERR_TIMEOUT. */
    int32_t threads_per_cell; /* G threads per active cell in the split colour pass:
                                1, 2, 4 or 8 [1].  The G lanes share the cell's
                                draws and proposals and split the overlap tests
                                against its eight neighbours, combined by a warp
                                ballot; the chain is the same.  G > 1 needs
                                HD_SWEEP_SPLIT and block_threads * G <= 512.    */
    const double *cell_min_per_replica; /* [R] minimum cell side of each replica
                                (>= 2 sigma), e.g. chosen per state point by an
                                autotuner; NULL: cell_min for every replica [NULL].
                                Read during hd_init / hd_batch_init only.       */
    int32_t strips;          /* graph wavefront of the steps hd_run captures, one
                                replica, HD_SWEEP_SPLIT, threads_per_cell 1: the
                                cell grid as K strips of two-cell-row bands, each
                                strip's rebuild and colour passes on its own graph
                                branch, a strip's phase waiting only for the
                                previous phase in itself and the two next to it
                                (in the checkerboard of Sec. II.B a pass reads
                                one cell row beyond its own cells and a rebuild
                                moves a disk by at most one cell).  Same chain.
                                0: automatic (16 when the colour pass is 1.5 to
                                3.5 waves of resident blocks deep, 8 when it is
                                deeper, none when it is shallower);
                                1: none; 2 .. 64: K strips (at most m / 2, and
                                only for one replica, the split kernels and one
                                thread per cell; else HD_ERR_ARG) [0]          */
    int32_t replica_branches; /* the steps hd_run captures for 2 .. 64 replicas
                                (HD_SWEEP_SPLIT, threads_per_cell 1) run each
                                replica's sweeps on its own graph branch with
                                one-replica launches, the replicas' chains
                                concurrently (independent chains, Sec. IV.A's
                                scan); the measurement stays one batched launch.
                                Same chains.  0: automatic (on where it applies);
                                1: off [0]                                      */
} hd_opts;

enum { HD_SWEEP_SPLIT = 0, HD_SWEEP_FUSED = 1, HD_SWEEP_TMA = 2, HD_SWEEP_PERSISTENT = 3 };

/* Geometry of one replica as realised by the library. */
typedef struct hd_geometry {
    int64_t N;
    int32_t m;          /* cells per side (even, >= 4)                            */
    int32_t capacity;   /* disk slots per cell                                    */
    int32_t trials_per_cell;
    int32_t precision;
    int32_t hist_bins;  /* K of the contact histogram                             */
    int32_t graph_branches; /* concurrent branches of the sweeps of hd_run's step
                               graphs: the strips of a one-replica context, the
                               replicas of a batch with replica branches, else 1 */
    double L;           /* box side in sigma (fixed form: m * W * 2^-24)          */
    double w;           /* cell side in sigma                                     */
    double delta;       /* maximum displacement per axis in sigma (realised)      */
    double eta;         /* realised packing fraction N pi / L^2                   */
    double hist_dr;     /* realised histogram bin width in sigma                  */
    int64_t sweeps;     /* sweeps done                                            */
} hd_geometry;

/* Fill *o with the defaults of each field (the cell side of Sec. II.B, the
 * trials per cell of Sec. II.B, the histogram of Sec. II.C.1). */
void hd_default_opts(hd_opts *o);

/* Human-readable name of a status code (static storage).  Bookkeeping of the
 * library: the paper has no counterpart. */
const char *hd_status_string(hd_status s);

/*
 * Create one chain of N disks of radius sigma at packing fraction eta
 * (Sec. II.A), trial displacements uniform in [-delta, delta]^2 (sigma units
 * scale with sigma), Philox4x32-10 keyed by seed.  Disks start on the lattice
 * of opts->lattice, binned into an unshifted grid of m x m cells where m is
 * the largest even integer with L/m >= cell_min (Sec. II.B).
 * Errors: HD_ERR_ARG if N < 2, eta <= 0, the lattice would overlap
 * (L / ceil(sqrt N) < 2 sigma), m < 4, delta < 0 or delta >= cell side, a
 * delta / sigma in (0, 2^-900) (the FP64 step's exact scaling assumes a
 * normal result), a cell could hold more than 9 disks, or the fixed form
 * would overflow int32.
 * *out receives the context (NULL on error); release it with hd_destroy.
 */
hd_status hd_init(hd_ctx **out, int64_t N, double eta, double sigma, double delta,
                  uint64_t seed, const hd_opts *opts);

/*
 * Create R independent chains in one context (the equation-of-state scan of
 * Sec. IV.A as one batch).  N[R], eta[R], delta[R], seed[R] are per replica;
 * sigma and opts are shared.  Same errors as hd_init, per replica, and
 * HD_ERR_ARG unless 1 <= R <= 65535.
 */
hd_status hd_batch_init(hd_ctx **out, int32_t R, const int64_t *N, const double *eta, double sigma,
                        const double *delta, const uint64_t *seed, const hd_opts *opts);

/* Release all device and host memory of the context.  NULL is allowed.
 * Bookkeeping of the library: the paper has no counterpart. */
hd_status hd_destroy(hd_ctx *ctx);

/* Launch all later work of the context on this CUDA stream (a cudaStream_t
 * passed as void*; NULL = the legacy default stream).  Bookkeeping of the
 * library: the paper has no counterpart. */
hd_status hd_set_stream(hd_ctx *ctx, void *stream);

/*
 * Advance every replica by n checkerboard sweeps (Sec. II.B).  One sweep:
 * draw a uniform grid shift in [0, w)^2 and a random order of the four
 * colours; move every disk into the shifted cell frame (cell lists rebuilt,
 * occupants ordered by id); then, for each colour in that order, every
 * active cell shuffles its occupants and makes n_t serial trial moves,
 * rejecting moves that leave the cell or overlap a disk of the 3 x 3 cell
 * neighbourhood.  Asynchronous on the context stream.  n >= 0.
 */
hd_status hd_sweep(hd_ctx *ctx, int64_t n);

/*
 * Contact-value pressure (Eqs. 2 and 4): histogram of pair distances in
 * [2 sigma, 2 sigma + K dr) with K bins, g(r_k) = (n_k / p) / (2 pi r_k dr /
 * V) at bin centres with p = N^2 / 2, least-squares quartic in r - 2 sigma
 * extrapolated to contact (Sec. II.C.1), beta P / rho = 1 + 2 eta g(2 sigma+).
 * Outputs (host, caller-owned, any may be NULL): betaP_over_rho[R],
 * g_contact[R], hist[R * K] raw counts.  Synchronises.
 * Errors: HD_ERR_REACH if 2 sigma + K dr needs a cell stencil wider than the
 * box.
 */
hd_status hd_pressure(hd_ctx *ctx, double *betaP_over_rho, double *g_contact, uint64_t *hist);

/*
 * Bond-orientational order (Eq. 8): psi_j = (1/6) sum over the six nearest
 * neighbours (minimum image, ties by lower id) of exp(6 i phi_jk), phi from
 * the +x axis; Psi_6 = (1/N) sum_j psi_j per replica.  Outputs (host,
 * caller-owned, any may be NULL): re[R], im[R], local[2 * sum N_r]
 * interleaved (re, im) by disk id.  The fixed form computes psi_j in float
 * and reduces in double.  Synchronises.
 * Errors: HD_ERR_REACH if a disk has fewer than six neighbours within the
 * largest stencil the box allows.
 */
hd_status hd_psi6(hd_ctx *ctx, double *re, double *im, double *local);

/*
 * The configuration: the disk centres in the periodic L x L box of Sec. II.A,
 * as global coordinates in [0, L) (the cell frame of Sec. II.B undone).
 *   hd_positions         host array, caller-owned, [2 * sum N_r] interleaved
 *                        x, y by disk id.  Synchronises.
 *   hd_positions_device  the same into a device buffer of 2 * sum N_r doubles
 *                        (caller-owned).  Asynchronous.
 */
hd_status hd_positions(hd_ctx *ctx, double *xy);
hd_status hd_positions_device(hd_ctx *ctx, double *xy_device);

/*
 * Replace all positions of the configuration (Sec. II.A) (host,
 * [2 * sum N_r], periodic images allowed; pinned memory gives the fastest
 * copy).  The positions are copied to the device
 * and binned there into the unshifted cell frame; counters and the sweep
 * index are kept.  Overlapping input is accepted (measurements then count
 * it); the fixed form rounds to the 2^-24 sigma grid.  Synchronises.
 * Errors (the previous state is kept): HD_ERR_OVERFLOW if a cell would hold
 * more disks than its capacity; HD_ERR_ARG for a non-finite coordinate.
 */
hd_status hd_set_positions(hd_ctx *ctx, const double *xy);

/* Attempted and accepted trial moves since creation, per replica [R] (the
 * trial moves of Sec. II.B; Table II counts displacements per disk).
 * Attempts count every trial, including moves rejected at the cell
 * boundary.  Host arrays, either may be NULL.  Synchronises. */
hd_status hd_stats(hd_ctx *ctx, uint64_t *attempts, uint64_t *accepts);

/* Geometry of replica r: box and packing fraction (Sec. II.A, Eq. 1), cell
 * grid (Sec. II.B), histogram bin width (Sec. II.C.1).  HD_ERR_ARG unless
 * 0 <= r < R. */
hd_status hd_get_geometry(hd_ctx *ctx, int32_t r, hd_geometry *g);

/* Number of replicas of the context (independent chains of the
 * equation-of-state scan, Sec. IV.A); 0 for NULL. */
int32_t hd_replicas(const hd_ctx *ctx);

/*
 * Batched engine for long runs (the equation-of-state scan of Sec. IV.A as
 * one batch): `steps` steps, each `sweeps_per_step` sweeps (as hd_sweep) and,
 * when `measure` != 0, one measurement of every replica -- the contact
 * pressure of hd_pressure and the global Psi_6 of hd_psi6 -- appended on the
 * device to a series (no host synchronisation).  measure == 2 also keeps the
 * local psi_j field of each measurement (Eq. 8) on the device, for
 * hd_psi6_local_device.  Each distinct step is captured once as a CUDA graph
 * and replayed, its sweeps on concurrent branches where hd_opts asks for strips
 * or replica branches (graph_branches of hd_get_geometry); while profiling is
 * enabled the graph instead runs every kernel in order, with a timing event
 * before and after it, and each replay is followed by a synchronisation that
 * adds the kernels' times to hd_kernel_times.  Capturing and instantiating a
 * step graph is a one-time cost per distinct step (at N = 2^20 about 6 ms
 * serial, about 0.13 s as 16 strips, whose graph holds ~8000 kernel nodes per
 * 100 sweeps).
 * Asynchronous on the context stream (unless profiling).  R <= 1024.
 * Errors: HD_ERR_ARG for negative counts, an empty step or measure outside
 * 0..2; HD_ERR_REACH as hd_pressure when measuring.
 */
hd_status hd_run(hd_ctx *ctx, int64_t steps, int32_t sweeps_per_step, int32_t measure);

/* The local psi_j field (Eq. 8) of the last measurement that kept it
 * (hd_psi6 with a local output, or hd_run with measure == 2), copied into a
 * caller-owned device buffer of 2 * sum N_r doubles, (Re, Im) by disk id.
 * Asynchronous. */
hd_status hd_psi6_local_device(hd_ctx *ctx, double *local_device);

/* Capacity of the measurement series of hd_run (pressure, Sec. II.C.1, and
 * Psi_6, Sec. III) in steps [4096, allocated by the first measuring hd_run];
 * reserving clears the series.  A full series keeps its first entries and
 * drops later ones. */
hd_status hd_series_reserve(hd_ctx *ctx, int64_t steps);

/* Copy up to max_steps recorded steps to out[n][R][4] = (beta P / rho of
 * Eq. 4, g(2 sigma+), Re and Im Psi_6 of Eq. 8); *n_steps receives the
 * number copied.  Synchronises. */
hd_status hd_series(hd_ctx *ctx, int64_t *n_steps, double *out, int64_t max_steps);

/*
 * Autocorrelation of the global orientational order over the recorded series
 * (Sec. III, Eq. 9): C(d) = <Psi_6(t) Psi_6*(t + d)>_t / <|Psi_6|^2>, the
 * numerator averaged over the T - d pairs of a series of T entries, the
 * denominator over all T, so C(0) = 1.  Lags d = 0 .. max_lag in units of
 * recorded steps.  acf (host, caller-owned): [R][max_lag + 1][2] = (Re, Im).
 * Synchronises.  Errors: HD_ERR_ARG if max_lag < 0 or max_lag >= T.
 */
hd_status hd_psi6_acf(hd_ctx *ctx, int64_t max_lag, double *acf);

/*
 * Correlation time from the purely exponential part of C (Sec. III, Table
 * II): the least-squares line through (d, ln Re C(d)) over
 * lag_lo <= d <= lag_hi where Re C(d) > 0; tau = -1 / slope, in recorded
 * steps (multiply by sweeps per step and attempts per disk per sweep for
 * Table II's displacements per disk).  tau (host, caller-owned): [R]; NaN
 * where fewer than two lags qualify or the slope is not negative.
 * Synchronises.  Errors: HD_ERR_ARG unless 0 <= lag_lo <= lag_hi < T.
 */
hd_status hd_psi6_tau(hd_ctx *ctx, int64_t lag_lo, int64_t lag_hi, double *tau);

/*
 * Coarse-grained psi_6 field of the current state (the sampling-area
 * averages of Sec. IV, Figs. 5-6): the mean of psi_j (as hd_psi6) over the
 * disks whose centres lie in each of bins x bins half-open squares of side
 * L / bins; area index floor(x bins / L) per axis (fixed form:
 * floor(X bins / LF) of the exact integer coordinate).  field (host,
 * caller-owned): [R][bins][bins][2] = (Re, Im), indexed [r][iy][ix]; NaN for
 * an empty area.  Sums are accumulated with atomics (summation order not
 * fixed).  Synchronises.
 * Errors: HD_ERR_ARG unless 1 <= bins <= 65536 and R bins^2 <= 2^28;
 * HD_ERR_REACH as hd_psi6.
 */
hd_status hd_psi6_field(hd_ctx *ctx, int32_t bins, double *field);

/*
 * Structure factor (Sec. IV.C, Eq. 10) of the current state:
 * S(q) = (1/N) |sum_n exp(i q . x_n)|^2 at the box-periodic wave vectors
 * q = 2 pi (h, k) / L.  hk (host): [R][nq][2] integers (h, k) per replica;
 * S (host, caller-owned): [R][nq].  Phases are reduced to turn fractions
 * (exactly, in integers, in the fixed form) before the sine and cosine.
 * Synchronises.  Errors: HD_ERR_ARG unless 1 <= nq <= 65536 (and the
 * partial sums fit the scratch bound).
 */
hd_status hd_structure_factor(hd_ctx *ctx, int32_t nq, const int32_t *hk, double *S);

/*
 * q_0 of the positional order (Sec. IV.C): the wave vector of largest S
 * among the (2 half_width + 1)^2 box-grid points around the first-shell
 * reciprocal vector of a triangular lattice of the same density
 * (|q| = 4 pi / (a sqrt 3), area per disk sqrt(3) a^2 / 2), oriented by the
 * global Psi_6 (angle arg(Psi_6) / 6 + 30 degrees); the paper leaves q_0 to
 * the maximum of S because defects stretch the effective lattice constant.
 * hk0 (host): [R][2] = (h, k); S0 (host, nullable): [R].  Synchronises.
 * Errors: HD_ERR_ARG unless 0 <= half_width <= 64; HD_ERR_REACH as hd_psi6.
 */
hd_status hd_positional_q0(hd_ctx *ctx, int32_t half_width, int32_t *hk0, double *S0);

/*
 * Positional order field (Sec. IV.C, Eq. 11): chi_j = exp(i q_0 . x_j) with
 * q_0 = 2 pi hk0[r] / L, averaged over bins x bins sampling areas as in
 * hd_psi6_field.  hk0 (host): [R][2]; field (host, caller-owned):
 * [R][bins][bins][2], NaN for an empty area.  Synchronises.
 * Errors: HD_ERR_ARG unless 1 <= bins <= 65536 and R bins^2 <= 2^28.
 */
hd_status hd_positional_field(hd_ctx *ctx, const int32_t *hk0, int32_t bins, double *field);

/*
 * Positional correlation function (Sec. IV.D, Eq. 12):
 * C(r_k) = < exp(i q_0 . (x_n - x_m)) > over the ordered pairs n != m whose
 * minimum-image separation d (from the global positions,
 * d = x_m - x_n - L rint((x_m - x_n) / L), d^2 = dx dx + dy dy) satisfies
 * max(r_k - sigma, 0)^2 <= d^2 <= (r_k + sigma)^2, at r_k = (k + 1) dr,
 * k = 0 .. nr - 1 (dr in the caller's length unit).  hk0 (host): [R][2];
 * C (host, caller-owned): [R][nr][2] = (Re, Im), NaN where no pair
 * qualifies.  Sums are accumulated with atomics.  Synchronises.
 * Errors: HD_ERR_ARG unless 1 <= nr <= 1024 and dr > 0; HD_ERR_REACH if the
 * cells within reach of r_nr + sigma would wrap around the box.
 */
hd_status hd_positional_corr(hd_ctx *ctx, const int32_t *hk0, int32_t nr, double dr, double *C);

/* Forget the recorded steps of the series of Eq. 4 and Eq. 8 values
 * (asynchronous). */
hd_status hd_series_clear(hd_ctx *ctx);

/*
 * Checkpoint and resume of long runs (the paper's production runs span
 * 10^11 - 10^13 displacements, Table I).  The chain state is the cell frame
 * (occupancy, offsets and ids in slot order), the current frame shift, the
 * sweep counters and the trial counters; with the counter-based generator a
 * restored context continues the chain bit-exactly.
 *   hd_checkpoint_size  *bytes receives the size of the checkpoint.
 *   hd_checkpoint       writes it to a caller-owned host buffer of at least
 *                       that size; synchronises.
 *   hd_restore          loads a checkpoint into a context created with the
 *                       same N, eta, sigma, delta, seed and options
 *                       (HD_ERR_ARG if the header does not match); the
 *                       measurement series is kept.  Synchronises.
 */
hd_status hd_checkpoint_size(hd_ctx *ctx, size_t *bytes);
hd_status hd_checkpoint(hd_ctx *ctx, void *buf, size_t bytes);
hd_status hd_restore(hd_ctx *ctx, const void *buf, size_t bytes);

/*
 * Maximum trial displacement per replica: the delta of the trial moves of
 * Sec. II.B (Sec. III runs each algorithm at its optimal parameters).
 *   hd_set_delta   sets delta[R] (sigma units; 2^-900 sigma <= delta < cell
 *                  side, and at least one 2^-24 sigma step in the fixed form).
 *   hd_tune_delta  runs `probes` bursts of `sweeps_per_probe` sweeps,
 *                  measuring each replica's acceptance and scaling its delta
 *                  by (acceptance/target)^0.7 (clamped to a factor 1/4..4 and
 *                  to the valid range) toward `target` in (0, 1); the chains
 *                  advance during tuning and delta is frozen afterwards, so
 *                  production sweeps keep detailed balance.  delta_out[R]
 *                  (nullable) receives the tuned values.  Synchronises.
 */
hd_status hd_set_delta(hd_ctx *ctx, const double *delta);
hd_status hd_tune_delta(hd_ctx *ctx, double target, int32_t sweeps_per_probe, int32_t probes, double *delta_out);

/*
 * Global Psi_6 = (1/N) sum_j psi_j from a per-disk field that the caller
 * already holds on the device (for instance the local field of hd_psi6,
 * copied to device memory), for callers that may not allocate device memory
 * at this point: inside a CUDA stream capture, under a framework that owns
 * every allocation, or in a loop where an allocation could block or fail.
 * The paper has no counterpart; it is a deployment variant of the reduction
 * behind hd_psi6, with the same exact sum, so on the same field it returns
 * hd_psi6's value bit for bit.
 *   psi_local_device  device array of N (Re, Im) double pairs, by disk id,
 *                     8-byte aligned (HD_ERR_ARG otherwise)
 *   N                 1 <= N <= 16,777,216 (4096 blocks of 4096 values);
 *                     larger N returns HD_ERR_ARG
 *   out_device        device array of 2 doubles receiving (Re, Im), 8-byte
 *                     aligned
 *   stream            cudaStream_t as void* (NULL: legacy default stream)
 * The call allocates and frees nothing: its block partial sums live in a
 * fixed 256 KiB device array of the library, held on every device that loads
 * the library until the process exits.  Its device address is looked up on
 * every call (cudaGetSymbolAddress, which allocates nothing); the first call
 * on a device may load the library's device code, so make it outside any
 * stream capture.  All calls share that array, so calls that may overlap on
 * the GPU race and must be ordered by the caller.  Asynchronous; returns
 * HD_ERR_ARG for NULL or misaligned pointers or N out of range, HD_ERR_CUDA
 * if a launch or the lookup fails.
 */
hd_status hd_psi6_mean_noalloc(const double *psi_local_device, int64_t N, double *out_device, void *stream);

/*
 * Instrumentation (no counterpart in the paper).  The library counts every
 * kernel it launches, by class.  With profiling enabled it also brackets each
 * launch with CUDA events on the context stream; hd_kernel_times then
 * synchronises and reports the summed device time per class.  Enabling
 * (enable != 0) resets both tallies; disabling keeps them readable.
 * ms[HD_KERNEL_CLASSES] and launches[HD_KERNEL_CLASSES] are host arrays, either
 * may be NULL.
 */
typedef enum hd_kernel_class {
    HD_K_DRAWS = 0,      /* per-sweep shift and colour-order draws           */
    HD_K_REBUILD = 1,    /* move disks into the shifted frame, rebuild cells  */
    HD_K_PASS = 2,       /* one colour pass of trial moves                    */
    HD_K_HIST = 3,       /* contact-shell pair histogram                      */
    HD_K_FIT = 4,        /* g(r) normalisation, quartic fit, pressure         */
    HD_K_PSI6 = 5,       /* local psi_6                                       */
    HD_K_PSI6_REDUCE = 6,/* global Psi_6 reduction                            */
    HD_K_POSITIONS = 7,  /* cell frame to global positions                    */
    HD_K_SWEEP = 8,      /* whole sweeps in one launch (fused or persistent)  */
    HD_K_ANALYSIS = 9,   /* Psi_6 autocorrelation, correlation time, field    */
    HD_KERNEL_CLASSES = 10
} hd_kernel_class;

hd_status hd_profile(hd_ctx *ctx, int32_t enable);
hd_status hd_kernel_times(hd_ctx *ctx, double *ms, int64_t *launches);

#ifdef __cplusplus
}
#endif

#endif /* HD_H */
