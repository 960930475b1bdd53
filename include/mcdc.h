/*
 * mcdc.h -- C-ABI of the B300 (sm_103a) Monte Carlo neutron transport library.
 *
 * Scope: time-dependent, multigroup, fixed-source transport in
 * non-multiplying media on a uniform Cartesian mesh with a track-length flux
 * tally into (cell, group, time bin), analog or with weight windows.
 *
 * Paper passages the calls stand for (arXiv 2409.04668, "Performant and
 * Portable Monte Carlo Neutron Transport via Numba"):
 *  - "MC/DC on CPUs": the user describes physics, materials and parameters
 *    through input functions; initialisation builds one typed global record
 *    holding inputs, meshes, particle banks and tallies (-> the problem
 *    handle); a fixed-source run transports every particle until capture,
 *    a time or space boundary, a time census or a variance-reduction event
 *    ends its history (-> mcdc_run); finalisation returns the tallies with
 *    their statistical error (-> mean and relative error outputs).
 *  - "MC/DC on GPUs": device memory is allocated and the global record is
 *    copied to the GPU once at initialisation, transport kernels run until
 *    the work is done, and the results are copied back once (-> create
 *    uploads, run downloads); the profile in "Performance" shows why the
 *    allocation must not be repeated per run.
 *  - Figure "jitfunctions" (move_particle) and Figure "forcpuvgpu"
 *    (loc2index + atomic add into a tally) define one flight's move and
 *    tally scatter.
 *
 * Conventions
 *  - Every call returns MCDC_OK (0) or a negative MCDC_ERR_* code;
 *    mcdc_last_error() gives a message for the calling thread.
 *  - Input arrays are read during the call and copied: the caller keeps
 *    ownership and may free them afterwards.
 *  - Output arrays are caller-owned and may be host or device pointers
 *    (the library asks CUDA which); device outputs are written on the run's
 *    stream, host outputs are complete when the call returns.
 *  - Tally layout: [nz][ny][nx][G][T] (x fastest among cells), T = number
 *    of time bins, or 1 in steady state.  Values are track length per
 *    source particle per unit cell volume, integrated over the time bin.
 *  - A problem handle is not thread-safe; runs are deterministic for a
 *    given (seed, history offset, histories, batches) up to the order of
 *    floating-point additions.
 */
#ifndef MCDC_B300_H
#define MCDC_B300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define MCDC_OK                  0
#define MCDC_ERR_INVALID        -1   /* bad argument or problem data            */
#define MCDC_ERR_OOM            -2   /* device allocation failed                */
#define MCDC_ERR_CUDA           -3   /* a CUDA call failed                      */
#define MCDC_ERR_BANK_OVERFLOW  -4   /* reserved: a split that finds no room is
                                        skipped (mcdc_stats.splits_dropped)    */
#define MCDC_ERR_TIMEOUT        -5   /* a bounded device wait gave up (tensor-core
                                        kernels of the importance network)     */
#define MCDC_ERR_NO_DEVICE      -6   /* no usable sm_103 device                 */
#define MCDC_ERR_CHECK          -7   /* checked build only: an index failed its
                                        bounds check and its access was skipped
                                        (mcdc_last_error: the site and index)  */

#define MCDC_BC_VACUUM   0
#define MCDC_BC_REFLECT  1

#define MCDC_SRC_ISOTROPIC 0
#define MCDC_SRC_BEAM      1

#define MCDC_PREC_FP64   0   /* every step in FP64: event-exact with the FP64 reference      */
#define MCDC_PREC_FP32   1   /* FP32 direction/distance/xs, FP64 position, time and tallies
                                (see mcdc_options.flight_sampling)                          */
#define MCDC_PREC_FP32_LOCAL 2 /* FP32 flights: positions as FP32 offsets from exact FP64 cell
                                  faces, time as FP32 time to the next exact FP64 census edge;
                                  FP64 tally reduction                                         */

#define MCDC_TALLY_AUTO    0
#define MCDC_TALLY_SHARED  1  /* per-CTA privatised tally in shared memory, one batch per CTA */
#define MCDC_TALLY_GLOBAL  2  /* device-wide tally, batches run one after another            */

/* Flux estimators (mcdc_options.estimator).  Both estimate the same flux per
 * (cell, group, time bin), normalised by N x cell volume. */
#define MCDC_EST_TRACK     0  /* track length: every flight scores w x d                     */
#define MCDC_EST_COLLISION 1  /* collision: every collision scores w / sigma_t of the arriving
                                 particle (its group, cell and time bin before the collision) */
#define MCDC_EST_COMBINED  2  /* both, from the same histories, into two tallies; the output
                                 per bin (and for the region scalar) is their minimum-variance
                                 combination a x + (1 - a) y of the track-length (x) and
                                 collision (y) batch means, a = (s_yy - s_xy) / (s_xx + s_yy -
                                 2 s_xy) from the sample (co)variances of the batch values
                                 (a = 1/2 when that denominator is not positive), clipped to
                                 [0, 1]; error from the variance of the combination at a  */

/* Uniform Cartesian mesh.  An axis with n == 1 and width <= 0 or infinite is
 * unbounded (no faces): a 1-D slab is nx cells with ny = nz = 1 and
 * dy = dz = INFINITY.  material[(k*ny + j)*nx + i] < n_materials. */
typedef struct mcdc_mesh {
    int32_t nx, ny, nz;
    double x0, y0, z0;          /* low corner (cm) */
    double dx, dy, dz;          /* cell widths (cm) */
    const uint8_t *material;    /* [nz][ny][nx], host pointer */
    int32_t bc[6];              /* -x,+x,-y,+y,-z,+z: MCDC_BC_* */
} mcdc_mesh;

/* Multigroup data.  sigma_s <= sigma_t; transfer rows are P(g -> g') given a
 * scatter in g and must sum to 1 (checked to 1e-9). */
typedef struct mcdc_materials {
    int32_t n_materials, n_groups;   /* 1..255, 1..16 */
    const double *sigma_t;           /* [M][G] 1/cm */
    const double *sigma_s;           /* [M][G] 1/cm */
    const double *transfer;          /* [M][G][G]   */
    const double *speed;             /* [G] cm per time unit, > 0 */
} mcdc_materials;

/* Source: position uniform in the box [lo, hi] (lo == hi on an axis gives a
 * plane or a point), isotropic or a beam along dir, group from group_pdf,
 * birth time uniform in [t0, t1] (t0 == t1: a pulse). */
typedef struct mcdc_source {
    double lo[3], hi[3];
    int32_t kind;                    /* MCDC_SRC_* */
    double dir[3];                   /* unit vector, BEAM only */
    const double *group_pdf;         /* [G], sums to 1 */
    double t0, t1;
} mcdc_source;

/* Time census grid: n_bins > 0 edges[0] < ... < edges[n_bins] (the last edge
 * ends the run: particles alive then are "censused"); n_bins == 0 is steady
 * state (one tally time slot, no census). */
typedef struct mcdc_time_grid {
    int32_t n_bins;
    const double *edges;             /* [n_bins + 1], may be NULL if n_bins == 0 */
} mcdc_time_grid;

/* Run-independent options fixed at create.  Zero means "choose for me". */
typedef struct mcdc_options {
    int32_t precision;          /* MCDC_PREC_*                                    */
    int32_t tally_mode;         /* MCDC_TALLY_*                                   */
    int32_t n_batches;          /* batches for the error estimate (>= 2); 0: auto */
    int32_t block_size;         /* threads per CTA; 0: autotuned                  */
    int32_t bank_per_cta;       /* ignored: each warp parks up to 96 particles    */
    int32_t ctas_per_sm;        /* resident CTAs per SM; 0: autotuned             */
    int32_t warp_aggregate;     /* -1 off, 1 on, 0 auto                           */
    int32_t autotune;           /* 1 (default): when block_size is 0, time candidate
                                   launch shapes (threads per CTA, whole batches per
                                   CTA, warp aggregation) on this problem at create
                                   and keep the fastest; cached per problem shape */
    int32_t overflow_per_cta;   /* split-children stack slots per CTA (shared by its
                                   warps, >= 64 each, <= 256 with the global tally);
                                   0: 1024 per warp with the shared tally, 64 with
                                   the global tally, whose children beyond the
                                   stack spill to device-wide banks drained by
                                   every warp in later passes                    */
    int32_t region_lo[3];       /* cell box [lo, hi) of the scalar tally used for */
    int32_t region_hi[3];       /*   the figure of merit; hi == 0: whole mesh      */
    int32_t estimator;          /* MCDC_EST_* (default track length)              */
    int32_t implicit_capture;   /* 1: survival biasing -- a collision never absorbs;
                                   the weight is multiplied by sigma_s / sigma_t and
                                   the removed part counts as absorbed weight     */
    double weight_cutoff;       /* implicit capture: a weight below this after a
                                   collision is rouletted (default 0.25) ...      */
    double cutoff_survival;     /*   ... surviving with this weight (default 0.5);
                                   need 0 < weight_cutoff < cutoff_survival       */
    int32_t pc_target;          /* population control: 0 off; else every batch runs
                                   as a time-stepped simulation whose census bank
                                   (particles reaching an interior time edge) is
                                   combed to pc_target particles of equal weight.
                                   Needs >= 2 time bins, every source particle
                                   born in the first bin, the global tally, no
                                   weight windows and no per-history records      */
    int32_t flight_sampling;    /* FP32 modes, distance to collision: 0 (default)
                                   carries the optical depth (mean free paths) to
                                   the next collision across surface and census
                                   events and draws it only at births, collisions
                                   and for new split children -- the same
                                   distribution, no random number per flight; 1
                                   samples it afresh every flight as FP64 mode
                                   does, so an FP32 run draws the same random
                                   numbers as its FP64 twin (paired precision
                                   studies).  FP64 mode always samples afresh.   */
    int64_t max_children;       /* weight windows: split children one run may make
                                   (0: 4096 per history, at least 2^27; negative:
                                   no limit).  A split past the
                                   budget makes no child and the parent keeps its
                                   weight (unbiased, counted in splits_dropped):
                                   windows that would split without end cost a
                                   bounded run instead of an endless one        */
    int64_t slice_bytes_max;    /* global tally: a run puts every batch in one
                                   launch, each scoring its own tally slice, when
                                   the slices (batches x bins x 8 bytes in FP64
                                   mode, 4 in the FP32 modes, whose slices are
                                   FP32 and are folded in FP64) fit in this many
                                   bytes (0: 8 GiB; negative: never -- one launch
                                   and one fold per batch into an FP64 tally).
                                   If the slices cannot be allocated the run
                                   falls back to one launch per batch.
                                   Population control always uses slices.       */
    int32_t overflow_tail;      /* global tally with weight windows: stack slots a
                                   warp keeps for new split children once its own
                                   particles (source histories, or a pass's share
                                   of the spilled ones) are used up; the children
                                   beyond go to the device-wide banks, which every
                                   warp shares in the next pass, instead of one
                                   warp working through a large family while the
                                   others have finished (-1: the whole stack;
                                   default 8)                                   */
    int64_t spill_particles;    /* global tally with weight windows: particles each
                                   of the two device-wide spill banks holds; a
                                   child that finds them full is not made (counted
                                   in splits_dropped; 0: 2^26)                   */
} mcdc_options;

/* Event and weight counts of one run (summed over all particles). */
typedef struct mcdc_stats {
    uint64_t histories, segments, collisions, crossings, census;
    uint64_t absorbed, leaked, censused, splits, children;
    uint64_t roulette_killed, roulette_survived;
    double w_source, w_absorbed, w_leaked, w_censused;
    double kernel_ms;           /* device time of the transport kernels      */
    double total_ms;            /* device time of the whole run              */
    int32_t block_size, bank_per_cta, ctas_per_sm, tally_mode, n_batches, warp_aggregate;
                                /* launch shape used: threads per CTA, parked-
                                   particle slots per CTA (warps x 96), CTAs per
                                   SM, MCDC_TALLY_*, batches, warp aggregation  */
    uint64_t splits_dropped;    /* weight-window children not made because the warp
                                   stack and the spill bank were full: the parent
                                   kept their weight (unbiased, less variance
                                   reduction)                                   */
    uint64_t pc_combs, pc_in, pc_out;   /* population control: combs, particles
                                           into and out of them             */
    double w_pc_in, w_pc_out;           /* weight into and out of the combs */
} mcdc_stats;

/* Per-history summary of the primary particle (serial 0), for checking a run
 * history by history against a reference tracker. */
typedef struct mcdc_record {
    uint64_t hid;
    int32_t end;                /* 1 absorbed, 2 leaked, 3 censused, 4 rouletted */
    int32_t g;
    uint32_t ctr;               /* random-number counter after the last draw    */
    uint32_t n_seg, n_col, n_cross;
    double x, y, z, t, w;
} mcdc_record;

typedef struct mcdc_run_args {
    uint64_t n_histories;       /* > 0                                            */
    int32_t n_batches;          /* >= 2 and <= n_histories; 0: the create option, else auto */
    uint64_t seed;              /* Philox key                                     */
    uint64_t hist_offset;       /* histories [offset, offset + n) are run         */
    double *mean_out;           /* [n_bins] or NULL; host or device               */
    double *relerr_out;         /* [n_bins] or NULL; host or device               */
    double *sum1_out;           /* [n_bins] sum over batches of batch sums, or NULL;
                                   combined estimator: [2][n_bins], track length then
                                   collision                                      */
    double *sum2_out;           /* [n_bins] sum of squared batch sums, or NULL (combined:
                                   [2][n_bins])                                   */
    double *scalar_out;         /* [2] region scalar mean and relative error, or NULL (host) */
    mcdc_record *records;       /* [n_records] for histories offset..offset+n_records-1, or NULL (host or device) */
    uint64_t n_records;
    void *stream;               /* cudaStream_t; NULL: the legacy default stream  */
    /* combined estimator only (ignored otherwise); host or device, or NULL: */
    double *sum12_out;          /* [n_bins] sum over batches of (track-length batch sum x
                                   collision batch sum)                           */
    double *parts_out;          /* [5][n_bins] track-length mean, its relative error,
                                   collision mean, its relative error, coefficient a */
    double *scalar_parts_out;   /* [5] the same five for the region scalar (host)  */
} mcdc_run_args;

/* Fills *opt with defaults (FP32 split, automatic tally mode, autotuning on). */
void mcdc_default_options(mcdc_options *opt);

/* Validates the problem, builds its device tables (group-transfer CDFs,
 * FP32 copies), uploads them once and picks launch shapes.  A steady-state
 * problem whose bounded faces all reflect must absorb in every material and
 * group (0 <= sigma_s < sigma_t), else a history could run forever.  Errors:
 * MCDC_ERR_INVALID (bad sizes, negative or NaN data, sigma_s > sigma_t,
 * rows not summing to 1, source outside the mesh or before the first time
 * edge), MCDC_ERR_NO_DEVICE, MCDC_ERR_OOM, MCDC_ERR_CUDA.  On error *out is
 * NULL and nothing is leaked. */
int mcdc_problem_create(const mcdc_mesh *mesh, const mcdc_materials *mat,
                        const mcdc_source *src, const mcdc_time_grid *time,
                        const mcdc_options *opt, struct mcdc_problem **out);

/* Runs histories [0, n_histories) with the given seed and writes the mean
 * tally (layout above) to tally_out (host or device, may be NULL).  Blocks
 * until the result is complete. */
int mcdc_run(struct mcdc_problem *prob, uint64_t n_histories, uint64_t seed,
             double *tally_out);

/* Full form: history offset, error estimate, raw batch moments, region
 * scalar, per-history records, event statistics and a caller stream.  With a
 * non-NULL stream and only device outputs it returns once the work is queued
 * (stats->kernel_ms and total_ms are then 0); otherwise it synchronises. */
int mcdc_run_ex(struct mcdc_problem *prob, const mcdc_run_args *args, mcdc_stats *stats);

/* Weight windows: w_lower[cell][G][T] (double, host or device; <= 0 turns the
 * window off in that bin), w_U = upper_ratio*w_L, w_S = survival_ratio*w_L,
 * at most nmax copies per split.  NULL w_lower switches back to analog.
 * Errors: MCDC_ERR_INVALID for ratios that are not 1 < survival < upper or
 * nmax < 2. */
int mcdc_set_weight_windows(struct mcdc_problem *prob, const double *w_lower,
                            double upper_ratio, double survival_ratio, int32_t nmax);

/* Number of tally bins (cells * G * T). */
int64_t mcdc_tally_size(const struct mcdc_problem *prob);

void mcdc_problem_destroy(struct mcdc_problem *prob);

/* Many independent problems in one run: per batch, one persistent launch in
 * which CTAs claim (problem, history range) work items, largest first, and
 * load a problem's tables (its window table included) when they switch to
 * it; then one fused fold of every problem's batch tally; the whole run is
 * one CUDA graph, captured once per run shape and replayed.  All problems
 * must share device, precision and dimension and have no per-event network
 * windows, implicit capture, population control or combined estimator.
 * Table windows (mcdc_set_weight_windows) are applied per problem; a warp
 * keeps the split children of the work item it serves in a stack of 1024
 * (there is no spill bank here: a child that finds the stack full is not
 * made, counted in splits_dropped -- unbiased), within a children budget of
 * max(2^27, 4096 x all histories) per call.
 * Problem i uses seed + i * 0x9E3779B97F4A7C15 (mod 2^64) and
 * histories [0, n_histories[i]) in n_batches batches (0: 16).
 * mean_out[i] / relerr_out[i]: [n_bins of problem i], host or device, or
 * NULL; scalar_out: [2n] region mean and relative error, or NULL.
 * (The paper runs one problem per process; this batching has no paper
 * counterpart beyond its fixed-source loop.) */
int mcdc_run_batched(struct mcdc_problem *const *probs, int32_t n, const uint64_t *n_histories,
                     uint64_t seed, int32_t n_batches, double *const *mean_out,
                     double *const *relerr_out, double *scalar_out, mcdc_stats *stats);

/* ---- learned importance proposal ----------------------------------------
 * A 3-layer perceptron (4 + G) -> 64 -> 64 -> 1 with SiLU hidden layers maps
 * a tally bin (cell centre and bin-centre time scaled to [-1, 1], group
 * one-hot) to the log of its forward flux.  It is fit on the GPU (BF16
 * tensor-core forward/backward, FP32 master weights, Adam) to the log mean of
 * a pilot run, each bin weighted 1 / (1 + relerr^2), unscored bins left out;
 * then every bin's weight-window lower bound is set to
 * source_wl * phi_pred(bin) / max phi_pred (bounded below, see min_ratio), so
 * particles split on their way
 * into low-flux regions and are rouletted coming back.  The paper has no such
 * network; the weight windows it drives are the variance-reduction events of
 * "MC/DC on CPUs". */
typedef struct mcdc_mlp_options {
    int32_t epochs;             /* passes over the bins (default 40)             */
    int32_t batch;              /* samples per Adam step (default 65536, >= 64)  */
    double lr;                  /* Adam step size (default 2e-3)                 */
    uint64_t seed;              /* weight initialisation                          */
    double source_wl;           /* w_L of the highest-flux bin (default 0.5)     */
    double upper_ratio;         /* w_U / w_L (default 5)                         */
    double survival_ratio;      /* w_S / w_L (default 2.5)                       */
    int32_t nmax;               /* split cap (default 16)                        */
    double min_ratio;           /* floor of w_L / w_L(highest-flux bin) (default 1e-8);
                                   w_L is also kept above a tenth of the least-scored
                                   bin's value, so extrapolated windows cannot run away */
    int32_t time_resolved;      /* 0 (default): windows do not depend on the time
                                   bin (the largest over the bins); 1: one per bin.
                                   Per-time windows are tiny where few particles
                                   arrive early (deep cells, first time bins), and
                                   those few then split again and again          */
    int32_t group_resolved;     /* 0 (default): windows do not depend on the group
                                   (the largest over the groups); 1: one per group.
                                   Flux = density x speed, so per-group windows are
                                   low for slow groups, whose particles then split
                                   heavily while hardly moving                   */
    int32_t adjoint;            /* 0 (default): the pilot is a forward flux and
                                   w_L ~ predicted flux (uniform particle density);
                                   1: the pilot is an importance (e.g. the flux of
                                   a run whose source is the tally region, the
                                   adjoint by reciprocity when cross sections do not
                                   depend on the group) and w_L = source_wl x
                                   I(source cells) / I -- particles split on their
                                   way to the region and are rouletted away from it;
                                   time and group folds then keep the smallest w_L */
    int32_t per_event;          /* 0 (default): bake a table of windows; 1: no table --
                                   every window check evaluates a network at the
                                   particle (mcdc_set_network_windows).  With the
                                   time and group folds above (the defaults) the
                                   baked table depends on the cell alone, and a
                                   network of the position (3 inputs) is fitted to
                                   its log, one sample per cell centre: windows
                                   continuous in position, folded like the table.
                                   With time_resolved or group_resolved set, the
                                   trained network itself with the bake's
                                   constants (resolved in time and group).  Needs a
                                   forward pilot (adjoint 0) and the global tally   */
    int32_t distill_steps;      /* Adam steps of that position network, the step
                                   size falling from lr to lr / 20 (0: 8000)     */
    int32_t distill_hidden;     /* its hidden width, 1..64 (0: 16; the FP32 modes
                                   evaluate 16, 32 or 64 units, zero-padded)     */
} mcdc_mlp_options;

typedef struct mcdc_mlp_report {
    int64_t samples;            /* scored bins used for training                 */
    double loss_first, loss_last;   /* mean minibatch loss, first and last epoch (normalised targets) */
    double train_ms, bake_ms;   /* device time of training and of the bake       */
    int32_t steps;              /* Adam steps                                    */
    double target_mean;         /* weighted mean of the log-flux targets         */
    int32_t distill_steps;      /* per-event windows of a cell-only table: Adam
                                   steps of the position network fitted to it
                                   (0 otherwise)                                 */
    double distill_loss;        /* its mean minibatch loss in the last epoch
                                   (targets normalised to unit variance)         */
} mcdc_mlp_report;

void mcdc_default_mlp_options(mcdc_mlp_options *opt);

/* Trains the network on a pilot tally (pilot_mean required, pilot_relerr may
 * be NULL; [n_bins] doubles, host or device) and switches the problem to the
 * weight windows it predicts (a baked table, or the network per event).
 * Errors: MCDC_ERR_INVALID (no scored bin, more than 12 groups, bad options,
 * per_event with an adjoint pilot or a shared tally), MCDC_ERR_OOM,
 * MCDC_ERR_CUDA. */
int mcdc_train_importance(struct mcdc_problem *prob, const double *pilot_mean,
                          const double *pilot_relerr, const mcdc_mlp_options *opt,
                          mcdc_mlp_report *report);

/* Parameter count of the network for n_in inputs (1..16), -1 otherwise.
 * Flat FP32 layout: W1[64][n_in], b1[64], W2[64][64], b2[64], W3[64], b3. */
int64_t mcdc_mlp_param_count(int32_t n_in);

/* Prediction f(X[i]) for n samples (FP32 inputs [n][n_in]; pointers host or
 * device), on the tensor cores with BF16 weights and FP32 accumulation. */
int mcdc_mlp_forward(const float *params, int32_t n_in, const float *X, int64_t n, float *out);

/* Weighted least-squares loss sum_i w_i (f(X_i) - y_i)^2 / sum_i w_i and its
 * gradient with respect to every parameter (same layout as params). */
int mcdc_mlp_loss_grad(const float *params, int32_t n_in, const float *X, const float *y,
                       const float *w, int64_t n, float *grad, double *loss);

/* Trains the network on n given samples with the library's training kernel
 * (the one mcdc_train_importance runs): `epochs` passes of Adam (Kingma &
 * Ba; step lr, b1 0.9, b2 0.999, eps 1e-8, FP32 master weights and moments)
 * over minibatches of `batch` consecutive samples (the last one shorter),
 * each minibatch's loss and gradient as in mcdc_mlp_loss_grad; the whole
 * fit is one launch whose gradient sums have a fixed order, so it is
 * reproducible bit for bit.  params (FP32, host or device, the layout of
 * mcdc_mlp_forward) holds the starting parameters and receives the result;
 * X [n][n_in], y [n], w [n] (FP32, host or device) are copied.  loss_first,
 * loss_last (optional): the mean minibatch loss of the first and the last
 * epoch.  Errors: MCDC_ERR_INVALID (n_in outside 1..16, n < 1 or >= 2^31,
 * epochs < 1, batch < 64, lr <= 0, a minibatch whose weights sum to zero),
 * MCDC_ERR_TIMEOUT, MCDC_ERR_OOM, MCDC_ERR_CUDA.  The network has no
 * counterpart in the paper (the learned importance proposal is this
 * library's own). */
int mcdc_mlp_train(float *params, int32_t n_in, const float *X, const float *y, const float *w,
                   int64_t n, int32_t epochs, int32_t batch, double lr, double *loss_first,
                   double *loss_last);

/* Tries of the bounded waits on tensor-core completion inside the network's
 * kernels (default 4194304; a negative value restores it).  A wait that runs
 * out makes the kernel stop, await its work in flight, free its tensor
 * memory and return; the call (mcdc_mlp_forward, mcdc_mlp_loss_grad,
 * mcdc_train_importance) then fails with MCDC_ERR_TIMEOUT and the context
 * stays usable.  With 0 every wait gives up at once: a way to exercise that
 * failure path. */
int mcdc_set_wait_limit(int32_t tries);

/* Allocation-free run (the paper has no counterpart: this exists for
 * callers that cannot call cudaMalloc while transport runs, e.g. a code
 * whose pool allocator owns all device memory, or a loop where an
 * allocation would stall the device).  The problem must come from
 * mcdc_problem_create, made once at set-up.  The caller passes device
 * buffers sum1, sum2 [n_bins] (batch sums and sums of squares, as in
 * mcdc_run_args) and optionally mean, relerr [n_bins]; the work is queued on
 * `stream` (NULL: legacy default stream) and the call returns without
 * waiting.  Scratch (claim counters, global-mode batch tally, accumulators,
 * event counters) lives in one fixed __device__ array of about 1.1 MiB that
 * every GPU loading the library holds until exit; no cudaMalloc or cudaFree
 * is called.  Limits: n_batches <= 4096 and, for a problem using the global
 * tally, at most 131072 bins; larger requests, and problems with the combined
 * estimator, return MCDC_ERR_INVALID.  The
 * first call on a device looks up the array's device address, so make that
 * first call before any stream capture.  Calls share the array: each clears
 * what must start at zero, and calls that overlap on the GPU race.  Event
 * statistics, records and overflow errors are not reported.  Weight windows:
 * split children come from the same per-run budget as in mcdc_run_ex
 * (options.max_children), so a window map that would split without end
 * still ends; a child that finds its warp's stack full is not made (its
 * parent keeps the weight, which keeps the estimate unbiased).  mcdc_run_ex
 * spills such children to device-wide banks it allocates, so in the global
 * tally mode (64 stack slots per warp) a run that fills a stack differs from
 * mcdc_run_ex's; in the shared mode (1024 slots) they agree unless a stack
 * fills there too. */
int mcdc_run_noalloc(struct mcdc_problem *prob, uint64_t n_histories, uint64_t seed,
                     uint64_t hist_offset, int32_t n_batches, double *sum1, double *sum2,
                     double *mean, double *relerr, void *stream);

/* Measures the FP64 pipe of the current device (no problem needed): the
 * rate of FP64 adds (fused multiply-adds) and of FP32<->FP64 conversions, in
 * lane-operations per second, from two short kernels (8 independent chains
 * per thread, one 512-thread CTA per SM, best of three timed launches; about
 * 10 ms in all).  These are the operations an FP32-split flight spends on its
 * FP64 position and time, so the rates are the measured ceiling of that
 * mode's roofline.  Allocates and frees a small device buffer.  Errors:
 * MCDC_ERR_NO_DEVICE, MCDC_ERR_CUDA, MCDC_ERR_INVALID (NULL output). */
int mcdc_measure_fp64_pipe(double *add_per_s, double *cvt_per_s);

/* The generator of every random number of a run: out[4 i .. 4 i + 3] =
 * Philox4x32-10 (Salmon et al., SC'11; 10 rounds, the published multipliers
 * and Weyl constants) of the counter ctr[4 i .. 4 i + 3] under the key (seed
 * low 32 bits, seed high 32 bits), computed on the current device by the
 * tracker's own routine.  A transport draw uses the counter (event counter,
 * particle serial, history id low, history id high).  ctr and out: n x 4
 * words, host or device, caller-owned.  Errors: MCDC_ERR_INVALID (n < 0 or
 * NULL buffers), MCDC_ERR_NO_DEVICE, MCDC_ERR_OOM, MCDC_ERR_CUDA. */
int mcdc_philox(uint64_t seed, const uint32_t *ctr, int64_t n, uint32_t *out);

/* Per-event weight windows: instead of a table, every window check evaluates
 * the importance network (the layout of mcdc_mlp_forward with `hidden` units
 * per layer, 1..64) at the particle itself.  Inputs (n_in of them): position
 * scaled to [-1, 1] over each bounded mesh axis (0 on an unbounded one); with
 * n_in = 4 + G also time as 2 (j + (t - t_j) / (t_j+1 - t_j)) / T - 1 in time
 * bin j (0 in steady state) and the group one-hot -- the continuous versions
 * of the cell and bin centres a network is trained on; with n_in = 3 the
 * position alone.  With its output y the lower bound
 * is w_L = source_wl exp(min(0, max(y scale + shift, floor_lp) - top)); upper
 * and survival bounds and the split cap as in mcdc_set_weight_windows.
 * params: FP32, host or device, copied (FP64 mode evaluates in FP64 from the
 * same values, one check at a time; the FP32 modes evaluate the checks of a
 * warp together on the tensor cores, binary16 operands, FP32 accumulation);
 * NULL turns windows off.  Replaces any table.  Needs the global tally mode
 * (the other kernels are built without the evaluation).
 * Errors: MCDC_ERR_INVALID (sizes, ratios, non-finite values, population
 * control, a shared-tally problem). */
int mcdc_set_network_windows(struct mcdc_problem *prob, const float *params, int32_t n_in,
                             int32_t hidden, double shift, double scale, double top,
                             double floor_lp, double source_wl, double upper_ratio,
                             double survival_ratio, int32_t nmax);

/* The lower bounds of the last window table: set by mcdc_set_weight_windows
 * or baked by mcdc_train_importance (also the table a per-event position
 * network was fitted to), [n_bins] doubles in the tally's bin layout into
 * w_lower (host or device, caller-owned); blocks until copied.
 * Errors: MCDC_ERR_INVALID (NULL arguments, no table yet), MCDC_ERR_CUDA. */
int mcdc_get_weight_windows(const struct mcdc_problem *prob, double *w_lower);

/* The lower bounds w_L that the window checks of the network set by
 * mcdc_set_network_windows apply to particles in n given states: position
 * x[3 i .. 3 i + 2], time t[i], group g[i].  Each state becomes a particle in
 * the problem's own representation (the cell holding the position, clamped
 * into the mesh; in MCDC_PREC_FP32_LOCAL the FP32 offsets from the cell's low
 * faces and the time left to the next census edge) and goes through the
 * tracker's own evaluation: FP64 mode one state at a time in FP64, the FP32
 * modes 32 at a time on the tensor cores.  A group outside 0..G-1 gives NaN.
 * x, t, g, w_lower: host or device, caller-owned; blocks until done.
 * Errors: MCDC_ERR_INVALID (no network set, n < 0, NULL arrays),
 * MCDC_ERR_OOM, MCDC_ERR_CUDA. */
int mcdc_network_window_lower(struct mcdc_problem *prob, const double *x, const double *t,
                              const int32_t *g, int64_t n, double *w_lower);

/* The checked build.  Compiled with -DMCDC_CHECKS into libmcdc_b300_checks.so
 * (the same entry points), every tracker and comb kernel compares each index
 * it computes into a table (cell, material, group, time bin, window bin), a
 * tally (shared, step or global slices), a warp's particle pool or stack of
 * split children, an input bank or the comb's output with the extent of what
 * it indexes, before the access.  A bad index skips the access (its particle
 * or copy is lost) and the call that ran the kernel returns MCDC_ERR_CHECK,
 * mcdc_last_error naming the first failing site and its index.  Returns 1 in
 * the checked build, 0 in the normal one (which has no checks: its kernels
 * are compiled without them).  mcdc_run_noalloc reports no device errors,
 * checks included. */
int mcdc_build_checked(void);

/* Self-test of the checks: one warp indexes a 16-entry shared array at its
 * lane number (half of the lanes beyond the end), each access behind its
 * check and also behind an explicit bound, so no build accesses out of
 * bounds.  words[0..4] receives the kernel's error words (flags, site, index
 * low word, index high word) and the number of accesses made (16): in the
 * checked build flag 4, site 12 (the self-test) and an index in 16..31; in
 * the normal build zeros.  words: 5 host words, caller-owned.
 * Errors: MCDC_ERR_INVALID (NULL), MCDC_ERR_NO_DEVICE, MCDC_ERR_OOM, MCDC_ERR_CUDA. */
int mcdc_check_selftest(int32_t *words);

/* Message of the last error on the calling thread ("" if none). */
const char *mcdc_last_error(void);

#ifdef __cplusplus
}
#endif
#endif
