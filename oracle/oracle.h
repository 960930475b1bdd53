/*
 * oracle.h -- plain, slow, FP64 CPU oracle for time-dependent multigroup
 * fixed-source Monte Carlo neutron transport (track-length flux tally).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may include, link,
 * load or execute this code: only the tests, the smoke check and the CPU
 * baseline leg of the benchmark use it.  It shares no code, header, table or
 * constant generator with the CUDA library.
 *
 * What it follows (the paper gives prose, two listings and no equations):
 *  - "MC/DC on CPUs": a fixed-source run loops over particles and transports
 *    each one until its history ends by a physical event (capture, time or
 *    space boundary), a simulation event (time census) or a variance
 *    reduction event.
 *  - Figure "jitfunctions" (move_particle): the particle record holds
 *    x, y, z, ux, uy, uz and speed v; a move of length d advances the
 *    position by u*d and the time by d/v.
 *  - Figure "forcpuvgpu": a tally bin index is found from the particle's
 *    location (loc2index) and the score is added to that bin.
 *  - "Monte Carlo Neutron Transport and MC/DC": hash-based random numbers
 *    make a run replicable history by history.
 * Everything else (sampling laws, the counter-based generator, event order,
 * tie rules, normalisation, batch statistics, weight windows) is the
 * textbook analog Monte Carlo loop (Lewis & Miller, cited in that section)
 * in the readings listed at the top of each function.
 */
#ifndef MCDC_ORACLE_H
#define MCDC_ORACLE_H
#include <stdint.h>

enum { ORC_BC_VACUUM = 0, ORC_BC_REFLECT = 1 };
enum { ORC_SRC_ISOTROPIC = 0, ORC_SRC_BEAM = 1 };
enum { ORC_EV_COLLISION = 0, ORC_EV_SURFACE = 1, ORC_EV_CENSUS = 2 };
enum { ORC_END_ABSORBED = 1, ORC_END_LEAKED = 2, ORC_END_CENSUSED = 3,
       ORC_END_ROULETTE = 4 };
enum { ORC_EST_TRACK = 0, ORC_EST_COLLISION = 1, ORC_EST_COMBINED = 2 };

/* One problem: mesh, materials, source, time grid, optional weight windows. */
typedef struct {
    int32_t n[3];          /* cells along x, y, z                                */
    double origin[3];      /* low corner                                         */
    double width[3];       /* cell width; an axis with n==1 and width<=0 or inf
                              is unbounded (no faces), e.g. y and z of a slab    */
    const uint8_t *material;   /* [nz][ny][nx] material id                       */
    int32_t bc[6];         /* -x,+x,-y,+y,-z,+z : ORC_BC_*                       */

    int32_t n_mat, n_grp;
    const double *sigma_t;     /* [M][G] total cross section (1/cm)              */
    const double *sigma_s;     /* [M][G] total scattering cross section          */
    const double *transfer;    /* [M][G][G] P(g -> g') given a scatter in g      */
    const double *speed;       /* [G] particle speed                             */

    double src_lo[3], src_hi[3];   /* uniform box                                */
    int32_t src_kind;              /* ORC_SRC_*                                  */
    double src_dir[3];             /* beam direction (unit)                      */
    const double *src_pdf;         /* [G] source group probabilities             */
    double src_t0, src_t1;         /* birth time uniform in [t0, t1]             */

    int32_t n_tbin;            /* T; 0 = steady state                            */
    const double *edges;       /* [T+1] time-bin edges (census times)            */

    const double *ww_lower;    /* [cells][G][max(T,1)] or NULL (analog)          */
    double ww_upper_ratio;     /* w_U = ratio * w_L                              */
    double ww_survival_ratio;  /* w_S = ratio * w_L                              */
    int32_t ww_nmax;           /* split cap                                      */

    /* R15: per-event windows from the importance network instead of a table */
    const double *ww_net;      /* network parameters (mlp.c layout), or NULL      */
    int32_t ww_net_in, ww_net_h;   /* inputs (4 + G) and hidden width            */
    double ww_net_shift, ww_net_scale; /* log importance = output * scale + shift */
    double ww_net_top, ww_net_floor, ww_net_wl0;  /* w_L = wl0 exp(min(0,
                                  max(log importance, floor) - top))            */

    int32_t region_lo[3], region_hi[3];  /* cell box of the scalar tally [lo,hi) */

    int32_t estimator;         /* ORC_EST_TRACK, ORC_EST_COLLISION or ORC_EST_COMBINED */
    int32_t implicit_capture;  /* 1: survival biasing at collisions              */
    double weight_cutoff;      /* implicit capture: roulette below this weight   */
    double cutoff_survival;    /*   ... surviving with this weight               */

    int32_t pc_target;         /* population control: particles per batch after
                                  each comb at an interior census edge; 0 = off */
} orc_problem;

typedef struct {
    uint64_t histories, segments, collisions, crossings, census;
    uint64_t absorbed, leaked, censused, splits, children;
    uint64_t roulette_killed, roulette_survived;
    double w_source, w_absorbed, w_leaked, w_censused;
    uint64_t pc_combs, pc_in, pc_out;      /* combs, particles in, particles out */
    double w_pc_in, w_pc_out;              /* weight into and out of the combs   */
} orc_counts;

/* Summary of one primary particle (serial 0) of one history. */
typedef struct {
    uint64_t hid;
    int32_t end;        /* ORC_END_* */
    int32_t g;
    uint32_t ctr;       /* counter value after the last draw */
    uint32_t n_seg;
    uint32_t n_col;
    uint32_t n_cross;
    double x, y, z, t, w;
} orc_record;

/* The comb of population control: n particles of weights w (in their bank
 * order) -> M teeth at (k + xi) W / M, W = sum w; sel[k] = the particle whose
 * cumulative-weight interval [S_i, S_i + w_i) holds tooth k. */
void orc_comb(int64_t n, const double *w, int64_t M, double xi, int64_t *sel);

/* Philox4x32-10 block (Salmon, Moraes, Dror, Shaw, SC'11). */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);
/* Two 32-bit words -> double in (0, 1]. */
double orc_uniform(uint32_t hi, uint32_t lo);
/* (xi_mu, xi_phi) -> isotropic unit vector. */
void orc_isotropic(double xi_mu, double xi_phi, double u[3]);

/* Full run: histories [offset, offset+n) split into n_batches contiguous
 * batches; mean/relerr are [cells][G][max(T,1)]; scalar = {mean, relerr} of
 * the region sum.  With ORC_EST_COMBINED, sum1/sum2 hold [2][bins] (track
 * length, then collision), sum12 [bins] the sums over batches of the product
 * of the two batch sums, mean/relerr/scalar the combined estimate (R14) and
 * scalar[2] the region's coefficient a; otherwise sum12 and scalar[2] are not
 * written.  Returns 0, or a negative value on invalid
 * input. */
int orc_run(const orc_problem *p, uint64_t n_hist, uint64_t seed,
            uint64_t offset, int32_t n_batches, int32_t n_threads,
            double *mean, double *relerr, double *sum1, double *sum2, double *sum12,
            double *scalar, orc_counts *counts);

/* R14: minimum-variance combination of two correlated batch series for n
 * bins, from their batch sums s1, squared batch sums s2 and summed products
 * s12 over B batches of n_hist histories, normalised by volume; any of mean,
 * rel, alpha may be NULL. */
void orc_combine(int64_t n, const double *s1x, const double *s2x, const double *s1y,
                 const double *s2y, const double *s12, uint64_t n_hist, int32_t B,
                 double vol, double *mean, double *rel, double *alpha);

/* Test hook: RNG-injection quadrature of collision-order-resolved track
 * lengths (a product rule over chosen draw slots; see transport.c). */
int orc_inject_grid(const orc_problem *p, int32_t n_slots, const double *fixed, int32_t n_dims,
                    const int32_t *dim_slot, const int32_t *dim_m, const double *nodes,
                    const double *weights, int32_t max_order, int32_t threads, double *out);

/* Replays the listed histories one by one and summarises each primary. */
int orc_trace(const orc_problem *p, uint64_t seed, const uint64_t *hids,
              int64_t n, orc_record *out);

/* Importance network (mlp.c): in -> H -> H -> 1, SiLU hidden layers.
 * bf16 = 1 rounds every operand of the matrix products to BF16 (the
 * precision fixed for the network: BF16 weights, FP32 accumulation). */
int64_t orc_mlp_param_count(int32_t in, int32_t H);
void orc_mlp_forward(int32_t in, int32_t H, int32_t bf16, const double *p, int64_t n,
                     const double *X, double *out);
/* R15: the network's inputs for a particle at (x, y, z, t) in time bin tbin
 * (a network of ww_net_in = 3 inputs takes the position alone)
 * and group g (see transport.c). */
void orc_net_features(const orc_problem *p, double x, double y, double z, double t,
                      int32_t tbin, int32_t g, double *f);
double orc_mlp_loss_grad(int32_t in, int32_t H, int32_t bf16, const double *p, int64_t n,
                         const double *X, const double *y, const double *w, double *grad);
/* Test tolerance: first-order bounds of the rounding error of a BF16-operand,
 * FP32-accumulation evaluation, per output and per gradient element. */
void orc_mlp_error_bounds(int32_t in, int32_t H, const double *p, int64_t n, const double *X,
                          const double *y, const double *w, double *f_bound, double *g_bound,
                          double *loss_bound, double *g_abssum, double *g_absmax);
/* First-order bound of the warp-batched window evaluation's error per sample:
 * inputs with absolute error x_abs, operands rounded with unit roundoff u,
 * FP32 sums, activations h + h tanh(h) with tanh within eps_t (mlp.c). */
void orc_mlp_window_bound(int32_t in, int32_t H, const double *p, int64_t n, const double *X,
                          double u, double eps_t, double x_abs, double *f_bound);
void orc_adam_step(int64_t np, double *p, double *m, double *v, const double *g, double lr,
                   double b1, double b2, double eps, int64_t t);
/* Adam over minibatches of consecutive samples, `epochs` passes (mlp.c). */
void orc_mlp_train(int32_t in, int32_t H, int32_t bf16, double *p, int64_t n, const double *X,
                   const double *y, const double *w, int32_t epochs, int32_t batch, double lr,
                   double *loss_first, double *loss_last);

#endif
