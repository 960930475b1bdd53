/*
 * transport.c -- oracle particle tracker, FP64, one history at a time.
 * TEST INFRASTRUCTURE ONLY (see oracle.h).
 *
 * Readings of the paper used here (it states the loop in prose only):
 *  R1 random numbers: block = Philox4x32-10(key = seed, counter = (event
 *     counter, particle serial, history id low, history id high)); one
 *     double in (0,1] from words (0,1), a second from words (2,3).
 *  R2 draws: source uses counters 0..3 (x,y | z,group | mu,phi | t); each
 *     flight uses one block (distance to collision); a collision uses two
 *     blocks (absorb-or-scatter, new group | mu, phi); a roulette one.
 *  R3 the distance to collision is sampled afresh at every flight (the
 *     exponential law is memoryless), so every flight is the same step.
 *  R4 event = nearest of collision, mesh surface, time census; exact ties
 *     go census first, then surface, then collision; among axes the lowest
 *     index wins.
 *  R5 a census at the last time edge ends the history ("censused"); the
 *     time coordinate is set to the edge.
 *  R6 a surface event snaps the crossed coordinate onto the face; leaving
 *     the mesh through a vacuum face ends the history ("leaked"), through a
 *     reflecting face flips that direction cosine.
 *  R7 tally: track length w*d into bin (cell, group, time bin); the output
 *     is the sum over histories divided by (N * cell volume).
 *  R8 batches: histories split into B contiguous batches (the first N%B
 *     batches one history longer); per-bin variance of the mean from the
 *     spread of the batch means.
 *  R10 a flight with nothing ahead (infinite distance) is a leak.
 *  R9 weight windows at collisions and cell crossings: above w_U split into
 *     n = min(ceil(w/w_U), nmax) equal copies, below w_L roulette with
 *     survival probability w/w_S to weight w_S.  Children get a new serial
 *     hashed from (serial, counter, child index) and restart their counter.
 *  R11 collision estimator (optional, replaces R7's score): every collision
 *     scores w / sigma_t into the bin (cell, group, time bin) of the particle
 *     as it arrives, before the collision changes its group; same
 *     normalisation as R7.  Its expectation is the same flux.
 *  R12 implicit capture (optional): a collision never ends the history by
 *     absorption; the weight is multiplied by sigma_s / sigma_t and the
 *     removed part w (1 - sigma_s / sigma_t) is counted as absorbed weight (a
 *     weight that becomes 0, sigma_s = 0, ends the history as absorbed).  The
 *     collision draws the same two blocks as an analog one (the first number
 *     then goes unused).  After the scatter a weight below the cutoff w_c is
 *     rouletted: it survives with probability w / w_s at weight w_s (one more
 *     block), else the history branch ends.  Weight windows, if any, follow.
 *  R13 population control (optional; needs every source particle born in the
 *     first time bin and no weight windows): each batch is one time-stepped
 *     simulation.  Step j transports the batch's bank until every particle
 *     has ended or reached the census edge t_{j+1}; particles at an interior
 *     edge are banked, in the order the step ran them (source order --
 *     history id -- in the first step, tooth order after a comb).  The bank
 *     is combed to M particles of weight W/M (W = the bank's weight): tooth k at
 *     (k + xi) W/M picks the particle whose cumulative-weight interval holds
 *     it, xi = U from the block (key seed; counter 0xFFFFFFFC, j, first
 *     history id of the batch lo, hi).  Tooth k's particle keeps the parent's
 *     state and history id, takes serial = word 0 of the block (key seed;
 *     counter 0xFFFFFFFD, parent serial, j, k) and restarts its counter.
 *     The next step runs the combed bank.
 *  R14 combined estimator (optional): one run scores both R7 and R11 from
 *     the same histories, into two tallies.  Per bin, with batch values x_b
 *     (track length) and y_b (collision), the output is the minimum-variance
 *     linear combination a x + (1 - a) y of the two batch means (the
 *     combination of correlated estimators in Lux & Koblinger, "Monte Carlo
 *     Particle Transport Methods", 1991): a = (s_yy - s_xy) / (s_xx + s_yy -
 *     2 s_xy) from the sample (co)variances of the batch values, a = 1/2 when
 *     that denominator is not positive (the two differ by a constant), then
 *     clipped to [0, 1], and the variance of the mean is that of the
 *     combination at this a divided by B.  (Unclipped, a bin that only one
 *     batch scores has perfectly correlated estimators, and their minimum-
 *     variance combination extrapolates to an estimate of zero with zero
 *     variance; clipped, the estimate stays between the two.)  The region
 *     scalar is combined the same way from its two batch series.
 *  R15 per-event windows (optional, instead of the table of R9): at every
 *     window check the lower bound comes from the importance network
 *     evaluated at the particle itself.  Inputs: position scaled to [-1, 1]
 *     over each bounded axis of the mesh (0 on an unbounded axis), time as
 *     2 (j + (t - t_j) / (t_j+1 - t_j)) / T - 1 in time bin j (0 in steady
 *     state), then the group one-hot -- the continuous versions of the cell
 *     centre and bin centre the network is trained on.  With the output y,
 *     lp = y scale + shift and w_L = wl0 exp(min(0, max(lp, floor) - top));
 *     upper and survival bounds and the split cap as in R9.
 */
#include <math.h>
#include <pthread.h>
#include <stdlib.h>
#include <string.h>
#include "oracle.h"

/* ---- the particle record (Figure "jitfunctions" plus group, weight,
 *      cell, time bin and random-number state) ------------------------ */
typedef struct {
    double x, y, z;        /* position                                     */
    double ux, uy, uz;     /* direction cosines                            */
    double v;              /* speed of the current group                   */
    double t;              /* time                                         */
    double w;              /* statistical weight                           */
    int32_t g;             /* energy group                                 */
    int32_t idx[3];        /* mesh cell (i, j, k)                          */
    int32_t tbin;          /* current time bin                             */
    uint32_t serial;       /* particle id inside the history (0 = primary) */
    uint32_t ctr;          /* event counter of the random stream           */
    uint32_t n_seg, n_col, n_cross;
    uint64_t hid;          /* history the particle belongs to (its stream)  */
} part;

typedef struct {
    const orc_problem *p;
    double *scat_ratio;    /* [M][G] sigma_s / sigma_t                      */
    double *cdf;           /* [M][G][G] cumulative transfer probabilities   */
    double *src_cdf;       /* [G]                                           */
    int bounded[3];
    int64_t n_cells;
    int32_t T1;            /* time slots per (cell, group) = max(T, 1)       */
    int64_t n_bins;
    double volume;
} tables;

typedef struct {
    part *items;
    int64_t size, cap;
} stack;

static void push(stack *s, const part *P)
{
    if (s->size == s->cap) {
        s->cap = s->cap ? 2 * s->cap : 64;
        s->items = (part *)realloc(s->items, (size_t)s->cap * sizeof(part));
    }
    s->items[s->size++] = *P;
}

/* ---- random numbers (R1) ------------------------------------------- */
typedef struct { double a, b; } pair;

/* Test hook (orc_inject_grid only): while g_inj is set on a thread, draws
 * return its numbers in order, two per draw, instead of Philox blocks, and
 * the track length of every segment is also added to g_order[k], k the
 * number of collisions the particle has had; a history ends once it would
 * start a segment of order beyond g_max_order. */
static __thread const double *g_inj = NULL;
static __thread int64_t g_inj_n = 0, g_inj_pos = 0;
static __thread double *g_order = NULL;
static __thread int32_t g_max_order = 0;

static pair draw(uint64_t seed, uint64_t hid, part *P)
{
    if (g_inj) {
        pair r = { 0.5, 0.5 };
        if (g_inj_pos + 2 <= g_inj_n) { r.a = g_inj[g_inj_pos]; r.b = g_inj[g_inj_pos + 1]; }
        g_inj_pos += 2;
        P->ctr += 1;
        return r;
    }
    uint32_t key[2] = { (uint32_t)seed, (uint32_t)(seed >> 32) };
    uint32_t ctr[4] = { P->ctr, P->serial, (uint32_t)hid, (uint32_t)(hid >> 32) };
    uint32_t out[4];
    orc_philox4x32_10(ctr, key, out);
    P->ctr += 1;
    pair r = { orc_uniform(out[0], out[1]), orc_uniform(out[2], out[3]) };
    return r;
}

/* ---- geometry ------------------------------------------------------- */
static int axis_bounded(const orc_problem *p, int a)
{
    return !(p->n[a] == 1 && (!(p->width[a] > 0.0) || isinf(p->width[a])));
}

static double *pos(part *P, int a) { return a == 0 ? &P->x : (a == 1 ? &P->y : &P->z); }
static double *dir(part *P, int a) { return a == 0 ? &P->ux : (a == 1 ? &P->uy : &P->uz); }

/* loc2index (Figure "forcpuvgpu"): cell of a position; clamped so a point
 * on the outer face belongs to the last cell. */
static int32_t loc2index_axis(const orc_problem *p, const tables *tb, int a, double x)
{
    if (!tb->bounded[a]) return 0;
    double f = floor((x - p->origin[a]) / p->width[a]);
    int32_t i = (int32_t)f;
    if (f < 0.0) i = 0;
    if (f > (double)(p->n[a] - 1)) i = p->n[a] - 1;
    return i;
}

static int64_t cell_of(const orc_problem *p, const part *P)
{
    return ((int64_t)P->idx[2] * p->n[1] + P->idx[1]) * p->n[0] + P->idx[0];
}

/* face coordinate of the cell side that a particle moving with sign s meets */
static double face(const orc_problem *p, int a, int32_t i, double u)
{
    int32_t k = (u > 0.0) ? i + 1 : i;
    return p->origin[a] + (double)k * p->width[a];
}

/* ---- move_particle (Figure "jitfunctions") --------------------------- */
static void move_particle(part *P, double distance)
{
    P->x += P->ux * distance;
    P->y += P->uy * distance;
    P->z += P->uz * distance;
    P->t += distance / P->v;
}

/* first k with xi <= cdf[k]; cdf is flat at 1.0 after its last rise */
static int32_t sample_cdf(const double *cdf, int32_t n, double xi)
{
    for (int32_t k = 0; k < n; ++k)
        if (xi <= cdf[k]) return k;
    return n - 1;
}

static void build_cdf(const double *pdf, int32_t n, double *cdf)
{
    double acc = 0.0;
    int32_t last = 0;
    for (int32_t k = 0; k < n; ++k) {
        acc += pdf[k];
        cdf[k] = acc;
        if (pdf[k] > 0.0) last = k;
    }
    for (int32_t k = last; k < n; ++k) cdf[k] = 1.0;
}

/* ---- source (R2: counters 0..3) -------------------------------------- */
static part source_particle(const orc_problem *p, const tables *tb,
                            uint64_t seed, uint64_t hid)
{
    part P;
    memset(&P, 0, sizeof P);
    P.serial = 0;
    P.ctr = 0;
    P.hid = hid;
    pair r0 = draw(seed, hid, &P);   /* x, y        */
    pair r1 = draw(seed, hid, &P);   /* z, group    */
    pair r2 = draw(seed, hid, &P);   /* mu, phi     */
    pair r3 = draw(seed, hid, &P);   /* t           */
    P.x = p->src_lo[0] + r0.a * (p->src_hi[0] - p->src_lo[0]);
    P.y = p->src_lo[1] + r0.b * (p->src_hi[1] - p->src_lo[1]);
    P.z = p->src_lo[2] + r1.a * (p->src_hi[2] - p->src_lo[2]);
    P.g = sample_cdf(tb->src_cdf, p->n_grp, r1.b);
    if (p->src_kind == ORC_SRC_BEAM) {
        P.ux = p->src_dir[0]; P.uy = p->src_dir[1]; P.uz = p->src_dir[2];
    } else {
        double u[3];
        orc_isotropic(r2.a, r2.b, u);
        P.ux = u[0]; P.uy = u[1]; P.uz = u[2];
    }
    P.t = p->src_t0 + r3.a * (p->src_t1 - p->src_t0);
    P.v = p->speed[P.g];
    P.w = 1.0;
    P.idx[0] = loc2index_axis(p, tb, 0, P.x);
    P.idx[1] = loc2index_axis(p, tb, 1, P.y);
    P.idx[2] = loc2index_axis(p, tb, 2, P.z);
    P.tbin = 0;
    if (p->n_tbin > 0)
        while (P.tbin < p->n_tbin && p->edges[P.tbin + 1] <= P.t) P.tbin += 1;
    return P;
}

/* ---- weight windows (R9) ------------------------------------------- */
/* Returns 1 if the particle survives.  Children go on the stack. */
void orc_net_features(const orc_problem *p, double x, double y, double z, double t,
                      int32_t tbin, int32_t g, double *f)
{
    const double pos[3] = { x, y, z };
    for (int a = 0; a < 3; ++a)
        f[a] = axis_bounded(p, a)
                   ? 2.0 * (pos[a] - p->origin[a]) / ((double)p->n[a] * p->width[a]) - 1.0
                   : 0.0;
    if (p->ww_net_in == 3) return;         /* a network over the position alone */
    if (p->n_tbin > 0) {
        int32_t j = tbin < p->n_tbin ? tbin : p->n_tbin - 1;
        double u = (t - p->edges[j]) / (p->edges[j + 1] - p->edges[j]);
        f[3] = 2.0 * ((double)j + u) / (double)p->n_tbin - 1.0;
    } else {
        f[3] = 0.0;
    }
    for (int32_t k = 4; k < p->ww_net_in; ++k) f[k] = (k - 4 == g) ? 1.0 : 0.0;
}

/* R15: the window's lower bound from the network at the particle */
static double net_window(const orc_problem *p, const part *P)
{
    double f[64], out;
    orc_net_features(p, P->x, P->y, P->z, P->t, P->tbin, P->g, f);
    orc_mlp_forward(p->ww_net_in, p->ww_net_h, 0, p->ww_net, 1, f, &out);
    double lp = out * p->ww_net_scale + p->ww_net_shift;
    if (lp < p->ww_net_floor) lp = p->ww_net_floor;
    double e = lp - p->ww_net_top;
    return p->ww_net_wl0 * exp(e < 0.0 ? e : 0.0);
}

static int weight_window(const orc_problem *p, const tables *tb, uint64_t seed,
                         uint64_t hid, part *P, stack *bank, orc_counts *c)
{
    if (p->ww_lower == NULL && p->ww_net == NULL) return 1;
    double wl = p->ww_net != NULL
                    ? net_window(p, P)
                    : p->ww_lower[(cell_of(p, P) * p->n_grp + P->g) * tb->T1
                                  + (p->n_tbin > 0 ? P->tbin : 0)];
    if (!(wl > 0.0)) return 1;
    double wu = p->ww_upper_ratio * wl;
    if (P->w > wu) {
        double nd = ceil(P->w / wu);
        int32_t n = nd > (double)p->ww_nmax ? p->ww_nmax : (int32_t)nd;
        if (n > 1) {
            double wc = P->w / (double)n;
            uint32_t key[2] = { (uint32_t)seed, (uint32_t)(seed >> 32) };
            for (int32_t k = 1; k < n; ++k) {
                uint32_t ctr[4] = { 0xFFFFFFFFu, P->serial, P->ctr, (uint32_t)k };
                uint32_t out[4];
                orc_philox4x32_10(ctr, key, out);
                part C = *P;
                C.w = wc;
                C.serial = out[0];
                C.ctr = 0;
                C.n_seg = C.n_col = C.n_cross = 0;
                push(bank, &C);
            }
            P->w = wc;
            c->splits += 1;
            c->children += (uint64_t)(n - 1);
        }
        return 1;
    }
    if (P->w < wl) {
        double ws = p->ww_survival_ratio * wl;
        pair r = draw(seed, hid, P);
        if (r.a < P->w / ws) {
            P->w = ws;
            c->roulette_survived += 1;
            return 1;
        }
        c->roulette_killed += 1;
        return 0;
    }
    return 1;
}

/* internal return of transport(): reached an interior census edge with
 * population control on (not an end of the history) */
enum { BANKED = 100 };

/* ---- one particle until its history branch ends -------------------- */
static int32_t transport(const orc_problem *p, const tables *tb, uint64_t seed,
                         uint64_t hid, part *P, double *tally, stack *bank,
                         orc_counts *c)
{
    const int32_t G = p->n_grp;
    for (;;) {
        int64_t cell = cell_of(p, P);
        int32_t m = p->material[cell];
        double sig_t = p->sigma_t[m * G + P->g];

        /* distance to collision */
        pair r = draw(seed, hid, P);
        double d_coll = sig_t > 0.0 ? -log(r.a) / sig_t : INFINITY;

        /* distance to the mesh surface: nearest face over bounded axes */
        double d_surf = INFINITY;
        int ax = -1;
        for (int a = 0; a < 3; ++a) {
            double u = *dir(P, a);
            if (!tb->bounded[a] || u == 0.0) continue;
            double d = (face(p, a, P->idx[a], u) - *pos(P, a)) / u;
            if (d < 0.0) d = 0.0;
            if (d < d_surf) { d_surf = d; ax = a; }
        }

        /* distance to the time census */
        double d_time = INFINITY;
        if (p->n_tbin > 0) {
            d_time = P->v * (p->edges[P->tbin + 1] - P->t);
            if (d_time < 0.0) d_time = 0.0;   /* t may sit one ulp past the edge */
        }

        /* nearest event; ties: census, then surface, then collision */
        int ev = ORC_EV_COLLISION;
        double d = d_coll;
        if (d_surf <= d) { d = d_surf; ev = ORC_EV_SURFACE; }
        if (d_time <= d) { d = d_time; ev = ORC_EV_CENSUS; }

        P->n_seg += 1;
        c->segments += 1;
        if (isinf(d)) {
            /* nothing ahead (void, no face in the flight direction, steady
             * state): the particle leaves to infinity */
            c->leaked += 1;
            c->w_leaked += P->w;
            return ORC_END_LEAKED;
        }

        /* track-length tally into (cell, group, time bin) */
        int64_t bin = (cell * G + P->g) * tb->T1 + (p->n_tbin > 0 ? P->tbin : 0);
        if (p->estimator != ORC_EST_COLLISION) tally[bin] += P->w * d;
        if (g_order) g_order[P->n_col] += P->w * d;          /* test hook */

        move_particle(P, d);

        if (ev == ORC_EV_CENSUS) {
            c->census += 1;
            P->t = p->edges[P->tbin + 1];
            P->tbin += 1;
            if (P->tbin == p->n_tbin) {
                c->censused += 1;
                c->w_censused += P->w;
                return ORC_END_CENSUSED;
            }
            if (p->pc_target > 0) return BANKED;     /* R13: wait for the comb */
        } else if (ev == ORC_EV_SURFACE) {
            double u = *dir(P, ax);
            *pos(P, ax) = face(p, ax, P->idx[ax], u);
            int32_t step = u > 0.0 ? 1 : -1;
            int32_t inext = P->idx[ax] + step;
            if (inext < 0 || inext >= p->n[ax]) {
                int side = 2 * ax + (step > 0 ? 1 : 0);
                if (p->bc[side] == ORC_BC_REFLECT) {
                    *dir(P, ax) = -u;
                } else {
                    c->leaked += 1;
                    c->w_leaked += P->w;
                    return ORC_END_LEAKED;
                }
            } else {
                P->idx[ax] = inext;
                P->n_cross += 1;
                c->crossings += 1;
                if (!weight_window(p, tb, seed, hid, P, bank, c)) return ORC_END_ROULETTE;
            }
        } else {
            /* collision: absorb or scatter, new group, new direction */
            P->n_col += 1;
            c->collisions += 1;
            if (g_order && (int32_t)P->n_col > g_max_order) return ORC_END_ABSORBED;  /* test hook */
            if (p->estimator != ORC_EST_TRACK)                                 /* R11, R14 */
                tally[(p->estimator == ORC_EST_COMBINED ? tb->n_bins : 0) + bin] += P->w / sig_t;
            pair r1 = draw(seed, hid, P);
            pair r2 = draw(seed, hid, P);
            double ratio = tb->scat_ratio[m * G + P->g];
            if (p->implicit_capture) {                                         /* R12 */
                c->w_absorbed += P->w * (1.0 - ratio);
                P->w *= ratio;
                if (!(P->w > 0.0)) {
                    c->absorbed += 1;
                    return ORC_END_ABSORBED;
                }
            } else if (!(r1.a < ratio)) {
                c->absorbed += 1;
                c->w_absorbed += P->w;
                return ORC_END_ABSORBED;
            }
            P->g = sample_cdf(tb->cdf + ((int64_t)m * G + P->g) * G, G, r1.b);
            P->v = p->speed[P->g];
            double u[3];
            orc_isotropic(r2.a, r2.b, u);
            P->ux = u[0]; P->uy = u[1]; P->uz = u[2];
            if (p->implicit_capture && P->w < p->weight_cutoff) {
                pair r = draw(seed, hid, P);
                if (r.a < P->w / p->cutoff_survival) {
                    P->w = p->cutoff_survival;
                    c->roulette_survived += 1;
                } else {
                    c->roulette_killed += 1;
                    return ORC_END_ROULETTE;
                }
            }
            if (!weight_window(p, tb, seed, hid, P, bank, c)) return ORC_END_ROULETTE;
        }
    }
}

/* One history: the primary and every child it splits into. */
static void run_history(const orc_problem *p, const tables *tb, uint64_t seed,
                        uint64_t hid, double *tally, orc_counts *c, orc_record *rec)
{
    stack bank = { NULL, 0, 0 };
    part P = source_particle(p, tb, seed, hid);
    c->histories += 1;
    c->w_source += P.w;
    if (p->n_tbin > 0 && P.tbin >= p->n_tbin) {
        /* born after the last census time: censused at birth */
        c->censused += 1;
        c->w_censused += P.w;
        if (rec) {
            rec->hid = hid; rec->end = ORC_END_CENSUSED; rec->g = P.g; rec->ctr = P.ctr;
            rec->n_seg = 0; rec->n_col = 0; rec->n_cross = 0;
            rec->x = P.x; rec->y = P.y; rec->z = P.z; rec->t = P.t; rec->w = P.w;
        }
        return;
    }
    push(&bank, &P);
    int first = 1;
    while (bank.size > 0) {
        part Q = bank.items[--bank.size];
        int32_t end = transport(p, tb, seed, hid, &Q, tally, &bank, c);
        if (first && rec) {
            rec->hid = hid; rec->end = end; rec->g = Q.g; rec->ctr = Q.ctr;
            rec->n_seg = Q.n_seg; rec->n_col = Q.n_col; rec->n_cross = Q.n_cross;
            rec->x = Q.x; rec->y = Q.y; rec->z = Q.z; rec->t = Q.t; rec->w = Q.w;
        }
        first = 0;
    }
    free(bank.items);
}

/* ---- population control (R13) ---------------------------------------- */
void orc_comb(int64_t n, const double *w, int64_t M, double xi, int64_t *sel)
{
    double W = 0.0;
    for (int64_t i = 0; i < n; ++i) W += w[i];
    double S = 0.0;          /* cumulative weight before particle i */
    int64_t i = 0;
    for (int64_t k = 0; k < M; ++k) {
        double tooth = ((double)k + xi) * (W / (double)M);
        while (i < n - 1 && S + w[i] <= tooth) { S += w[i]; ++i; }
        sel[k] = i;
    }
}

/* One batch [h0, h1) as a time-stepped simulation with a comb at every
 * interior census edge.  All source particles are born in the first bin. */
static void run_batch_pc(const orc_problem *p, const tables *tb, uint64_t seed, uint64_t h0,
                         uint64_t h1, double *tally, orc_counts *c)
{
    const int64_t M = p->pc_target;
    int64_t cap = (int64_t)(h1 - h0) > M ? (int64_t)(h1 - h0) : M;
    part *bank = (part *)malloc(sizeof(part) * (size_t)(cap > 0 ? cap : 1));
    part *cen = (part *)malloc(sizeof(part) * (size_t)(cap > 0 ? cap : 1));
    double *w = (double *)malloc(sizeof(double) * (size_t)(cap > 0 ? cap : 1));
    int64_t *sel = (int64_t *)malloc(sizeof(int64_t) * (size_t)(M > 0 ? M : 1));
    int64_t n = 0;
    stack none = { NULL, 0, 0 };      /* weight windows are off: no children */
    for (uint64_t h = h0; h < h1; ++h) {
        part P = source_particle(p, tb, seed, h);
        c->histories += 1;
        c->w_source += P.w;
        bank[n++] = P;
    }
    for (int32_t j = 0; j < p->n_tbin && n > 0; ++j) {
        int64_t nc = 0;
        for (int64_t i = 0; i < n; ++i) {
            part Q = bank[i];
            int32_t end = transport(p, tb, seed, Q.hid, &Q, tally, &none, c);
            if (end == BANKED) cen[nc++] = Q;
        }
        if (nc == 0) break;
        /* the comb, in bank order (the order the step ran its particles),
         * M teeth, new streams */
        uint32_t key[2] = { (uint32_t)seed, (uint32_t)(seed >> 32) };
        uint32_t cx[4] = { 0xFFFFFFFCu, (uint32_t)j, (uint32_t)h0, (uint32_t)(h0 >> 32) };
        uint32_t ox[4];
        orc_philox4x32_10(cx, key, ox);
        double xi = orc_uniform(ox[0], ox[1]);
        double W = 0.0;
        for (int64_t i = 0; i < nc; ++i) { w[i] = cen[i].w; W += cen[i].w; }
        orc_comb(nc, w, M, xi, sel);
        c->pc_combs += 1;
        c->pc_in += (uint64_t)nc;
        c->pc_out += (uint64_t)M;
        c->w_pc_in += W;
        for (int64_t k = 0; k < M; ++k) {
            part Q = cen[sel[k]];
            uint32_t cs[4] = { 0xFFFFFFFDu, Q.serial, (uint32_t)j, (uint32_t)k };
            uint32_t os[4];
            orc_philox4x32_10(cs, key, os);
            Q.serial = os[0];
            Q.ctr = 0;
            Q.w = W / (double)M;
            c->w_pc_out += Q.w;
            bank[k] = Q;
        }
        n = M;
    }
    free(bank); free(cen); free(w); free(sel);
}

/* ---- problem checks and derived tables -------------------------------- */
static int make_tables(const orc_problem *p, tables *tb)
{
    memset(tb, 0, sizeof *tb);
    tb->p = p;
    if (p->n_mat < 1 || p->n_grp < 1 || p->n_tbin < 0) return -1;
    for (int a = 0; a < 3; ++a) {
        if (p->n[a] < 1) return -1;
        tb->bounded[a] = axis_bounded(p, a);
    }
    tb->n_cells = (int64_t)p->n[0] * p->n[1] * p->n[2];
    tb->T1 = p->n_tbin > 0 ? p->n_tbin : 1;
    tb->n_bins = tb->n_cells * p->n_grp * tb->T1;
    tb->volume = 1.0;
    for (int a = 0; a < 3; ++a)
        if (tb->bounded[a]) tb->volume *= p->width[a];
    const int32_t M = p->n_mat, G = p->n_grp;
    tb->scat_ratio = (double *)calloc((size_t)M * G, sizeof(double));
    tb->cdf = (double *)calloc((size_t)M * G * G, sizeof(double));
    tb->src_cdf = (double *)calloc((size_t)G, sizeof(double));
    for (int32_t m = 0; m < M; ++m)
        for (int32_t g = 0; g < G; ++g) {
            double st = p->sigma_t[m * G + g], ss = p->sigma_s[m * G + g];
            if (!(st >= 0.0) || !(ss >= 0.0) || ss > st) return -1;
            tb->scat_ratio[m * G + g] = st > 0.0 ? ss / st : 0.0;
            build_cdf(p->transfer + ((int64_t)m * G + g) * G, G,
                      tb->cdf + ((int64_t)m * G + g) * G);
        }
    build_cdf(p->src_pdf, G, tb->src_cdf);
    if (p->n_tbin > 0 && p->src_t0 < p->edges[0]) return -1;
    if (p->src_t1 < p->src_t0) return -1;
    if (p->estimator != ORC_EST_TRACK && p->estimator != ORC_EST_COLLISION &&
        p->estimator != ORC_EST_COMBINED) return -1;
    if (p->implicit_capture &&
        !(p->weight_cutoff > 0.0 && p->cutoff_survival > p->weight_cutoff)) return -1;
    if (p->pc_target < 0) return -1;
    if (p->pc_target > 0 &&
        (p->n_tbin < 2 || p->ww_lower != NULL || p->ww_net != NULL ||
         !(p->src_t1 < p->edges[1]))) return -1;
    if (p->ww_net != NULL && ((p->ww_net_in != 4 + p->n_grp && p->ww_net_in != 3) ||
                              p->ww_net_in > 64 ||
                              p->ww_net_h < 1)) return -1;
    for (int64_t c = 0; c < tb->n_cells; ++c)
        if (p->material[c] >= M) return -1;
    return 0;
}

static void free_tables(tables *tb)
{
    free(tb->scat_ratio);
    free(tb->cdf);
    free(tb->src_cdf);
}

static int in_region(const orc_problem *p, int64_t cell)
{
    int64_t i = cell % p->n[0];
    int64_t j = (cell / p->n[0]) % p->n[1];
    int64_t k = cell / ((int64_t)p->n[0] * p->n[1]);
    return i >= p->region_lo[0] && i < p->region_hi[0] &&
           j >= p->region_lo[1] && j < p->region_hi[1] &&
           k >= p->region_lo[2] && k < p->region_hi[2];
}

/* ---- batches over threads (R8) ---------------------------------------- */
typedef struct {
    const orc_problem *p;
    const tables *tb;
    uint64_t n, seed, offset;
    int32_t B, nthreads, tid;
    double *s1, *s2;          /* thread partial sums over its batches ([ne n_bins]) */
    double *s12;              /* R14: sums of products track x collision, or NULL */
    double r[5];              /* region scalar partials: s1, s2 (track or the one
                                 estimator), s1, s2 (collision), s12 (R14)      */
    orc_counts c;
} worker;

static uint64_t batch_start(uint64_t n, int32_t B, int32_t b)
{
    uint64_t q = n / (uint64_t)B, r = n % (uint64_t)B;
    uint64_t bb = (uint64_t)b;
    return bb * q + (bb < r ? bb : r);
}

static void *work(void *arg)
{
    worker *wk = (worker *)arg;
    const tables *tb = wk->tb;
    const int64_t nb = tb->n_bins;
    const int ne = wk->p->estimator == ORC_EST_COMBINED ? 2 : 1;
    double *tally = (double *)malloc((size_t)(ne * nb) * sizeof(double));
    for (int32_t b = wk->tid; b < wk->B; b += wk->nthreads) {
        memset(tally, 0, (size_t)(ne * nb) * sizeof(double));
        uint64_t h0 = batch_start(wk->n, wk->B, b), h1 = batch_start(wk->n, wk->B, b + 1);
        if (wk->p->pc_target > 0)
            run_batch_pc(wk->p, tb, wk->seed, wk->offset + h0, wk->offset + h1, tally, &wk->c);
        else
            for (uint64_t h = h0; h < h1; ++h)
                run_history(wk->p, tb, wk->seed, wk->offset + h, tally, &wk->c, NULL);
        double region[2] = {0.0, 0.0};
        for (int e = 0; e < ne; ++e)
            for (int64_t k = 0; k < nb; ++k) {
                double v = tally[e * nb + k];
                wk->s1[e * nb + k] += v;
                wk->s2[e * nb + k] += v * v;
                if (in_region(wk->p, k / ((int64_t)wk->p->n_grp * tb->T1))) region[e] += v;
            }
        if (ne == 2)
            for (int64_t k = 0; k < nb; ++k) wk->s12[k] += tally[k] * tally[nb + k];
        wk->r[0] += region[0];
        wk->r[1] += region[0] * region[0];
        wk->r[2] += region[1];
        wk->r[3] += region[1] * region[1];
        wk->r[4] += region[0] * region[1];
    }
    free(tally);
    return NULL;
}

static void add_counts(orc_counts *a, const orc_counts *b)
{
    a->histories += b->histories; a->segments += b->segments;
    a->collisions += b->collisions; a->crossings += b->crossings;
    a->census += b->census; a->absorbed += b->absorbed; a->leaked += b->leaked;
    a->censused += b->censused; a->splits += b->splits; a->children += b->children;
    a->roulette_killed += b->roulette_killed;
    a->roulette_survived += b->roulette_survived;
    a->w_source += b->w_source; a->w_absorbed += b->w_absorbed;
    a->w_leaked += b->w_leaked; a->w_censused += b->w_censused;
    a->pc_combs += b->pc_combs; a->pc_in += b->pc_in; a->pc_out += b->pc_out;
    a->w_pc_in += b->w_pc_in; a->w_pc_out += b->w_pc_out;
}

/* mean and relative error from batch sums: m_b = B s_b / (N V) */
static void batch_moments(double s1, double s2, uint64_t n, int32_t B, double vol,
                          double *mean, double *rel)
{
    double nv = (double)n * vol;
    double m = s1 / nv;
    double ss = s2 - s1 * s1 / (double)B;
    if (ss < 0.0) ss = 0.0;
    double var = ((double)B * (double)B / (nv * nv)) * ss / ((double)B * (double)(B - 1));
    *mean = m;
    *rel = m != 0.0 ? sqrt(var) / fabs(m) : 0.0;
}

/* R14: minimum-variance combination of two correlated batch series, bin by
 * bin.  Batch values are x_b = B s_b / (N V); from the batch sums the sample
 * moments are mean = sum / B and (co)variance = (sum of products - B mean
 * mean') / (B - 1). */
void orc_combine(int64_t n, const double *s1x, const double *s2x, const double *s1y,
                 const double *s2y, const double *s12, uint64_t n_hist, int32_t B,
                 double vol, double *mean, double *rel, double *alpha)
{
    const double Bd = (double)B, c = Bd / ((double)n_hist * vol);
    for (int64_t k = 0; k < n; ++k) {
        double mx = c * s1x[k] / Bd, my = c * s1y[k] / Bd;
        double sxx = (c * c * s2x[k] - Bd * mx * mx) / (Bd - 1.0);
        double syy = (c * c * s2y[k] - Bd * my * my) / (Bd - 1.0);
        double sxy = (c * c * s12[k] - Bd * mx * my) / (Bd - 1.0);
        double den = sxx + syy - 2.0 * sxy;
        double a = den > 0.0 ? (syy - sxy) / den : 0.5;
        if (a < 0.0) a = 0.0;
        if (a > 1.0) a = 1.0;
        double m = a * mx + (1.0 - a) * my;
        double var = (a * a * sxx + (1.0 - a) * (1.0 - a) * syy + 2.0 * a * (1.0 - a) * sxy) / Bd;
        if (var < 0.0) var = 0.0;
        if (mean) mean[k] = m;
        if (rel) rel[k] = m != 0.0 ? sqrt(var) / fabs(m) : 0.0;
        if (alpha) alpha[k] = a;
    }
}

int orc_run(const orc_problem *p, uint64_t n_hist, uint64_t seed,
            uint64_t offset, int32_t n_batches, int32_t n_threads,
            double *mean, double *relerr, double *sum1, double *sum2, double *sum12,
            double *scalar, orc_counts *counts)
{
    tables tb;
    if (n_batches < 2 || n_hist < (uint64_t)n_batches) return -1;
    if (make_tables(p, &tb) != 0) { free_tables(&tb); return -1; }
    if (n_threads < 1) n_threads = 1;
    if (n_threads > n_batches) n_threads = n_batches;
    const int64_t nb = tb.n_bins;
    const int ne = p->estimator == ORC_EST_COMBINED ? 2 : 1;

    worker *wk = (worker *)calloc((size_t)n_threads, sizeof(worker));
    pthread_t *th = (pthread_t *)calloc((size_t)n_threads, sizeof(pthread_t));
    for (int32_t t = 0; t < n_threads; ++t) {
        wk[t].p = p; wk[t].tb = &tb; wk[t].n = n_hist; wk[t].seed = seed;
        wk[t].offset = offset; wk[t].B = n_batches; wk[t].nthreads = n_threads;
        wk[t].tid = t;
        wk[t].s1 = (double *)calloc((size_t)(ne * nb), sizeof(double));
        wk[t].s2 = (double *)calloc((size_t)(ne * nb), sizeof(double));
        wk[t].s12 = ne == 2 ? (double *)calloc((size_t)nb, sizeof(double)) : NULL;
        pthread_create(&th[t], NULL, work, &wk[t]);
    }
    for (int32_t t = 0; t < n_threads; ++t) pthread_join(th[t], NULL);

    orc_counts c;
    memset(&c, 0, sizeof c);
    double *S1 = (double *)calloc((size_t)(ne * nb), sizeof(double));
    double *S2 = (double *)calloc((size_t)(ne * nb), sizeof(double));
    double *S12 = (double *)calloc((size_t)nb, sizeof(double));
    double R[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
    for (int32_t t = 0; t < n_threads; ++t) {
        for (int64_t k = 0; k < ne * nb; ++k) { S1[k] += wk[t].s1[k]; S2[k] += wk[t].s2[k]; }
        if (ne == 2)
            for (int64_t k = 0; k < nb; ++k) S12[k] += wk[t].s12[k];
        for (int q = 0; q < 5; ++q) R[q] += wk[t].r[q];
        add_counts(&c, &wk[t].c);
        free(wk[t].s1); free(wk[t].s2); free(wk[t].s12);
    }
    if (sum1) memcpy(sum1, S1, (size_t)(ne * nb) * sizeof(double));
    if (sum2) memcpy(sum2, S2, (size_t)(ne * nb) * sizeof(double));
    if (sum12 && ne == 2) memcpy(sum12, S12, (size_t)nb * sizeof(double));
    if (ne == 2) {
        orc_combine(nb, S1, S2, S1 + nb, S2 + nb, S12, n_hist, n_batches, tb.volume,
                    mean, relerr, NULL);
        if (scalar)
            orc_combine(1, &R[0], &R[1], &R[2], &R[3], &R[4], n_hist, n_batches, tb.volume,
                        &scalar[0], &scalar[1], &scalar[2]);
    } else {
        for (int64_t k = 0; k < nb; ++k) {
            double m, rel;
            batch_moments(S1[k], S2[k], n_hist, n_batches, tb.volume, &m, &rel);
            if (mean) mean[k] = m;
            if (relerr) relerr[k] = rel;
        }
        if (scalar) batch_moments(R[0], R[1], n_hist, n_batches, tb.volume, &scalar[0], &scalar[1]);
    }
    if (counts) *counts = c;
    free(S1); free(S2); free(S12);
    free(wk); free(th);
    free_tables(&tb);
    return 0;
}

int orc_trace(const orc_problem *p, uint64_t seed, const uint64_t *hids,
              int64_t n, orc_record *out)
{
    tables tb;
    if (p->pc_target > 0) return -1;     /* histories are not separate under a comb */
    if (make_tables(p, &tb) != 0) { free_tables(&tb); return -1; }
    double *tally = (double *)calloc((size_t)tb.n_bins, sizeof(double));
    orc_counts c;
    memset(&c, 0, sizeof c);
    for (int64_t i = 0; i < n; ++i)
        run_history(p, &tb, seed, hids[i], tally, &c, &out[i]);
    free(tally);
    free_tables(&tb);
    return 0;
}


/* ---- RNG-injection quadrature (test hook) ------------------------------
 * Averages, over a midpoint grid of the uniform numbers a history draws, the
 * track length its particles make after exactly k collisions, k = 0 ..
 * max_order (out[k]).  The history draws the numbers slot by slot (two per
 * draw, in the order of the loop above); slot dim_slot[d] runs over the
 * dim_m[d] nodes of its rule (nodes[], weights[], the rules of the
 * dimensions one after the other, each rule's weights summing to 1), every
 * other slot holds fixed[slot]; a grid point counts with the product of its
 * nodes' weights.  On a problem whose histories draw the same slots for the
 * same events (one cell, no census), out[k] is a product quadrature rule for
 * the expected order-k track length, which converges to its integral as the
 * rules are refined.  Threads split the grid. */
typedef struct {
    const orc_problem *p;
    const tables *tb;
    int32_t n_slots, n_dims, max_order;
    const double *fixed, *nodes, *weights;
    const int32_t *dim_slot, *dim_m, *dim_off;
    int64_t i0, i1;
    double out[16];
} inj_job;

static void *inj_work(void *arg)
{
    inj_job *J = (inj_job *)arg;
    double *slots = (double *)malloc(sizeof(double) * J->n_slots);
    double *tally = (double *)calloc((size_t)J->tb->n_bins * 2, sizeof(double));
    double order[16];
    orc_counts c;
    memset(&c, 0, sizeof c);
    memcpy(slots, J->fixed, sizeof(double) * J->n_slots);
    for (int k = 0; k <= J->max_order; ++k) J->out[k] = 0.0;
    g_inj = slots;
    g_inj_n = J->n_slots;
    g_order = order;
    g_max_order = J->max_order;
    for (int64_t i = J->i0; i < J->i1; ++i) {
        int64_t q = i;
        double wt = 1.0;
        for (int32_t d = 0; d < J->n_dims; ++d) {
            const int64_t m = J->dim_m[d], j = q % m;
            slots[J->dim_slot[d]] = J->nodes[J->dim_off[d] + j];
            wt *= J->weights[J->dim_off[d] + j];
            q /= m;
        }
        for (int k = 0; k <= J->max_order; ++k) order[k] = 0.0;
        g_inj_pos = 0;
        run_history(J->p, J->tb, 0, 0, tally, &c, NULL);
        for (int k = 0; k <= J->max_order; ++k) J->out[k] += wt * order[k];
    }
    g_inj = NULL;
    g_order = NULL;
    free(slots);
    free(tally);
    return NULL;
}

int orc_inject_grid(const orc_problem *p, int32_t n_slots, const double *fixed, int32_t n_dims,
                    const int32_t *dim_slot, const int32_t *dim_m, const double *nodes,
                    const double *weights, int32_t max_order, int32_t threads, double *out)
{
    if (max_order < 0 || max_order > 15 || n_dims < 1 || n_dims > 32 || threads < 1) return -1;
    tables tb;
    if (make_tables(p, &tb)) return -1;
    int64_t total = 1;
    int32_t off[32];
    for (int32_t d = 0, o = 0; d < n_dims; ++d) {
        if (dim_slot[d] < 0 || dim_slot[d] >= n_slots || dim_m[d] < 1) { free_tables(&tb); return -1; }
        total *= dim_m[d];
        off[d] = o;
        o += dim_m[d];
    }
    inj_job *jobs = (inj_job *)calloc((size_t)threads, sizeof(inj_job));
    pthread_t *th = (pthread_t *)calloc((size_t)threads, sizeof(pthread_t));
    for (int32_t t = 0; t < threads; ++t) {
        inj_job *J = &jobs[t];
        J->p = p; J->tb = &tb; J->n_slots = n_slots; J->n_dims = n_dims;
        J->max_order = max_order; J->fixed = fixed; J->dim_slot = dim_slot; J->dim_m = dim_m;
        J->dim_off = off; J->nodes = nodes; J->weights = weights;
        J->i0 = total * t / threads;
        J->i1 = total * (t + 1) / threads;
        pthread_create(&th[t], NULL, inj_work, J);
    }
    for (int k = 0; k <= max_order; ++k) out[k] = 0.0;
    for (int32_t t = 0; t < threads; ++t) {                 /* fixed order of the sums */
        pthread_join(th[t], NULL);
        for (int k = 0; k <= max_order; ++k) out[k] += jobs[t].out[k];
    }
    free(jobs);
    free(th);
    free_tables(&tb);
    return 0;
}
