// common.cuh -- device data layout shared by the tracker kernels and the host
// side of the library: problem tables, run arguments, the counter-based
// generator and the warp-aggregated queue append.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace mcdc {

constexpr int kMaxGroups = 16;
constexpr int kWarp = 32;

enum End : int32_t { END_NONE = 0, END_ABSORBED = 1, END_LEAKED = 2, END_CENSUSED = 3,
                     END_ROULETTE = 4 };

enum ErrBits : int32_t { ERRBIT_OVERFLOW = 1, ERRBIT_TIMEOUT = 2, ERRBIT_CHECK = 4 };

// Bounds checks of the checked build (compiled with -DMCDC_CHECKS): each
// index a kernel computes into a table, a tally, a stack, a bank or a record
// array is compared with the extent of what it indexes before the access.  A
// bad one sets ERRBIT_CHECK in error[0], the first failing site and its index
// go to error[1] and error[2..3] (low, high word), and the access is skipped.
// In the normal build every check is the constant `true` and its operands are
// not evaluated, so the checks leave no code behind.
enum CheckSite : int32_t {
  CHK_NONE = 0,
  CHK_CELL = 1,        // cell index of a particle (flight, collision, window)
  CHK_GROUP = 2,       // energy group of a particle (shared cross-section tables)
  CHK_MATERIAL = 3,    // material id of a cell
  CHK_TBIN = 4,        // time bin of a scoring particle
  CHK_TALLY = 5,       // tally entry (shared, step or global slices)
  CHK_WW_BIN = 6,      // window-table entry
  CHK_POOL = 7,        // slot of a warp's particle pool
  CHK_STACK = 8,       // warp stack of split children (push or pop)
  CHK_SPILL_IN = 9,    // position in the bank a pass runs
  CHK_COMB_OUT = 10,   // comb output slot
  CHK_COMB_IN = 11,    // comb input position
  CHK_SELFTEST = 12,   // the checked build's self-test
  CHK_SITES = 13
};

#ifdef MCDC_CHECKS
static __device__ __noinline__ bool check_failed(int32_t *err, int32_t site, long long idx) {
  if (err != nullptr) {
    atomicOr(err, ERRBIT_CHECK);
    if (atomicCAS(err + 1, 0, site) == 0) {
      err[2] = (int32_t)(idx & 0xFFFFFFFFll);
      err[3] = (int32_t)(idx >> 32);
    }
  }
  return false;
}
#define MCDC_CHK(err, site, ok, idx) \
  ((ok) ? true : ::mcdc::check_failed((err), (site), (long long)(idx)))
#define MCDC_CHECKED_ONLY(x) (x)     // an operand only the checks use
constexpr bool kChecked = true;
#else
#define MCDC_CHK(err, site, ok, idx) true
#define MCDC_CHECKED_ONLY(x) 0
constexpr bool kChecked = false;
#endif

// Problem tables in device memory (built once at create).
struct DevProblem {
  int32_t n[3];
  int32_t bounded[3];
  double origin[3];
  double width[3];
  int32_t bc[6];
  int32_t M, G, T, T1;        // T time bins (0: steady), T1 = max(T, 1)
  int64_t n_cells, n_bins;
  int64_t n_tally;            // n_est x n_bins: one tally per estimator scored (2 when combined)
  double volume;
  const uint8_t *material;    // [cells]
  const double *faces[3];     // [n_a + 1] face coordinates origin + k * width (bounded axes)
  float width32[3];           // cell widths in FP32 (cell-local mode)
  const float *binw32;        // [T] time-bin widths in FP32 (cell-local mode)
  // FP64 tables
  const double *sigma_t;      // [M*G]
  const double *scat;         // [M*G]  sigma_s / sigma_t
  const double *cdf;          // [M*G*G] cumulative transfer, flat 1.0 after the last rise
  const double *speed;        // [G]
  const double *edges;        // [T+1]
  const double *src_cdf;      // [G]
  // FP32 copies
  const float *sigma_t32, *scat32, *cdf32, *speed32, *inv_speed32, *src_cdf32;
  // source
  double src_lo[3], src_hi[3];
  float src_cell_a[3], src_cell_b[3];   // FP32 modes: a source coordinate in cell
                                        // units is a + xi b (bounded axes)
  int32_t src_kind;
  double src_dir[3];
  double t0, t1;
  // weight windows (nullptr: analog)
  const double *ww_lower;     // [n_bins]
  const float *ww_lower32;
  // per-event windows from the importance network instead of the table
  // (nullptr: off): parameters, inputs (4 + G) and hidden width, and the
  // map of its output y to w_L = wl0 exp(min(0, max(y scale + shift, floor) - top))
  const double *ww_net64;
  const float *ww_net32;
  const uint32_t *ww_netfrag; // the same network as binary16 mma.sync fragments (FP32 modes)
  float ww_net_b3;            // its output bias
  float net_cell[3], net_off[3];   // input of axis a: cell i, offset o in it -> i net_cell[a]
                                   // + o net_off[a] - 1 (2 / n, 2 / (n width); 0 unbounded)
  int32_t ww_net_in, ww_net_h;
  double ww_net_shift, ww_net_scale, ww_net_top, ww_net_floor, ww_net_wl0;
  double ww_upper, ww_survival;
  // FP32 copies (rounded to nearest on the host) for the FP32 modes' checks:
  // a conversion in the kernel would occupy the FP64 pipe at every check
  float ww_net_shift32, ww_net_scale32, ww_net_top32, ww_net_floor32, ww_net_wl0_32;
  float ww_upper32, ww_survival32;
  int32_t ww_nmax;
  int32_t region_lo[3], region_hi[3];
  // estimator and collision physics options
  int32_t estimator;          // 0 track length, 1 collision, 2 both (combined estimate)
  int32_t implicit;           // 1: implicit capture with weight-cutoff roulette
  double wcut, wsurv;         // cutoff and survival weight (implicit capture)
  float wcut32, wsurv32;
  int32_t pc_target;          // population control: particles per batch after a comb (0: off)
  int32_t fresh_tau;          // FP32 modes: 1 = sample the distance to collision every flight
  int32_t sum_weights;        // 1: sum weights even when every particle keeps weight 1
};

// weight windows are on: a table or the network
__host__ __device__ inline bool ww_on(const DevProblem &P) {
  return P.ww_lower != nullptr || P.ww_net64 != nullptr;
}

// particle weights are summed on the device (births and ends): weighted runs,
// and every problem of a batched run (whose problems share one sum)
__host__ __device__ inline bool weights_summed(const DevProblem &P) {
  return P.sum_weights || ww_on(P) || P.implicit || P.pc_target > 0;
}

// One particle as it moves between the tracker phases (kept in registers).
// Q = double: x, y, z are the position and t the time.  Q = float (the
// cell-local FP32 mode): x, y, z are offsets from the low faces of the cell
// and t is the time left to the next census edge.
template <class R, class Q = double>
struct Part {
  Q x, y, z;          // position (or cell-local offsets)
  Q t;                // time (or time to the next census edge)
  R ux, uy, uz;       // direction
  R w;                // weight
  int32_t g;
  int32_t i, j, k;    // cell
  int32_t tbin;
  uint32_t ctr, serial;
  uint64_t hid;
  uint32_t nseg, ncol, ncross;
  float tau;          // FP32 modes: mean free paths left to the next collision (< 0: draw afresh)
  uint32_t slot;      // population control: the particle's position in this step's input
};

// Per-history record (mirrors mcdc_record).
struct Record {
  uint64_t hid;
  int32_t end, g;
  uint32_t ctr, n_seg, n_col, n_cross;
  double x, y, z, t, w;
};

// Event counters; summed per warp, then one atomic per warp per field.
struct Stats {
  unsigned long long histories, segments, collisions, crossings, census;
  unsigned long long absorbed, leaked, censused, splits, children;
  unsigned long long roulette_killed, roulette_survived;
  double w_source, w_absorbed, w_leaked, w_censused;
  unsigned long long splits_dropped;
  unsigned long long pc_combs, pc_in, pc_out;
  double w_pc_in, w_pc_out;
};

// Philox round keys of one seed: (k0 + r W0, k1 + r W1) for rounds r = 0..9,
// computed once per run so each round reads its key instead of adding it.
struct RoundKeys {
  uint32_t k[20];
};

// Unsigned 32-bit division by a run constant d >= 1 as a multiply-high, two
// subtractions and shifts (Granlund & Montgomery, "Division by invariant
// integers using multiplication", PLDI 1994, Fig. 4.1): with l = ceil(log2 d)
// and m = floor(2^32 (2^l - d) / d) + 1, n / d = (t + ((n - t) >> min(l, 1)))
// >> max(l - 1, 0), t = mulhi(m, n), exactly for every 32-bit n.
struct Div32 {
  uint32_t m = 1;
  int s1 = 0, s2 = 0;
  __host__ void set(uint32_t d) {
    int l = 0;
    while (l < 32 && (1ull << l) < (uint64_t)d) ++l;
    m = (uint32_t)(((1ull << 32) * ((1ull << l) - d)) / d + 1);
    s1 = l < 1 ? l : 1;
    s2 = l > 1 ? l - 1 : 0;
  }
  __device__ __forceinline__ uint32_t div(uint32_t n) const {
    const uint32_t t = __umulhi(m, n);
    return (t + ((n - t) >> s1)) >> s2;
  }
};

struct RunArgs {
  RoundKeys rk;               // round keys of `seed`
  uint64_t n_hist;            // histories in the whole run
  uint64_t offset;            // first history id
  uint64_t seed;
  int32_t n_batches;
  // shared-tally mode: CTAs claim whole batches through *work
  // global-tally mode: this launch covers batch `batch`; CTAs claim chunks
  unsigned long long *work;
  int32_t batch;
  int32_t chunk;
  double *tally;              // global mode: batch tally [n_est x n_bins]
  float *tally32;             // FP32 modes, one-launch runs: FP32 batch slices
                              // (used instead of tally when set; folded in FP64)
  double *sum1, *sum2;        // shared mode: folded per batch ([n_est x n_bins])
  double *sum12;              // combined estimator: sums of track x collision batch products
  double *region;             // [5]: region batch sums and squares (track or the one
                              // estimator; collision), sum of their products
  Stats *stats;
  Record *records;            // or nullptr
  uint64_t n_records;
  int32_t *error;             // ERRBIT_* flags
  // per-warp overflow stacks for split children: [warps in grid][overflow_cap]
  void *overflow;
  int32_t overflow_cap;       // per warp
  int32_t overflow_tail;      // slots a warp keeps once its own particles are exhausted
                              // (children beyond spill; -1: overflow_cap)
  int32_t warp_aggregate;
  // global-tally mode with weight windows: children beyond the warp's stack
  // spill to a device-wide bank, run in a later pass by every warp
  void *spill_out;            // bank written by this pass (nullptr: no spill)
  unsigned long long *spill_out_count;
  unsigned long long spill_cap;
  const void *spill_in;       // bank this pass runs instead of new histories
  const unsigned long long *spill_in_count;
  unsigned long long *spill_in_cursor;
  // population control: a particle reaching an interior census edge is
  // written to census_out[slot] (its position in the step's input) with its
  // weight in census_w[slot], instead of flying on (nullptr: off)
  void *census_out;
  double *census_w;
  unsigned long long *census_count;
  unsigned long long census_cap;
  // population control runs every batch in each launch: the global tally is
  // one slice of n_est x n_bins per batch, picked from the particle's history id
  int32_t tally_per_batch;
  uint64_t batch_q, batch_r;  // n_hist / n_batches and n_hist % n_batches
  Div32 div_q1, div_q;        // division by batch_q + 1 and by batch_q (n_hist < 2^32)
  // population control, one time step: every particle of the launch is in
  // time bin step_tbin, so it scores into a CTA-private shared tally of
  // step_bins = n_est x n_batches x cells x groups entries, added into the
  // per-batch slices at the end of the launch (0: score the slices directly)
  int32_t step_tally;
  int32_t step_tbin;
  int32_t step_bins;
  // weight windows: children made so far in the run (device counter) and the
  // run's budget; nullptr: no budget
  unsigned long long *children_made;
  unsigned long long children_budget;
  // population control after a comb: every warp stages its next 32 births
  // from the combed bank (pool layout) in shared memory with bulk async
  // copies while its particles fly (the launch's shared memory has room)
  int32_t prefetch;
};

// batch of history h (0-based within the run) from the run's precomputed
// quotient and remainder; 32-bit division when the run allows it
__device__ __forceinline__ int32_t batch_of_run(const RunArgs &A, uint64_t h) {
  const uint64_t big = A.batch_r * (A.batch_q + 1);
  if (A.n_hist <= 0xFFFFFFFFull) {
    const uint32_t h32 = (uint32_t)h;
    return (int32_t)(h < big ? A.div_q1.div(h32)
                             : (uint32_t)A.batch_r + A.div_q.div(h32 - (uint32_t)big));
  }
  return (int32_t)(h < big ? h / (A.batch_q + 1) : A.batch_r + (h - big) / A.batch_q);
}

// ---- counter-based generator: Philox4x32-10 (Salmon et al., SC'11) -------
struct U4 { uint32_t a, b, c, d; };

__device__ __forceinline__ U4 philox4x32_10(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                                            uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint32_t lo0 = 0xD2511F53u * c0;
    const uint32_t hi0 = __umulhi(0xD2511F53u, c0);
    const uint32_t lo1 = 0xCD9E8D57u * c2;
    const uint32_t hi1 = __umulhi(0xCD9E8D57u, c2);
    const uint32_t n0 = hi1 ^ c1 ^ k0;
    const uint32_t n2 = hi0 ^ c3 ^ k1;
    c0 = n0; c1 = lo1; c2 = n2; c3 = lo0;
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  return U4{c0, c1, c2, c3};
}

// the same ten rounds with the round keys given
__device__ __forceinline__ U4 philox4x32_10_rk(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                                               const RoundKeys &rk) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint32_t lo0 = 0xD2511F53u * c0;
    const uint32_t hi0 = __umulhi(0xD2511F53u, c0);
    const uint32_t lo1 = 0xCD9E8D57u * c2;
    const uint32_t hi1 = __umulhi(0xCD9E8D57u, c2);
    const uint32_t n0 = hi1 ^ c1 ^ rk.k[2 * r];
    const uint32_t n2 = hi0 ^ c3 ^ rk.k[2 * r + 1];
    c0 = n0; c1 = lo1; c2 = n2; c3 = lo0;
  }
  return U4{c0, c1, c2, c3};
}

__host__ __device__ inline RoundKeys round_keys(uint64_t seed) {
  RoundKeys rk;
  uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
  for (int r = 0; r < 10; ++r) {
    rk.k[2 * r] = k0;
    rk.k[2 * r + 1] = k1;
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  return rk;
}

// draw one block for the particle and advance its counter
template <class PartT>
__device__ __forceinline__ U4 draw(const PartT &p, uint32_t &ctr, const RoundKeys &rk) {
  U4 r = philox4x32_10_rk(ctr, p.serial, (uint32_t)p.hid, (uint32_t)(p.hid >> 32), rk);
  ctr += 1;
  return r;
}

// 53 bits -> (0, 1]
__device__ __forceinline__ double u01_f64(uint32_t hi, uint32_t lo) {
  const uint64_t bits = ((uint64_t)hi << 32) | (uint64_t)lo;
  return (double)((bits >> 11) + 1ull) * 0x1.0p-53;
}

// 24 bits -> (0, 1]: the top 24 bits of the same word pair, so an FP32 run
// follows its FP64 twin until the first decision the rounding flips.
__device__ __forceinline__ float u01_f32(uint32_t hi) {
  return (float)((hi >> 8) + 1u) * 0x1.0p-24f;
}

// ---- warp-level queue append: ballot + popc prefix, one atomic per warp ---
__device__ __forceinline__ int warp_append(bool pred, int *counter) {
  const unsigned mask = __ballot_sync(0xffffffffu, pred);
  const int lane = threadIdx.x & 31;
  int base = 0;
  if (lane == 0 && mask) base = atomicAdd(counter, __popc(mask));
  base = __shfl_sync(0xffffffffu, base, 0);
  return base + __popc(mask & ((1u << lane) - 1u));
}

// batch of history h (0-based within the run): the first n % B batches hold
// one history more than the others
__host__ __device__ __forceinline__ int32_t batch_of(uint64_t n, int32_t B, uint64_t h) {
  const uint64_t q = n / (uint64_t)B, r = n % (uint64_t)B;
  const uint64_t big = r * (q + 1);
  return (int32_t)(h < big ? h / (q + 1) : r + (h - big) / q);
}

__host__ __device__ __forceinline__ uint64_t batch_start(uint64_t n, int32_t B, int32_t b) {
  const uint64_t q = n / (uint64_t)B, r = n % (uint64_t)B;
  const uint64_t bb = (uint64_t)b;
  return bb * q + (bb < r ? bb : r);
}

}  // namespace mcdc
