// batched.cu -- many independent problems in one run: per batch, one
// persistent launch in which CTAs claim (problem, history range) work items
// (largest first), load the item's problem tables into shared memory when the
// problem changes, and score into that problem's device tally; then one fused
// fold of every problem's batch tally.  The whole sequence is captured once
// as a CUDA graph per batch shape and replayed by later calls.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/mcdc.h"
#include "launch.h"
#include "problem.h"
#include "tracker.cuh"

namespace mcdc {

// Fold of every problem's batch tally: sum1 += x, sum2 += x^2, x = 0, and the
// batch's region sum per problem (one row of blocks per problem).
struct FoldItem {
  double *tally, *sum1, *sum2, *region_batch;
};

__global__ void __launch_bounds__(512) k_fold_multi(const DevProblem *__restrict__ probs,
                                                    const FoldItem *__restrict__ fi) {
  // blockIdx.y: the problem; its bins in a grid-stride loop over blockIdx.x
  __shared__ double red[16];
  const DevProblem &P = probs[blockIdx.y];
  const FoldItem f = fi[blockIdx.y];
  const RegionTest region(P);
  const long long nb = P.n_bins;
  double rs = 0.0;
  for (long long b = blockIdx.x * (long long)blockDim.x + threadIdx.x; b < nb;
       b += (long long)gridDim.x * blockDim.x) {
    const double v = f.tally[b];
    if (v != 0.0) {
      f.sum1[b] += v;
      f.sum2[b] += v * v;
      f.tally[b] = 0.0;
      if (region(P, b)) rs += v;
    }
  }
  // the block's region sum: one atomic per block instead of one per bin
  for (int o = 16; o > 0; o >>= 1) rs += __shfl_xor_sync(0xffffffffu, rs, o);
  const int nw = (int)(blockDim.x >> 5);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = rs;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < nw; ++w) t += red[w];
    if (t != 0.0) atomicAdd(f.region_batch, t);
  }
}

// Zeroes every problem's batch sums and region accumulators (one row of
// blocks per problem) at the start of a batched run.
__global__ void k_zero_multi(const DevProblem *__restrict__ probs, const FoldItem *__restrict__ fi,
                             double *const *regions) {
  const FoldItem f = fi[blockIdx.y];
  const long long nb = probs[blockIdx.y].n_bins;
  for (long long b = blockIdx.x * (long long)blockDim.x + threadIdx.x; b < nb;
       b += (long long)gridDim.x * blockDim.x) {
    f.sum1[b] = 0.0;
    f.sum2[b] = 0.0;
  }
  if (blockIdx.x == 0 && threadIdx.x < 4) regions[blockIdx.y][threadIdx.x] = 0.0;
}

__global__ void k_region_fold_multi(const FoldItem *__restrict__ fi, double *const *regions, int n) {
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < n; p += gridDim.x * blockDim.x) {
    const double b = *fi[p].region_batch;
    regions[p][0] += b;
    regions[p][1] += b * b;
    *fi[p].region_batch = 0.0;
  }
}

}  // namespace mcdc

using namespace mcdc;

namespace {
int fail(int code, const std::string &m) { return mcdc::set_error(code, m); }

struct DevFree {
  std::vector<void *> v;
  ~DevFree() { for (void *p : v) cudaFree(p); }
};

#define CKB(call)                                                                        \
  do {                                                                                   \
    cudaError_t e_ = (call);                                                             \
    if (e_ != cudaSuccess)                                                               \
      return fail(e_ == cudaErrorMemoryAllocation ? MCDC_ERR_OOM : MCDC_ERR_CUDA,        \
                  std::string(#call) + ": " + cudaGetErrorString(e_));                   \
  } while (0)

template <class T>
cudaError_t dnew(DevFree &f, T **p, size_t n) {
  cudaError_t e = cudaMalloc((void **)p, std::max<size_t>(n * sizeof(T), 16));
  if (e == cudaSuccess) f.v.push_back(*p);
  return e;
}

bool dev_ptr(const void *p) {
  if (!p) return false;
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) { cudaGetLastError(); return false; }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}
}  // namespace

namespace {
// A batched run's plan: its device argument buffers and the whole run
// captured once as a CUDA graph (zero the sums, per batch one persistent
// launch over every problem and one fused fold, the per-problem
// finalisations into device outputs).  Plans are cached by the run's shape
// -- the problems (by identity), their history counts, the batches, the
// launch shape and the device outputs -- so a repeated call uploads the
// per-problem arguments (the seeds change) and replays the graph; nothing is
// captured or instantiated again.  Destroying a problem drops the plans that
// hold it.
struct BatchedPlan {
  std::vector<uint64_t> key;
  int device = 0, block = 0, cps = 0, B = 0;
  std::vector<uint64_t> uids;
  std::vector<RunArgs> ha;              // host copy of the per-problem arguments
  DevFree fr;                           // device buffers of the plan
  Stats *d_stats = nullptr;
  int32_t *d_err = nullptr;
  unsigned long long *d_children = nullptr;   // children made this call (windows)
  RunArgs *d_args = nullptr;
  double *scratch = nullptr;            // host outputs: [2][largest tally]
  long long max_bins = 0;
  cudaStream_t st = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  ~BatchedPlan() {
    cudaSetDevice(device);
    if (st) cudaStreamSynchronize(st);
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (st) cudaStreamDestroy(st);
    cudaGetLastError();
  }
};

constexpr int kBatchedStack = 1024;   // split-children slots per warp (weight windows)

std::mutex g_plan_mu;
std::vector<std::unique_ptr<BatchedPlan>> g_plans;   // most recently used last
constexpr size_t kMaxPlans = 4;

int build_plan(BatchedPlan &pl, struct mcdc_problem *const *probs, int32_t n,
               const uint64_t *n_histories, double *const *mean_dev, double *const *rel_dev,
               int B, int block, unsigned long long chunk, int cps_want) {
  mcdc_problem *p0 = probs[0];
  // launch shape: the largest tables of the batch, no shared tally
  TrackKey key = p0->key;
  key.shared = false;
  key.multi = true;
  key.net = false;
  key.pc = false;
  key.vr = false;
  for (int i = 0; i < n; ++i) key.vr = key.vr || ww_on(probs[i]->P);
  Layout L{};
  for (int i = 0; i < n; ++i) {
    L.M = std::max(L.M, probs[i]->P.M);
    L.G = std::max(L.G, probs[i]->P.G);
    L.T = std::max(L.T, probs[i]->P.T);
  }
  L.S = (block / 32) * kPool;
  L.tables_bytes = tables_bytes_of(key.f64, L.M, L.G, L.T);
  L.tally_bytes = 0;
  L.bank_bytes = L.S * slot_bytes(key.f64, p0->dim, key.local);
  L.total = (int)(L.tables_bytes + L.bank_bytes + 64);
  int smem_max = 0;
  CKB(cudaDeviceGetAttribute(&smem_max, cudaDevAttrMaxSharedMemoryPerBlockOptin, p0->device));
  if (L.total > smem_max - 2048) return fail(MCDC_ERR_INVALID, "tables too large for shared memory");
  CKB(prepare_track(key, smem_max - 2048));
  int cps = track_occupancy(key, block, L.total);
  if (cps < 1) return fail(MCDC_ERR_INVALID, "launch shape does not fit");
  if (cps_want > 0) {
    if (cps_want > cps) return fail(MCDC_ERR_INVALID, "CTAs per SM beyond what fits");
    cps = cps_want;
  }
  const int grid = p0->sms * cps;
  pl.device = p0->device;
  pl.block = block;
  pl.cps = cps;
  pl.B = B;

  CKB(dnew(pl.fr, &pl.d_stats, 1));
  CKB(dnew(pl.fr, &pl.d_err, 4));
  // weight windows: one stack of split children per warp of the launch
  // (kBatchedStack slots; there is no spill bank here, so a child that finds
  // the stack full is not made -- counted, and unbiased), and the run's
  // children budget as in a single-problem run
  bool windows = false;
  uint64_t hist_total = 0;
  for (int i = 0; i < n; ++i) {
    windows = windows || ww_on(probs[i]->P);
    hist_total += n_histories[i];
  }
  void *d_ovf = nullptr;
  unsigned long long *d_children = nullptr;
  if (windows) {
    const size_t pb = key.f64 ? sizeof(Part<double>)
                      : (key.local ? sizeof(Part<float, float>) : sizeof(Part<float>));
    const size_t warps = (size_t)grid * (block / 32);
    unsigned char *o = nullptr;
    CKB(dnew(pl.fr, &o, warps * kBatchedStack * pb));
    d_ovf = o;
    CKB(dnew(pl.fr, &d_children, 1));
  }
  pl.d_children = d_children;
  std::vector<DevProblem> hp(n);
  std::vector<FoldItem> hf(n);
  std::vector<double *> hreg(n);
  pl.ha.resize(n);
  for (int i = 0; i < n; ++i) {
    mcdc_problem *p = probs[i];
    hp[i] = p->P;
    // with windows in the run, every problem's weights are summed on the
    // device (one sum over problems with and without windows); analog runs
    // carry unit weights, and their counts are the weights
    hp[i].sum_weights = windows ? 1 : 0;
    RunArgs A{};
    A.n_hist = n_histories[i];
    A.offset = 0;
    A.n_batches = B;
    A.tally = p->tally;
    A.stats = pl.d_stats;
    A.error = pl.d_err;
    A.warp_aggregate = p->warp_aggregate;
    if (windows) {
      A.overflow = d_ovf;
      A.overflow_cap = kBatchedStack;
      A.overflow_tail = -1;
      A.children_made = d_children;
      A.children_budget = std::max<unsigned long long>(1ull << 27, 4096ull * hist_total);
    }
    pl.ha[i] = A;
    hf[i] = {p->tally, p->sum1, p->sum2, p->region_batch};
    hreg[i] = p->region;
    pl.uids.push_back(p->uid);
    pl.max_bins = std::max<long long>(pl.max_bins, p->P.n_bins);
  }
  // work items, batch by batch, largest first within a batch
  std::vector<WorkItem> items;
  std::vector<int> item_off(B + 1, 0);
  for (int b = 0; b < B; ++b) {
    std::vector<WorkItem> bi;
    for (int i = 0; i < n; ++i) {
      const uint64_t h0 = batch_start(n_histories[i], B, b), h1 = batch_start(n_histories[i], B, b + 1);
      for (uint64_t h = h0; h < h1; h += chunk) bi.push_back({i, 0, h, std::min<uint64_t>(h1, h + chunk)});
    }
    std::stable_sort(bi.begin(), bi.end(), [](const WorkItem &x, const WorkItem &y) {
      return (x.h1 - x.h0) > (y.h1 - y.h0);
    });
    items.insert(items.end(), bi.begin(), bi.end());
    item_off[b + 1] = (int)items.size();
  }
  DevProblem *d_probs;
  WorkItem *d_items;
  FoldItem *d_fold;
  double **d_reg;
  unsigned long long *d_ctr;
  CKB(dnew(pl.fr, &d_probs, n));
  CKB(dnew(pl.fr, &pl.d_args, n));
  CKB(dnew(pl.fr, &d_items, items.size()));
  CKB(dnew(pl.fr, &d_fold, n));
  CKB(dnew(pl.fr, &d_reg, n));
  CKB(dnew(pl.fr, &d_ctr, B));
  CKB(cudaMemcpy(d_probs, hp.data(), sizeof(DevProblem) * n, cudaMemcpyHostToDevice));
  CKB(cudaMemcpy(d_items, items.data(), sizeof(WorkItem) * items.size(), cudaMemcpyHostToDevice));
  CKB(cudaMemcpy(d_fold, hf.data(), sizeof(FoldItem) * n, cudaMemcpyHostToDevice));
  CKB(cudaMemcpy(d_reg, hreg.data(), sizeof(double *) * n, cudaMemcpyHostToDevice));

  CKB(cudaStreamCreateWithFlags(&pl.st, cudaStreamNonBlocking));
  CKB(cudaEventCreate(&pl.e0));
  CKB(cudaEventCreate(&pl.e1));
  cudaStream_t st = pl.st;
  // fold grid: x blocks per problem (enough for the largest), one row per problem
  const dim3 row_grid((unsigned)std::max<long long>(1, std::min<long long>((pl.max_bins + 511) / 512, 64)),
                      (unsigned)n);
  CKB(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
  cudaMemsetAsync(pl.d_stats, 0, sizeof(Stats), st);
  cudaMemsetAsync(pl.d_err, 0, 4 * sizeof(int32_t), st);
  cudaMemsetAsync(d_ctr, 0, sizeof(unsigned long long) * B, st);
  if (d_children) cudaMemsetAsync(d_children, 0, sizeof(unsigned long long), st);
  k_zero_multi<<<row_grid, 512, 0, st>>>(d_probs, d_fold, d_reg);
  for (int b = 0; b < B; ++b) {
    MultiArgs MA{d_probs, pl.d_args, d_items + item_off[b], item_off[b + 1] - item_off[b], d_ctr + b};
    launch_track(key, grid, block, L.total, st, hp[0], pl.ha[0], L, &MA);
    k_fold_multi<<<row_grid, 512, 0, st>>>(d_probs, d_fold);
    k_region_fold_multi<<<(n + 255) / 256, 256, 0, st>>>(d_fold, d_reg, n);
  }
  for (int i = 0; i < n; ++i) {
    mcdc_problem *p = probs[i];
    double *m = mean_dev ? mean_dev[i] : nullptr;
    double *r = rel_dev ? rel_dev[i] : nullptr;
    if (m || r)
      launch_finalize(st, p->P.n_bins, p->sum1, p->sum2, n_histories[i], B, p->P.volume, m, r, p->sms);
  }
  const cudaError_t ec = cudaStreamEndCapture(st, &pl.graph);
  if (ec != cudaSuccess) return fail(MCDC_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(ec));
  CKB(cudaGraphInstantiate(&pl.exec, pl.graph, 0));
  return MCDC_OK;
}

// One batched run with a given launch shape: threads per CTA and histories
// per work item.
// cache = false (the autotuner's trial runs): the plan is built for this call
// only and not kept.
int run_batched(struct mcdc_problem *const *probs, int32_t n, const uint64_t *n_histories,
                uint64_t seed, int32_t n_batches, double *const *mean_out,
                double *const *relerr_out, double *scalar_out, mcdc_stats *stats, int block,
                unsigned long long chunk, int cps_want = 0, bool cache = true) {
  if (!probs || n < 1 || !n_histories) return fail(MCDC_ERR_INVALID, "need problems and history counts");
  if (n > 65535) return fail(MCDC_ERR_INVALID, "at most 65535 problems per batched run");
  const int B = n_batches > 0 ? n_batches : 16;
  if (B < 2) return fail(MCDC_ERR_INVALID, "need at least 2 batches");
  mcdc_problem *p0 = probs[0];
  for (int i = 0; i < n; ++i) {
    const mcdc_problem *p = probs[i];
    if (!p) return fail(MCDC_ERR_INVALID, "problem is NULL");
    if (p->device != p0->device || p->key.f64 != p0->key.f64 || p->key.local != p0->key.local ||
        p->dim != p0->dim)
      return fail(MCDC_ERR_INVALID, "batched problems need the same device, precision and dimension");
    if (p->P.ww_net64 != nullptr || p->P.implicit || p->P.pc_target > 0)
      return fail(MCDC_ERR_INVALID, "batched runs take analog collisions and table windows "
                                    "(no per-event network windows, implicit capture or "
                                    "population control)");
    if (p->P.estimator == MCDC_EST_COMBINED)
      return fail(MCDC_ERR_INVALID, "batched runs score one estimator (no combined estimator)");
    if (n_histories[i] < (uint64_t)B) return fail(MCDC_ERR_INVALID, "every problem needs >= n_batches histories");
  }
  CKB(cudaSetDevice(p0->device));
  // every problem scores into a device tally of its own
  for (int i = 0; i < n; ++i) {
    mcdc_problem *p = probs[i];
    if (!p->tally) {
      double *t = nullptr;
      CKB(cudaMalloc(&t, sizeof(double) * p->P.n_bins));
      p->allocs.push_back(t);
      p->tally = t;
      CKB(cudaMemset(t, 0, sizeof(double) * p->P.n_bins));
    }
  }
  // the plan's key: problems, histories, outputs written by the graph, shape
  std::vector<double *> mdev(n, nullptr), rdev(n, nullptr);
  bool any_host = false;
  std::vector<uint64_t> key;
  key.reserve(4 * (size_t)n + 4);
  key.push_back((uint64_t)n);
  key.push_back((uint64_t)B);
  key.push_back((uint64_t)block);
  key.push_back(chunk);
  key.push_back((uint64_t)cps_want);
  for (int i = 0; i < n; ++i) {
    mdev[i] = mean_out && mean_out[i] && dev_ptr(mean_out[i]) ? mean_out[i] : nullptr;
    rdev[i] = relerr_out && relerr_out[i] && dev_ptr(relerr_out[i]) ? relerr_out[i] : nullptr;
    any_host = any_host || (mean_out && mean_out[i] && !mdev[i]) ||
               (relerr_out && relerr_out[i] && !rdev[i]);
    key.push_back(probs[i]->uid);
    key.push_back(probs[i]->p_version);
    key.push_back(n_histories[i]);
    key.push_back((uint64_t)(uintptr_t)mdev[i]);
    key.push_back((uint64_t)(uintptr_t)rdev[i]);
  }
  std::unique_lock<std::mutex> lk(g_plan_mu);
  BatchedPlan *pl = nullptr;
  std::unique_ptr<BatchedPlan> once;
  for (size_t k = 0; cache && k < g_plans.size(); ++k) {
    if (g_plans[k]->key == key) {
      std::unique_ptr<BatchedPlan> hit = std::move(g_plans[k]);
      g_plans.erase(g_plans.begin() + (long)k);
      g_plans.push_back(std::move(hit));
      pl = g_plans.back().get();
      break;
    }
  }
  if (!pl) {
    auto np = std::make_unique<BatchedPlan>();
    np->key = key;
    if (int rc = build_plan(*np, probs, n, n_histories, mdev.data(), rdev.data(), B, block, chunk,
                            cps_want))
      return rc;
    if (cache) {
      if (g_plans.size() >= kMaxPlans) g_plans.erase(g_plans.begin());
      g_plans.push_back(std::move(np));
      pl = g_plans.back().get();
    } else {
      once = std::move(np);
      pl = once.get();
    }
  }
  // a single-problem run that returned early left scores in a tally
  for (int i = 0; i < n; ++i) {
    mcdc_problem *p = probs[i];
    if (p->tally_dirty) {
      CKB(cudaMemsetAsync(p->tally, 0, sizeof(double) * p->P.n_bins, pl->st));
      p->tally_dirty = false;
    }
  }
  // this call's seeds: independent streams per problem
  for (int i = 0; i < n; ++i) {
    RunArgs &A = pl->ha[i];
    A.seed = seed + (uint64_t)i * 0x9E3779B97F4A7C15ull;
    A.rk = round_keys(A.seed);
  }
  cudaStream_t st = pl->st;
  CKB(cudaMemcpyAsync(pl->d_args, pl->ha.data(), sizeof(RunArgs) * n, cudaMemcpyHostToDevice, st));
  CKB(cudaEventRecord(pl->e0, st));
  CKB(cudaGraphLaunch(pl->exec, st));
  CKB(cudaEventRecord(pl->e1, st));

  // host outputs: finalise on the device into the plan's scratch, then copy
  if (any_host && !pl->scratch) CKB(dnew(pl->fr, &pl->scratch, 2 * (size_t)pl->max_bins));
  for (int i = 0; i < n; ++i) {
    mcdc_problem *p = probs[i];
    const size_t nb = (size_t)p->P.n_bins;
    const bool hm = mean_out && mean_out[i] && !mdev[i];
    const bool hr = relerr_out && relerr_out[i] && !rdev[i];
    if (hm || hr) {
      double *m = pl->scratch, *r = pl->scratch + pl->max_bins;
      CKB(launch_finalize(st, nb, p->sum1, p->sum2, n_histories[i], B, p->P.volume, m, r, p->sms));
      if (hm) CKB(cudaMemcpyAsync(mean_out[i], m, nb * 8, cudaMemcpyDeviceToHost, st));
      if (hr) CKB(cudaMemcpyAsync(relerr_out[i], r, nb * 8, cudaMemcpyDeviceToHost, st));
    }
  }
  std::vector<double> reg(scalar_out ? 2 * (size_t)n : 0);
  if (scalar_out)
    for (int i = 0; i < n; ++i)
      CKB(cudaMemcpyAsync(&reg[2 * i], probs[i]->region, 2 * sizeof(double), cudaMemcpyDeviceToHost, st));
  Stats h;
  int32_t herr_w[4] = {0, 0, 0, 0};
  CKB(cudaMemcpyAsync(&h, pl->d_stats, sizeof(Stats), cudaMemcpyDeviceToHost, st));
  CKB(cudaMemcpyAsync(herr_w, pl->d_err, 4 * sizeof(int32_t), cudaMemcpyDeviceToHost, st));
  CKB(cudaStreamSynchronize(st));
  if (scalar_out) {
    for (int i = 0; i < n; ++i) {
      const double nv = (double)n_histories[i] * probs[i]->P.volume, Bd = (double)B;
      const double mm = reg[2 * i] / nv;
      double ss = reg[2 * i + 1] - reg[2 * i] * reg[2 * i] / Bd;
      if (ss < 0.0) ss = 0.0;
      const double var = (Bd * Bd / (nv * nv)) * ss / (Bd * (Bd - 1.0));
      scalar_out[2 * i] = mm;
      scalar_out[2 * i + 1] = mm != 0.0 ? std::sqrt(var) / std::fabs(mm) : 0.0;
    }
  }
  if (stats) {
    std::memset(stats, 0, sizeof(*stats));
    stats->histories = h.histories; stats->segments = h.segments;
    stats->collisions = h.collisions; stats->crossings = h.crossings; stats->census = h.census;
    stats->absorbed = h.absorbed; stats->leaked = h.leaked; stats->censused = h.censused;
    stats->splits = h.splits; stats->children = h.children;
    stats->roulette_killed = h.roulette_killed; stats->roulette_survived = h.roulette_survived;
    stats->splits_dropped = h.splits_dropped;
    // summed on the device when the run has windows, else unit weights
    const bool wsum = h.w_source > 0.0;
    stats->w_source = wsum ? h.w_source : (double)h.histories;
    stats->w_absorbed = wsum ? h.w_absorbed : (double)h.absorbed;
    stats->w_leaked = wsum ? h.w_leaked : (double)h.leaked;
    stats->w_censused = wsum ? h.w_censused : (double)h.censused;
    float ms = 0.f;
    cudaEventElapsedTime(&ms, pl->e0, pl->e1);
    stats->kernel_ms = ms;
    stats->total_ms = ms;
    stats->block_size = pl->block;
    stats->ctas_per_sm = pl->cps;
    stats->tally_mode = MCDC_TALLY_GLOBAL;
    stats->n_batches = B;
  }
  if (herr_w[0] & ERRBIT_CHECK) return fail(MCDC_ERR_CHECK, mcdc::check_message(herr_w));
  if (herr_w[0]) return fail(MCDC_ERR_BANK_OVERFLOW, "device error flag set");
  return MCDC_OK;
}

// launch shapes tried by the autotuner, and its choices per batch shape
struct BatchedShape { int block; unsigned long long chunk; int cps; };
std::mutex g_batched_mu;
std::map<std::string, BatchedShape> g_batched_cache;
}  // namespace

extern "C" int mcdc_run_batched(struct mcdc_problem *const *probs, int32_t n,
                                const uint64_t *n_histories, uint64_t seed, int32_t n_batches,
                                double *const *mean_out, double *const *relerr_out,
                                double *scalar_out, mcdc_stats *stats) {
  NvtxRange nvtx("mcdc_run_batched");
  if (!probs || n < 1 || !n_histories || !probs[0]) return fail(MCDC_ERR_INVALID, "need problems and history counts");
  // autotuner: the first time a batch shape is seen (problem count, total
  // histories to a power of two, precision, dimension, largest tables),
  // time each candidate launch shape (threads per CTA, histories per work
  // item, all or half the CTAs per SM that fit) on the same problems with an
  // eighth of the histories and keep the fastest
  uint64_t total = 0;
  int maxM = 0, maxG = 0, maxT = 0;
  for (int i = 0; i < n; ++i) {
    if (!probs[i]) return fail(MCDC_ERR_INVALID, "problem is NULL");
    total += n_histories[i];
    maxM = std::max(maxM, probs[i]->P.M);
    maxG = std::max(maxG, probs[i]->P.G);
    maxT = std::max(maxT, probs[i]->P.T);
  }
  int lg = 0;
  while ((1ull << lg) < total && lg < 63) ++lg;
  char kb[160];
  snprintf(kb, sizeof kb, "%d|%d|%d|%d|%d|%d|%d|%d|%d", n, lg, (int)probs[0]->key.f64,
           (int)probs[0]->key.local, probs[0]->dim, maxM, maxG, maxT, n_batches);
  BatchedShape best{256, 1ull << 16, 0};
  bool have = false;
  {
    std::lock_guard<std::mutex> lk(g_batched_mu);
    auto it = g_batched_cache.find(kb);
    if (it != g_batched_cache.end()) { best = it->second; have = true; }
  }
  if (!have) {
    const int B = n_batches > 0 ? n_batches : 16;
    std::vector<uint64_t> trial(n);
    for (int i = 0; i < n; ++i) trial[i] = std::max<uint64_t>((uint64_t)B, n_histories[i] / 8);
    double best_ms = 1e300;
    bool any = false;
    for (int block : {128, 256, 512})
      for (unsigned long long chunk : {1ull << 14, 1ull << 16}) {
        int full_cps = 0;       // CTAs per SM of the full-occupancy trial
        for (int half : {0, 1}) {
          int cps = 0;
          if (half) {
            if (full_cps < 2) continue;
            cps = full_cps / 2;
          }
          mcdc_stats st{};
          const int rc = run_batched(probs, n, trial.data(), seed ^ 0x5bd1e995ull, n_batches,
                                     nullptr, nullptr, nullptr, &st, block, chunk, cps, false);
          if (rc == MCDC_ERR_INVALID) { mcdc::set_error(MCDC_OK, ""); continue; }   // does not fit
          if (rc != MCDC_OK) return rc;
          if (!half) full_cps = st.ctas_per_sm;
          any = true;
          if (st.kernel_ms < best_ms) { best_ms = st.kernel_ms; best = {block, chunk, cps}; }
        }
      }
    if (!any) best = {256, 1ull << 16, 0};
    std::lock_guard<std::mutex> lk(g_batched_mu);
    g_batched_cache[kb] = best;
  }
  return run_batched(probs, n, n_histories, seed, n_batches, mean_out, relerr_out, scalar_out, stats,
                     best.block, best.chunk, best.cps);
}

namespace mcdc {
void batched_forget(uint64_t uid) {
  std::vector<std::unique_ptr<BatchedPlan>> gone;
  {
    std::lock_guard<std::mutex> lk(g_plan_mu);
    for (size_t k = 0; k < g_plans.size();) {
      const auto &u = g_plans[k]->uids;
      if (std::find(u.begin(), u.end(), uid) != u.end()) {
        gone.push_back(std::move(g_plans[k]));
        g_plans.erase(g_plans.begin() + (long)k);
      } else {
        ++k;
      }
    }
  }
}
}  // namespace mcdc
