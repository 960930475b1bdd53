// api.cu -- the C-ABI (include/mcdc.h): problem validation, device tables,
// launch-shape selection and the run sequence.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include "../../include/mcdc.h"
#include "launch.h"
#include "comb.h"
#include "problem.h"
#include "tracker.cuh"

using namespace mcdc;

static_assert(sizeof(mcdc_record) == sizeof(Record), "record layout");

namespace {

thread_local std::string g_err;

int fail(int code, const std::string &msg) {
  g_err = msg;
  return code;
}

#define CK(call)                                                                      \
  do {                                                                                \
    cudaError_t e_ = (call);                                                          \
    if (e_ != cudaSuccess)                                                            \
      return fail(e_ == cudaErrorMemoryAllocation ? MCDC_ERR_OOM : MCDC_ERR_CUDA,     \
                  std::string(#call) + ": " + cudaGetErrorString(e_));                \
  } while (0)

bool finite_nonneg(double v) { return std::isfinite(v) && v >= 0.0; }

bool is_device_ptr(const void *p) {
  if (p == nullptr) return false;
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// device buffers owned by a problem
struct DevBuf {
  void *p = nullptr;
  size_t bytes = 0;
};

}  // namespace


namespace {

// Problems take their device memory from one stream-ordered pool per device
// that keeps up to 16 GiB of freed memory mapped (a global-tally problem's
// batch slices alone can take 8 GiB), so a loop that creates,
// runs and destroys problems (a serving loop) reuses it instead of paying
// the driver's allocation and page mapping on every create and first run.
// The pool's own non-blocking stream orders allocations and frees; each
// allocation is complete (synchronised) before its pointer is handed out,
// and a problem's memory is returned only after the device is idle.  Where
// pools are unavailable, plain cudaMalloc is used.
struct DevPool {
  cudaMemPool_t pool = nullptr;
  cudaStream_t stream = nullptr;
  bool ok = false;
};
std::mutex g_pool_mu;
std::map<int, DevPool> g_pools;

DevPool device_pool(int dev) {
  std::lock_guard<std::mutex> lk(g_pool_mu);
  auto it = g_pools.find(dev);
  if (it != g_pools.end()) return it->second;
  DevPool d;
  int supported = 0;
  cudaMemPoolProps props;
  std::memset(&props, 0, sizeof props);
  props.allocType = cudaMemAllocationTypePinned;
  props.handleTypes = cudaMemHandleTypeNone;
  props.location.type = cudaMemLocationTypeDevice;
  props.location.id = dev;
  if (cudaDeviceGetAttribute(&supported, cudaDevAttrMemoryPoolsSupported, dev) == cudaSuccess &&
      supported && cudaMemPoolCreate(&d.pool, &props) == cudaSuccess) {
    uint64_t keep = 16ull << 30;
    if (cudaMemPoolSetAttribute(d.pool, cudaMemPoolAttrReleaseThreshold, &keep) == cudaSuccess &&
        cudaStreamCreateWithFlags(&d.stream, cudaStreamNonBlocking) == cudaSuccess) {
      d.ok = true;
    } else {
      cudaMemPoolDestroy(d.pool);
      d.pool = nullptr;
    }
  }
  cudaGetLastError();
  g_pools[dev] = d;
  return d;
}

template <class T>
int dalloc(mcdc_problem *pr, T **out, size_t count) {
  void *p = nullptr;
  const size_t bytes = std::max<size_t>(count * sizeof(T), 16);
  const DevPool d = device_pool(pr->device);
  cudaError_t e;
  if (d.ok) {
    e = cudaMallocFromPoolAsync(&p, bytes, d.pool, d.stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(d.stream);
  } else {
    e = cudaMalloc(&p, bytes);
  }
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(MCDC_ERR_OOM, "device allocation of " + std::to_string(bytes) + " bytes failed");
  }
  (d.ok ? pr->pool_allocs : pr->allocs).push_back(p);
  *out = (T *)p;
  return MCDC_OK;
}

// Returns a buffer from dalloc to the device's pool (or frees it) once the
// device has finished with it.
void dfree(mcdc_problem *pr, void *p) {
  if (!p) return;
  cudaDeviceSynchronize();
  auto &pa = pr->pool_allocs;
  for (size_t i = 0; i < pa.size(); ++i) {
    if (pa[i] == p) {
      cudaFreeAsync(p, device_pool(pr->device).stream);
      pa.erase(pa.begin() + (long)i);
      cudaGetLastError();
      return;
    }
  }
  auto &al = pr->allocs;
  for (size_t i = 0; i < al.size(); ++i) {
    if (al[i] == p) {
      cudaFree(p);
      al.erase(al.begin() + (long)i);
      break;
    }
  }
  cudaGetLastError();
}

// A problem's tables and accumulators in one device allocation: uploads are
// gathered in a host buffer and copied once, device-only arrays follow them
// and are zeroed once (a create is a handful of API calls, not dozens).
struct Arena {
  std::vector<unsigned char> host;
  size_t device_bytes = 0;
  std::vector<std::pair<void **, size_t>> up, dev;   // field, offset
  static size_t round(size_t v) { return (v + 255) & ~size_t(255); }
  template <class T>
  void upload(const T **field, const std::vector<T> &src) {
    const size_t off = round(host.size());
    host.resize(off + std::max<size_t>(src.size() * sizeof(T), 16));
    if (!src.empty()) std::memcpy(host.data() + off, src.data(), src.size() * sizeof(T));
    up.push_back({reinterpret_cast<void **>(const_cast<T **>(field)), off});
  }
  template <class T>
  void device(T **field, size_t count) {
    const size_t off = round(device_bytes);
    device_bytes = off + std::max<size_t>(count * sizeof(T), 16);
    dev.push_back({reinterpret_cast<void **>(field), off});
  }
  int commit(mcdc_problem *pr) {
    const size_t hb = round(host.size());
    unsigned char *base = nullptr;
    if (dalloc(pr, &base, hb + device_bytes)) return MCDC_ERR_OOM;
    CK(cudaMemcpy(base, host.data(), host.size(), cudaMemcpyHostToDevice));
    if (device_bytes) CK(cudaMemset(base + hb, 0, device_bytes));
    for (auto &f : up) *f.first = base + f.second;
    for (auto &f : dev) *f.first = base + hb + f.second;
    return MCDC_OK;
  }
};

// Pinned host words a run reads back (statistics, error flags, a count),
// from a process-wide pool: pinned allocation costs far more than a run's
// setup, so blocks are allocated 16 at a time, reused across problems and
// kept until exit.
struct PinnedBlock {
  Stats stats;
  int32_t error[4];
  unsigned long long count;
};
std::mutex g_pin_mu;
std::vector<PinnedBlock *> g_pin_free;

PinnedBlock *pinned_get() {
  {
    std::lock_guard<std::mutex> lk(g_pin_mu);
    if (!g_pin_free.empty()) {
      PinnedBlock *b = g_pin_free.back();
      g_pin_free.pop_back();
      return b;
    }
  }
  constexpr int kSlab = 16;
  void *p = nullptr;
  if (cudaMallocHost(&p, kSlab * sizeof(PinnedBlock)) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  PinnedBlock *slab = static_cast<PinnedBlock *>(p);
  std::lock_guard<std::mutex> lk(g_pin_mu);
  for (int q = kSlab - 1; q >= 1; --q) g_pin_free.push_back(slab + q);
  return slab;
}

void pinned_put(PinnedBlock *b) {
  if (!b) return;
  std::lock_guard<std::mutex> lk(g_pin_mu);
  g_pin_free.push_back(b);
}

void release(mcdc_problem *pr) {
  if (!pr) return;
  if (pr->uid) mcdc::batched_forget(pr->uid);
  cudaSetDevice(pr->device);
  for (void *p : pr->allocs) cudaFree(p);
  pr->allocs.clear();
  if (!pr->pool_allocs.empty()) {
    // no kernel of this problem may still use the memory (cudaFree above
    // waits for the device the same way)
    cudaDeviceSynchronize();
    const DevPool d = device_pool(pr->device);
    for (void *p : pr->pool_allocs) cudaFreeAsync(p, d.stream);
    pr->pool_allocs.clear();
  }
  cudaGetLastError();
  if (pr->ev0) cudaEventDestroy(pr->ev0);
  if (pr->ev1) cudaEventDestroy(pr->ev1);
  if (pr->ev2) cudaEventDestroy(pr->ev2);
  pinned_put(static_cast<PinnedBlock *>(pr->pinned));
  delete pr;
}

void build_cdf(const double *pdf, int n, double *cdf) {
  double acc = 0.0;
  int last = 0;
  for (int k = 0; k < n; ++k) {
    acc += pdf[k];
    cdf[k] = acc;
    if (pdf[k] > 0.0) last = k;
  }
  for (int k = last; k < n; ++k) cdf[k] = 1.0;
}

// Shared memory one CTA needs for a given slot count.
Layout make_layout(const mcdc_problem *pr, int S, int tally_mode) {
  Layout L{};
  L.M = pr->P.M;
  L.G = pr->P.G;
  L.T = pr->P.T;
  L.S = S;
  const bool f64 = pr->key.f64;
  L.tables_bytes = tables_bytes_of(f64, pr->P.M, pr->P.G, pr->P.T);
  L.tally_bytes = tally_mode == MCDC_TALLY_SHARED
                      ? align16((long long)pr->P.n_tally * (f64 ? 8 : 4))
                      : 0;
  L.bank_bytes = S * slot_bytes(f64, pr->dim, pr->key.local);
  L.net_bytes = (pr->key.net && !f64) ? kNetFragBytes + (S / kPool) * kNetWarpBytes : 0;
  L.total = (int)(L.tables_bytes + L.tally_bytes + L.bank_bytes + L.net_bytes + 64);
  return L;
}

struct DeviceLimits {
  int sms, smem_sm, smem_block, max_threads_sm;
};

int device_limits(int dev, DeviceLimits *d) {
  CK(cudaDeviceGetAttribute(&d->sms, cudaDevAttrMultiProcessorCount, dev));
  CK(cudaDeviceGetAttribute(&d->smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev));
  CK(cudaDeviceGetAttribute(&d->smem_block, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
  CK(cudaDeviceGetAttribute(&d->max_threads_sm, cudaDevAttrMaxThreadsPerMultiProcessor, dev));
  return MCDC_OK;
}

// Picks block size, slots, CTAs per SM and the tally mode from the options
// and the device limits.  Shared mode needs the whole tally plus the bank in
// one CTA's shared memory.
int choose_shape(mcdc_problem *pr, const DeviceLimits &dl) {
  const mcdc_options &o = pr->opt;
  const bool f64 = pr->key.f64;
  int block = o.block_size > 0 ? o.block_size : 256;
  if (block % 32 != 0 || block > 512) return fail(MCDC_ERR_INVALID, "block_size must be a multiple of 32, <= 512");
  // the network instantiations are built for at most kNetBlockMax threads:
  // they take that many (their registers allow one such CTA per SM) unless
  // the caller asked for fewer
  if (pr->key.net) block = pr->user_block > 0 ? std::min(pr->user_block, kNetBlockMax) : kNetBlockMax;
  // every warp parks up to kPool particles besides its 32 in flight
  const int S = (block / 32) * kPool;
  int mode = o.tally_mode;
  const long long tally_b = (long long)pr->P.n_tally * (f64 ? 8 : 4);
  if (mode == MCDC_TALLY_AUTO) {
    const Layout Ls = make_layout(pr, S, MCDC_TALLY_SHARED);
    mode = (tally_b <= 96 * 1024 && Ls.total <= dl.smem_block - 1024) ? MCDC_TALLY_SHARED
                                                                       : MCDC_TALLY_GLOBAL;
  }
  Layout L = make_layout(pr, S, mode);
  const int dyn_max = dl.smem_block - 1024;   // room for the kernel's static shared memory
  pr->dyn_max = dyn_max;
  if (L.total > dyn_max) {
    if (o.tally_mode == MCDC_TALLY_SHARED)
      return fail(MCDC_ERR_INVALID, "shared tally + bank exceed shared memory; use the global tally");
    return fail(MCDC_ERR_INVALID, "block_size too large for shared memory");
  }
  pr->key.shared = (mode == MCDC_TALLY_SHARED);
  {
    cudaError_t e = prepare_track(pr->key, dyn_max);
    if (e != cudaSuccess) return fail(MCDC_ERR_CUDA, std::string("cudaFuncSetAttribute: ") + cudaGetErrorString(e));
  }
  int cps = track_occupancy(pr->key, block, L.total);
  if (cps < 1) return fail(MCDC_ERR_INVALID, "launch shape does not fit on an SM (registers or shared memory)");
  if (o.ctas_per_sm > 0) {
    // the tuner's choice for another instantiation: as many as fit when fewer
    // fit here; the caller's own choice must fit
    if (o.ctas_per_sm > cps && (pr->user_cps > 0 || !pr->key.net))
      return fail(MCDC_ERR_INVALID, "ctas_per_sm exceeds what fits on an SM");
    cps = std::min(cps, o.ctas_per_sm);
  }
  pr->block = block;
  pr->S = S;
  pr->ctas_per_sm = cps;
  pr->grid = dl.sms * cps;
  pr->smem = L.total;
  pr->L = L;
  pr->tally_mode = mode;
  if (o.warp_aggregate > 0) pr->warp_aggregate = 1;
  else if (o.warp_aggregate < 0) pr->warp_aggregate = 0;
  else pr->warp_aggregate = pr->P.n_bins <= 4096 ? 1 : 0;
  pr->key.shared = (mode == MCDC_TALLY_SHARED);
  return MCDC_OK;
}

int default_batches(const mcdc_problem *pr, uint64_t n) {
  int B = pr->opt.n_batches;
  if (B <= 0) {
    if (pr->tally_mode == MCDC_TALLY_SHARED) {
      // every CTA gets about two whole batches (a CTA drains between its
      // batches), each of at least a few thousand histories
      const uint64_t by_size = n / 4096;
      B = (int)std::min<uint64_t>(std::max<uint64_t>(by_size, 32),
                                  (uint64_t)pr->grid * (uint64_t)pr->batch_per_cta);
    } else {
      B = 32;
    }
  }
  if ((uint64_t)B > n) B = (int)n;
  return B;
}

// One zeroed device tally slice per batch, for runs that put every batch in
// one launch (population control, weight-window runs).
// Growing them returns the smaller buffers first, so a problem never holds
// two generations of slices.
// The FP32 modes score into FP32 slices (half the memory and atomic traffic,
// and no FP32-to-FP64 conversion on the FP64 pipe per score); the fold sums
// the batches in FP64.
int ensure_slices(mcdc_problem *pr, int B) {
  const long long bins = (long long)B * pr->P.n_tally;
  if (pr->pc_tally_bins >= bins) return MCDC_OK;
  dfree(pr, pr->pc_tally);
  dfree(pr, pr->slice_rb);
  pr->pc_tally = nullptr;
  pr->slice_rb = nullptr;
  pr->pc_tally_bins = 0;
  pr->slices_dirty = false;
  pr->slice_bytes = pr->key.f64 ? 8 : 4;
  int rc;
  unsigned char *t = nullptr;
  if ((rc = dalloc(pr, &t, (size_t)bins * pr->slice_bytes))) return rc;
  pr->pc_tally = t;
  if ((rc = dalloc(pr, &pr->slice_rb, (size_t)(2 * B)))) return rc;
  if (cudaMemset(pr->pc_tally, 0, (size_t)pr->slice_bytes * (size_t)bins) != cudaSuccess ||
      cudaMemset(pr->slice_rb, 0, sizeof(double) * (size_t)(2 * B)) != cudaSuccess)
    return fail(MCDC_ERR_CUDA, "cudaMemset of the tally slices failed");
  pr->pc_tally_bins = bins;
  return MCDC_OK;
}

// Folds the B tally slices of a one-launch run: one pass over the bins when
// the per-batch region partials fit a block's shared memory, else slice by
// slice.
template <class ST>
cudaError_t fold_slices_as(mcdc_problem *pr, cudaStream_t s, const DevProblem &P, ST *slices,
                           size_t nt, int B) {
  if (B <= 2048)
    return launch_fold_slices(s, P, slices, (long long)nt, B, pr->sum1, pr->sum2, pr->sum12,
                              pr->slice_rb, pr->region, pr->sms);
  for (int b = 0; b < B; ++b) {
    cudaError_t e = launch_fold(s, P, slices + (size_t)b * nt, pr->sum1, pr->sum2, pr->sum12,
                                pr->region_batch, pr->region, pr->sms);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}
cudaError_t fold_slices(mcdc_problem *pr, cudaStream_t s, const DevProblem &P, size_t nt, int B) {
  if (pr->slice_bytes == 4)
    return fold_slices_as(pr, s, P, static_cast<float *>(pr->pc_tally), nt, B);
  return fold_slices_as(pr, s, P, static_cast<double *>(pr->pc_tally), nt, B);
}
// the tracker's arguments for scoring into the slices
void use_slices(const mcdc_problem *pr, RunArgs &A) {
  if (pr->slice_bytes == 4) {
    A.tally = nullptr;
    A.tally32 = static_cast<float *>(pr->pc_tally);
  } else {
    A.tally = static_cast<double *>(pr->pc_tally);
    A.tally32 = nullptr;
  }
}

// Population control buffers: a census bank of cap particles, a combed
// bank of combed particles, B tally slices and the comb's scratch.
int ensure_pc(mcdc_problem *pr, int cap, long long combed, int B) {
  const size_t pb = bank_slot_bytes(pr->key);
  int rc;
  if (pr->pc_cap < cap) {
    unsigned char *bank = nullptr, *temp = nullptr;
    if ((rc = dalloc(pr, &bank, pb * (size_t)cap))) return rc;
    if ((rc = dalloc(pr, &pr->pc_w, (size_t)cap))) return rc;
    if ((rc = dalloc(pr, &pr->pc_S, (size_t)cap))) return rc;
    if ((rc = dalloc(pr, &pr->pc_key, (size_t)cap))) return rc;
    const size_t tb = comb_temp_bytes(cap);
    if ((rc = dalloc(pr, &temp, tb))) return rc;
    pr->pc_bank = bank;
    pr->pc_temp = temp;
    pr->pc_temp_bytes = tb;
    pr->pc_cap = cap;
  }
  if (pr->pc_combed_cap < combed) {
    unsigned char *c = nullptr;
    if ((rc = dalloc(pr, &c, pb * (size_t)combed))) return rc;
    pr->pc_combed = c;
    pr->pc_combed_cap = combed;
  }
  if (pr->pc_seg_cap < B) {
    if ((rc = dalloc(pr, &pr->pc_seg, 3 * (size_t)B))) return rc;
    if ((rc = dalloc(pr, &pr->pc_segd, 4 * (size_t)B))) return rc;
    if ((rc = dalloc(pr, &pr->pc_live, 2 * (size_t)B + 2))) return rc;
    pr->pc_seg_cap = B;
  }
  if ((rc = ensure_slices(pr, B))) return rc;
  if (!pr->pc_cnt && (rc = dalloc(pr, &pr->pc_cnt, 4))) return rc;
  return MCDC_OK;
}

int ensure_work_slots(mcdc_problem *pr, int n) {
  if (pr->work_slots >= n) return MCDC_OK;
  unsigned long long *w = nullptr;
  int rc = dalloc(pr, &w, (size_t)n);
  if (rc) return rc;
  pr->work = w;
  pr->work_slots = n;
  return MCDC_OK;
}

int ensure_overflow(mcdc_problem *pr) {
  if (!ww_on(pr->P)) return MCDC_OK;
  const int warps = pr->block / 32;
  int cap = pr->opt.overflow_per_cta > 0 ? std::max(64, pr->opt.overflow_per_cta / warps) : 1024;
  if (pr->tally_mode == MCDC_TALLY_GLOBAL) {
    // a small stack per warp (64 by default); the rest spills to the
    // device-wide banks so a large family of split children is shared by
    // every warp in the next pass instead of keeping one warp busy (on the
    // deep-penetration box 64 per warp ran 3-5x faster than 256)
    cap = pr->opt.overflow_per_cta > 0 ? std::min(cap, 256) : 64;
    if (!pr->spill[0]) {
      // particles per bank (2^26 by default: 4.3 GB in FP32)
      const unsigned long long scap =
          pr->opt.spill_particles > 0 ? (unsigned long long)pr->opt.spill_particles : 1ull << 26;
      const size_t pb = pr->key.f64 ? sizeof(Part<double>)
                        : (pr->key.local ? sizeof(Part<float, float>) : sizeof(Part<float>));
      unsigned char *a = nullptr, *b = nullptr;
      unsigned long long *c = nullptr;
      int rc;
      if ((rc = dalloc(pr, &a, scap * pb))) return rc;
      if ((rc = dalloc(pr, &b, scap * pb))) return rc;
      if ((rc = dalloc(pr, &c, 4))) return rc;
      pr->spill[0] = a;
      pr->spill[1] = b;
      pr->spill_cnt = c;
      pr->spill_cap = scap;
    }
  }
  const size_t part_b = pr->key.f64 ? sizeof(Part<double>)
                       : (pr->key.local ? sizeof(Part<float, float>) : sizeof(Part<float>));
  const size_t need = (size_t)pr->grid * warps * cap * part_b;
  if (pr->overflow_bytes >= need && pr->overflow_cap == cap) return MCDC_OK;
  unsigned char *p = nullptr;
  int rc = dalloc(pr, &p, need);
  if (rc) return rc;
  pr->overflow = p;
  pr->overflow_bytes = need;
  pr->overflow_cap = cap;
  return MCDC_OK;
}

// ---- autotuner ---------------------------------------------------------------
// Times candidate launch shapes on the problem itself -- threads per CTA
// (which sets the CTA's particle bank: warps x 96 parked slots plus one
// flying particle per lane), resident CTAs per SM (all that fit, or half),
// whole batches per CTA in the shared-tally mode, and warp aggregation of
// tally atomics -- and keeps the fastest.  Choices are cached per problem
// shape for the life of the process.  (The 96 parked slots per warp are not
// a tuning choice: the scheduler never parks more than 94, and fewer slots
// would break that bound.)
struct TuneChoice {
  int block, batch_per_cta, aggregate;
  int cps;      // resident CTAs per SM; 0: as many as fit
};
std::mutex g_tune_mu;
std::map<std::string, TuneChoice> g_tune_cache;

std::string tune_key(const mcdc_problem *pr) {
  const DevProblem &P = pr->P;
  char b[256];
  snprintf(b, sizeof b, "%d|%d|%d|%d|%d|%d|%d|%lld|%d|%d|%d|%d|%d|%d|%d|%d|%d|%d",
           (int)pr->key.f64, (int)pr->key.local, pr->dim, pr->tally_mode, P.M, P.G, P.T,
           (long long)P.n_bins, P.n[0], P.n[1], P.n[2], pr->sms, P.estimator, P.implicit,
           P.fresh_tau, (int)pr->key.net * 2 + (int)pr->key.vr, pr->user_aggregate, pr->user_cps);
  return b;
}

int apply_choice(mcdc_problem *pr, const DeviceLimits &dl, const TuneChoice &c) {
  pr->opt.block_size = c.block;
  pr->opt.warp_aggregate = c.aggregate ? 1 : -1;
  pr->opt.tally_mode = pr->tally_mode;
  pr->opt.ctas_per_sm = c.cps;
  pr->batch_per_cta = c.batch_per_cta;
  return choose_shape(pr, dl);
}

}  // namespace

extern "C" int mcdc_run_ex(struct mcdc_problem *pr, const mcdc_run_args *a, mcdc_stats *stats);

namespace {
int autotune(mcdc_problem *pr, const DeviceLimits &dl) {
  NvtxRange nvtx("autotune");
  const std::string key = tune_key(pr);
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tune_cache.find(key);
    if (it != g_tune_cache.end()) return apply_choice(pr, dl, it->second);
  }
  const bool shared = pr->tally_mode == MCDC_TALLY_SHARED;
  std::vector<TuneChoice> cand;
  for (int b : {128, 256, 512}) {
    // CTAs per SM: all that fit, and half of them when that is at least one
    const int full = track_occupancy(pr->key, b, make_layout(pr, (b / 32) * kPool, pr->tally_mode).total);
    // the caller's own choices (warp aggregation on or off, CTAs per SM) are
    // kept; the tuner chooses only what was left to it
    std::vector<int> cps{0};
    if (pr->user_cps > 0) cps = {pr->user_cps};
    else if (full >= 2) cps.push_back(full / 2);
    std::vector<int> aggs = pr->P.n_bins <= 65536 ? std::vector<int>{0, 1} : std::vector<int>{0};
    if (pr->user_aggregate != 0) aggs = {pr->user_aggregate > 0 ? 1 : 0};
    for (int c : cps)
      for (int bpc : shared ? std::vector<int>{1, 2, 4} : std::vector<int>{2})
        for (int agg : aggs) cand.push_back({b, bpc, agg, c});
  }
  const TuneChoice keep{pr->block, pr->batch_per_cta, pr->warp_aggregate, pr->opt.ctas_per_sm};
  const uint64_t n_trial = 1ull << 20;
  double best_t = 1e300;
  TuneChoice best = keep;
  for (const TuneChoice &c : cand) {
    if (apply_choice(pr, dl, c) != MCDC_OK) { g_err.clear(); continue; }
    mcdc_run_args a;
    std::memset(&a, 0, sizeof a);
    a.n_histories = n_trial;
    a.seed = 0x5eed;
    a.n_batches = shared ? 0 : 8;
    mcdc_stats st;
    double t = 0.0;
    bool ok = true;
    for (int rep = 0; rep < 2 && ok; ++rep) {
      a.hist_offset = (uint64_t)rep * n_trial;
      ok = mcdc_run_ex(pr, &a, &st) == MCDC_OK;
      t = st.kernel_ms;
    }
    if (ok && t < best_t) { best_t = t; best = c; }
    g_err.clear();
  }
  if (int rc = apply_choice(pr, dl, best)) return rc;
  std::lock_guard<std::mutex> lk(g_tune_mu);
  g_tune_cache[key] = best;
  return MCDC_OK;
}

}  // namespace

namespace {
// Switches the problem between the tracker built with and without the
// per-event network evaluation and redoes the launch shape for it (registers
// and so CTAs per SM may differ).
// IEEE binary16 of an FP32 value, rounded to nearest with ties to even
// (finite inputs below the binary16 overflow threshold; subnormals kept)
uint16_t f16_rne(float v) {
  uint32_t u;
  std::memcpy(&u, &v, 4);
  const uint32_t sign = (u >> 16) & 0x8000u, mant = u & 0x7fffffu;
  const int e = (int)((u >> 23) & 0xffu) - 127 + 15;   // binary16 biased exponent
  uint32_t q, rem, half;
  if (e >= 1) {                 // normal: 10 fraction bits, 13 dropped
    q = ((uint32_t)e << 10) | (mant >> 13);
    rem = mant & 0x1fffu;
    half = 0x1000u;
  } else {                      // subnormal: value / 2^-24, from the full significand
    const int shift = 14 - e;
    if (shift > 24) return (uint16_t)sign;
    const uint32_t sig = mant | 0x800000u;
    q = sig >> shift;
    rem = sig & ((1u << shift) - 1u);
    half = 1u << (shift - 1);
  }
  if (rem > half || (rem == half && (q & 1u))) q += 1u;   // a carry moves the exponent up
  return (uint16_t)(sign | q);
}

// The network (layout of mcdc_mlp_forward: W1[H][in], b1, W2[H][H], b2, W3, b3)
// as the tracker's fragment block: for n-tile j, K step s and lane L (column
// g = L / 4 of the tile's 8, pair t = L % 4), the two words of the mma.sync
// m16n8k16 B fragment, {B[16s+2t][g], B[16s+2t+1][g]} and {B[16s+2t+8][g],
// B[16s+2t+9][g]} in binary16 (the lower index in the low half), with
// B[k][g] = W[8j+g][k] / 2 for layers 1 and 2 and B[k][0] = W3[k] (other
// columns zero) for the output layer, zero outside the network; b1 / 2 and
// b2 / 2 in FP32, padded to 64.
std::vector<uint32_t> net_fragments(const float *prm, int in, int H) {
  std::vector<uint32_t> f(kNetFragWords, 0u);
  const float *W1 = prm, *b1 = W1 + (size_t)H * in, *W2 = b1 + H, *b2 = W2 + (size_t)H * H,
              *W3 = b2 + H;
  auto w1 = [&](int n, int k) { return (n < H && k < in) ? 0.5f * W1[n * in + k] : 0.0f; };
  auto w2 = [&](int n, int k) { return (n < H && k < H) ? 0.5f * W2[n * H + k] : 0.0f; };
  auto w3 = [&](int n, int k) { return (n == 0 && k < H) ? W3[k] : 0.0f; };
  auto pair = [](float lo, float hi) {
    return (uint32_t)f16_rne(lo) | ((uint32_t)f16_rne(hi) << 16);
  };
  for (int L = 0; L < 32; ++L) {
    const int g = L / 4, t = L % 4;
    for (int j = 0; j < 8; ++j) {
      const int n = 8 * j + g;
      for (int s = 0; s < 2; ++s) {
        const int k = 16 * s + 2 * t, at = kNetW1Frag + ((j * 2 + s) * 32 + L) * 2;
        f[at] = pair(w1(n, k), w1(n, k + 1));
        f[at + 1] = pair(w1(n, k + 8), w1(n, k + 9));
      }
      for (int s = 0; s < 4; ++s) {
        const int k = 16 * s + 2 * t, at = kNetW2Frag + ((j * 4 + s) * 32 + L) * 2;
        f[at] = pair(w2(n, k), w2(n, k + 1));
        f[at + 1] = pair(w2(n, k + 8), w2(n, k + 9));
      }
    }
    for (int s = 0; s < 4; ++s) {
      const int k = 16 * s + 2 * t, at = kNetW3Frag + (s * 32 + L) * 2;
      f[at] = pair(w3(g, k), w3(g, k + 1));
      f[at + 1] = pair(w3(g, k + 8), w3(g, k + 9));
    }
  }
  for (int n = 0; n < H; ++n) {
    const float h1 = 0.5f * b1[n], h2 = 0.5f * b2[n];
    std::memcpy(&f[kNetB1 + n], &h1, 4);
    std::memcpy(&f[kNetB2 + n], &h2, 4);
  }
  return f;
}

// Switches the problem's tracker instantiation: with the per-event network
// evaluation (net), with the window checks of a table (ww) -- or implicit
// capture, which also varies weights --, or analog; the
// launch shape is redone for it (registers, so CTAs per SM, may differ).
int set_track_kernel_impl(mcdc_problem *pr, bool net, bool ww) {
  const bool vr = ww || pr->P.implicit != 0;     // implicit capture varies weights too
  if (pr->key.net == net && pr->key.vr == vr) return MCDC_OK;
  pr->key.net = net;
  pr->key.vr = vr;
  DeviceLimits dl;
  if (int rc = device_limits(pr->device, &dl)) return rc;
  pr->opt.tally_mode = pr->tally_mode;
  return choose_shape(pr, dl);
}
}  // namespace

namespace mcdc {
int set_error(int code, const std::string &msg) { return fail(code, msg); }
int set_track_kernel(mcdc_problem *pr, bool net, bool ww) { return set_track_kernel_impl(pr, net, ww); }
int ensure_overflow_for(mcdc_problem *pr) { return ensure_overflow(pr); }
cudaMemPool_t device_mem_pool(int dev) {
  const DevPool d = device_pool(dev);
  return d.ok ? d.pool : nullptr;
}
}  // namespace mcdc

extern "C" {

void mcdc_default_options(mcdc_options *o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->precision = MCDC_PREC_FP32;
  o->tally_mode = MCDC_TALLY_AUTO;
  o->autotune = 1;
  o->estimator = MCDC_EST_TRACK;
  o->weight_cutoff = 0.25;
  o->cutoff_survival = 0.5;
  o->overflow_tail = 8;
}

const char *mcdc_last_error(void) { return g_err.c_str(); }

int mcdc_problem_create(const mcdc_mesh *mesh, const mcdc_materials *mat, const mcdc_source *src,
                        const mcdc_time_grid *time, const mcdc_options *opt,
                        struct mcdc_problem **out) {
  NvtxRange nvtx("mcdc_problem_create");
  g_err.clear();
  if (!out) return fail(MCDC_ERR_INVALID, "out is NULL");
  *out = nullptr;
  if (!mesh || !mat || !src) return fail(MCDC_ERR_INVALID, "mesh, materials and source are required");
  mcdc_options o;
  if (opt) o = *opt; else mcdc_default_options(&o);
  if (o.precision != MCDC_PREC_FP64 && o.precision != MCDC_PREC_FP32 &&
      o.precision != MCDC_PREC_FP32_LOCAL)
    return fail(MCDC_ERR_INVALID, "unknown precision");
  if (o.estimator != MCDC_EST_TRACK && o.estimator != MCDC_EST_COLLISION &&
      o.estimator != MCDC_EST_COMBINED)
    return fail(MCDC_ERR_INVALID, "unknown estimator");
  if (o.implicit_capture != 0 && o.implicit_capture != 1)
    return fail(MCDC_ERR_INVALID, "implicit_capture must be 0 or 1");
  if (o.implicit_capture &&
      !(std::isfinite(o.cutoff_survival) && o.weight_cutoff > 0.0 && o.cutoff_survival > o.weight_cutoff))
    return fail(MCDC_ERR_INVALID, "implicit capture needs 0 < weight_cutoff < cutoff_survival");
  if (o.pc_target < 0) return fail(MCDC_ERR_INVALID, "pc_target must be >= 0");
  if (o.flight_sampling != 0 && o.flight_sampling != 1)
    return fail(MCDC_ERR_INVALID, "flight_sampling must be 0 or 1");
  if (o.overflow_tail < -1) return fail(MCDC_ERR_INVALID, "overflow_tail must be >= -1");
  if (o.spill_particles < 0 || o.spill_particles > (1ll << 31))
    return fail(MCDC_ERR_INVALID, "spill_particles must be in 0..2^31");
  if (o.pc_target > 0 && o.tally_mode == MCDC_TALLY_SHARED)
    return fail(MCDC_ERR_INVALID, "population control runs on the global tally");

  // ---- mesh
  const int n[3] = {mesh->nx, mesh->ny, mesh->nz};
  const double org[3] = {mesh->x0, mesh->y0, mesh->z0};
  const double wid[3] = {mesh->dx, mesh->dy, mesh->dz};
  int bounded[3];
  for (int a = 0; a < 3; ++a) {
    if (n[a] < 1 || n[a] > 65535) return fail(MCDC_ERR_INVALID, "cells per axis must be in 1..65535");
    bounded[a] = !(n[a] == 1 && (!(wid[a] > 0.0) || std::isinf(wid[a])));
    if (bounded[a] && !(std::isfinite(wid[a]) && wid[a] > 0.0))
      return fail(MCDC_ERR_INVALID, "cell widths must be finite and > 0");
    if (!std::isfinite(org[a])) return fail(MCDC_ERR_INVALID, "mesh origin must be finite");
  }
  if (!mesh->material) return fail(MCDC_ERR_INVALID, "material map is NULL");
  for (int s = 0; s < 6; ++s)
    if (mesh->bc[s] != MCDC_BC_VACUUM && mesh->bc[s] != MCDC_BC_REFLECT)
      return fail(MCDC_ERR_INVALID, "unknown boundary condition");
  const int64_t n_cells = (int64_t)n[0] * n[1] * n[2];

  // ---- materials
  const int M = mat->n_materials, G = mat->n_groups;
  if (M < 1 || M > 255) return fail(MCDC_ERR_INVALID, "n_materials must be in 1..255");
  if (G < 1 || G > kMaxGroups) return fail(MCDC_ERR_INVALID, "n_groups must be in 1..16");
  if (!mat->sigma_t || !mat->sigma_s || !mat->transfer || !mat->speed)
    return fail(MCDC_ERR_INVALID, "material arrays must not be NULL");
  for (int64_t c = 0; c < n_cells; ++c)
    if (mesh->material[c] >= M) return fail(MCDC_ERR_INVALID, "material id out of range");
  std::vector<double> st(M * G), scat(M * G), cdf((size_t)M * G * G);
  for (int m = 0; m < M; ++m)
    for (int g = 0; g < G; ++g) {
      const double t = mat->sigma_t[m * G + g], s = mat->sigma_s[m * G + g];
      if (!finite_nonneg(t) || !finite_nonneg(s) || s > t)
        return fail(MCDC_ERR_INVALID, "need 0 <= sigma_s <= sigma_t, finite");
      st[m * G + g] = t;
      scat[m * G + g] = t > 0.0 ? s / t : 0.0;
      const double *row = mat->transfer + ((size_t)m * G + g) * G;
      double sum = 0.0;
      for (int h = 0; h < G; ++h) {
        if (!finite_nonneg(row[h])) return fail(MCDC_ERR_INVALID, "transfer entries must be >= 0");
        sum += row[h];
      }
      if (s > 0.0 && std::fabs(sum - 1.0) > 1e-9)
        return fail(MCDC_ERR_INVALID, "transfer rows must sum to 1");
      build_cdf(row, G, cdf.data() + ((size_t)m * G + g) * G);
    }
  std::vector<double> speed(G);
  for (int g = 0; g < G; ++g) {
    if (!(std::isfinite(mat->speed[g]) && mat->speed[g] > 0.0))
      return fail(MCDC_ERR_INVALID, "speeds must be finite and > 0");
    speed[g] = mat->speed[g];
  }

  // ---- time grid
  int T = 0;
  std::vector<double> edges(1, 0.0);
  if (time && time->n_bins > 0) {
    T = time->n_bins;
    if (T > 65534) return fail(MCDC_ERR_INVALID, "too many time bins");
    if (!time->edges) return fail(MCDC_ERR_INVALID, "time edges are NULL");
    edges.assign(time->edges, time->edges + T + 1);
    for (int j = 0; j <= T; ++j)
      if (!std::isfinite(edges[j]) || (j > 0 && !(edges[j] > edges[j - 1])))
        return fail(MCDC_ERR_INVALID, "time edges must be finite and increasing");
  } else if (time && time->n_bins < 0) {
    return fail(MCDC_ERR_INVALID, "negative number of time bins");
  }

  // ---- source
  if (!src->group_pdf) return fail(MCDC_ERR_INVALID, "source group pdf is NULL");
  std::vector<double> scdf(G);
  {
    double sum = 0.0;
    for (int g = 0; g < G; ++g) {
      if (!finite_nonneg(src->group_pdf[g])) return fail(MCDC_ERR_INVALID, "source pdf must be >= 0");
      sum += src->group_pdf[g];
    }
    if (std::fabs(sum - 1.0) > 1e-9) return fail(MCDC_ERR_INVALID, "source pdf must sum to 1");
    build_cdf(src->group_pdf, G, scdf.data());
  }
  for (int a = 0; a < 3; ++a) {
    if (!std::isfinite(src->lo[a]) || !std::isfinite(src->hi[a]) || src->lo[a] > src->hi[a])
      return fail(MCDC_ERR_INVALID, "source box must be finite with lo <= hi");
    if (bounded[a] && (src->lo[a] < org[a] || src->hi[a] > org[a] + n[a] * wid[a]))
      return fail(MCDC_ERR_INVALID, "source box must lie inside the mesh");
  }
  if (src->kind != MCDC_SRC_ISOTROPIC && src->kind != MCDC_SRC_BEAM)
    return fail(MCDC_ERR_INVALID, "unknown source kind");
  if (src->kind == MCDC_SRC_BEAM) {
    const double nn = src->dir[0] * src->dir[0] + src->dir[1] * src->dir[1] + src->dir[2] * src->dir[2];
    if (!(std::fabs(nn - 1.0) < 1e-9)) return fail(MCDC_ERR_INVALID, "beam direction must be a unit vector");
  }
  if (!std::isfinite(src->t0) || !std::isfinite(src->t1) || src->t1 < src->t0)
    return fail(MCDC_ERR_INVALID, "need finite t0 <= t1");
  if (T > 0 && src->t0 < edges[0]) return fail(MCDC_ERR_INVALID, "source starts before the first time edge");
  if (o.pc_target > 0 && (T < 2 || !(src->t1 < edges[1])))
    return fail(MCDC_ERR_INVALID, "population control needs >= 2 time bins and every source "
                                  "particle born in the first bin");
  if (T == 0) {
    // steady state closed by reflecting faces: only absorption ends a history
    bool open = false;
    for (int a = 0; a < 3; ++a)
      if (bounded[a] && (mesh->bc[2 * a] == MCDC_BC_VACUUM || mesh->bc[2 * a + 1] == MCDC_BC_VACUUM))
        open = true;
    if (!open) {
      std::vector<char> used(M, 0);
      for (int64_t c = 0; c < n_cells; ++c) used[mesh->material[c]] = 1;
      for (int m = 0; m < M; ++m)
        for (int g = 0; g < G && used[m]; ++g)
          if (!(mat->sigma_s[m * G + g] < mat->sigma_t[m * G + g]))
            return fail(MCDC_ERR_INVALID, "a steady-state problem closed by reflecting faces needs "
                                          "sigma_s < sigma_t in every material and group");
    }
  }

  // ---- device
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev < 1) {
    cudaGetLastError();
    return fail(MCDC_ERR_NO_DEVICE, "no CUDA device");
  }
  int dev = 0;
  CK(cudaGetDevice(&dev));
  cudaDeviceProp prop;
  CK(cudaGetDeviceProperties(&prop, dev));
  if (prop.major != 10 || prop.minor != 3)
    return fail(MCDC_ERR_NO_DEVICE, std::string("built for sm_103 (B300), found ") + prop.name);
  DeviceLimits dl;
  if (int rc = device_limits(dev, &dl)) return rc;

  mcdc_problem *pr = new mcdc_problem();
  static std::atomic<uint64_t> next_uid{1};
  pr->uid = next_uid.fetch_add(1);
  pr->device = dev;
  pr->sms = dl.sms;
  pr->opt = o;
  pr->user_aggregate = o.warp_aggregate;
  pr->user_cps = o.ctas_per_sm;
  pr->user_block = o.block_size;
  pr->edges = edges;
  DevProblem &P = pr->P;
  for (int a = 0; a < 3; ++a) {
    P.n[a] = n[a];
    P.bounded[a] = bounded[a];
    P.origin[a] = org[a];
    P.width[a] = bounded[a] ? wid[a] : 0.0;
  }
  for (int s = 0; s < 6; ++s) P.bc[s] = mesh->bc[s];
  P.M = M; P.G = G; P.T = T; P.T1 = T > 0 ? T : 1;
  P.n_cells = n_cells;
  P.n_bins = n_cells * G * P.T1;
  if (P.n_bins >= (1ll << 31)) {
    delete pr;
    return fail(MCDC_ERR_INVALID, "the tally needs fewer than 2^31 bins (cells x groups x time bins)");
  }
  P.volume = 1.0;
  for (int a = 0; a < 3; ++a)
    if (bounded[a]) P.volume *= wid[a];
  for (int a = 0; a < 3; ++a) {
    P.src_lo[a] = src->lo[a];
    P.src_hi[a] = src->hi[a];
    P.src_dir[a] = src->dir[a];
  }
  P.src_kind = src->kind;
  P.t0 = src->t0;
  P.t1 = src->t1;
  P.estimator = o.estimator;
  P.n_tally = P.n_bins * (o.estimator == MCDC_EST_COMBINED ? 2 : 1);
  P.implicit = o.implicit_capture;
  P.wcut = o.weight_cutoff;
  P.wsurv = o.cutoff_survival;
  P.wcut32 = (float)o.weight_cutoff;
  P.wsurv32 = (float)o.cutoff_survival;
  P.pc_target = o.pc_target;
  P.fresh_tau = o.flight_sampling;
  if (o.pc_target > 0) pr->opt.tally_mode = MCDC_TALLY_GLOBAL;
  for (int a = 0; a < 3; ++a) {
    int hi = o.region_hi[a] > 0 ? o.region_hi[a] : n[a];
    int lo = std::max(0, o.region_lo[a]);
    P.region_lo[a] = lo;
    P.region_hi[a] = std::min(hi, n[a]);
  }
  pr->dim = (!bounded[1] && !bounded[2]) ? 1 : 3;
  pr->key.f64 = (o.precision == MCDC_PREC_FP64);
  pr->key.local = (o.precision == MCDC_PREC_FP32_LOCAL);
  pr->key.dim = pr->dim;
  pr->key.pc = o.pc_target > 0;
  pr->key.vr = o.implicit_capture != 0;

  int rc = MCDC_OK;
  auto bail = [&](int code) {
    std::string keep = g_err;
    release(pr);
    g_err = keep;
    return code;
  };
  Arena arena;
  {
    std::vector<uint8_t> matv(mesh->material, mesh->material + n_cells);
    arena.upload(&P.material, matv);
    arena.upload(&P.sigma_t, st);
    arena.upload(&P.scat, scat);
    arena.upload(&P.cdf, cdf);
    arena.upload(&P.speed, speed);
    arena.upload(&P.edges, edges);
    arena.upload(&P.src_cdf, scdf);
    for (int a = 0; a < 3; ++a) {
      P.faces[a] = nullptr;
      if (!bounded[a]) continue;
      std::vector<double> fc(n[a] + 1);
      for (int k = 0; k <= n[a]; ++k) {
        const double step = (double)k * wid[a];   // two roundings, as on the device
        fc[k] = org[a] + step;
      }
      arena.upload(&P.faces[a], fc);
    }
    for (int a = 0; a < 3; ++a) P.width32[a] = bounded[a] ? (float)wid[a] : 0.0f;
    for (int a = 0; a < 3; ++a) {
      P.src_cell_a[a] = bounded[a] ? (float)((src->lo[a] - org[a]) / wid[a]) : 0.0f;
      P.src_cell_b[a] = bounded[a] ? (float)((src->hi[a] - src->lo[a]) / wid[a]) : 0.0f;
    }
    std::vector<float> bw(std::max(T, 1), 0.0f);
    for (int j = 0; j < T; ++j) bw[j] = (float)(edges[j + 1] - edges[j]);
    arena.upload(&P.binw32, bw);
    auto f32 = [](const std::vector<double> &v) {
      std::vector<float> r(v.size());
      for (size_t q = 0; q < v.size(); ++q) r[q] = (float)v[q];
      return r;
    };
    std::vector<float> inv(G);
    for (int g = 0; g < G; ++g) inv[g] = (float)(1.0 / speed[g]);
    arena.upload(&P.sigma_t32, f32(st));
    arena.upload(&P.scat32, f32(scat));
    arena.upload(&P.cdf32, f32(cdf));
    arena.upload(&P.speed32, f32(speed));
    arena.upload(&P.inv_speed32, inv);
    arena.upload(&P.src_cdf32, f32(scdf));
  }
  if ((rc = choose_shape(pr, dl))) return bail(rc);
  arena.device(&pr->sum1, (size_t)P.n_tally);
  arena.device(&pr->sum2, (size_t)P.n_tally);
  if (P.estimator == MCDC_EST_COMBINED) arena.device(&pr->sum12, (size_t)P.n_bins);
  if (pr->tally_mode == MCDC_TALLY_GLOBAL) arena.device(&pr->tally, (size_t)P.n_tally);
  // region[0..4]: sums (track or the one estimator), squares, collision sums,
  // squares, products; region + 5: the batch's two region sums
  arena.device(&pr->region, 8);
  arena.device(&pr->stats, 1);
  arena.device(&pr->error, 4);
  arena.device(&pr->work, 64);
  arena.device(&pr->children, 1);
  if ((rc = arena.commit(pr))) return bail(rc);
  pr->region_batch = pr->region + 5;
  pr->work_slots = 64;
  PinnedBlock *pin = pinned_get();
  if (!pin || cudaEventCreate(&pr->ev0) != cudaSuccess || cudaEventCreate(&pr->ev1) != cudaSuccess ||
      cudaEventCreate(&pr->ev2) != cudaSuccess) {
    cudaGetLastError();
    pinned_put(pin);
    fail(MCDC_ERR_CUDA, "event or pinned buffer creation failed");
    return bail(MCDC_ERR_CUDA);
  }
  pr->pinned = pin;
  pr->h_stats = &pin->stats;
  pr->h_error = pin->error;
  pr->h_spill = &pin->count;
  if (o.autotune && o.block_size == 0 && o.pc_target == 0) {
    if ((rc = autotune(pr, dl))) return bail(rc);
  }
  *out = pr;
  return MCDC_OK;
}

int64_t mcdc_tally_size(const struct mcdc_problem *pr) { return pr ? pr->P.n_bins : -1; }

void mcdc_problem_destroy(struct mcdc_problem *pr) { release(pr); }

int mcdc_set_weight_windows(struct mcdc_problem *pr, const double *w_lower, double upper_ratio,
                            double survival_ratio, int32_t nmax) {
  g_err.clear();
  if (!pr) return fail(MCDC_ERR_INVALID, "problem is NULL");
  pr->p_version += 1;
  if (w_lower == nullptr) {
    pr->P.ww_lower = nullptr;
    pr->P.ww_lower32 = nullptr;
    pr->P.ww_net64 = nullptr;
    pr->P.ww_net32 = nullptr;
    pr->P.ww_netfrag = nullptr;
    return set_track_kernel_impl(pr, false, false);
  }
  if (pr->P.pc_target > 0)
    return fail(MCDC_ERR_INVALID, "weight windows and population control do not combine");
  if (!(upper_ratio > survival_ratio && survival_ratio > 1.0) || nmax < 2 || nmax > 1024)
    return fail(MCDC_ERR_INVALID, "need 1 < survival_ratio < upper_ratio and 2 <= nmax <= 1024");
  CK(cudaSetDevice(pr->device));
  const size_t nb = (size_t)pr->P.n_bins;
  std::vector<double> h(nb);
  if (is_device_ptr(w_lower)) CK(cudaMemcpy(h.data(), w_lower, nb * 8, cudaMemcpyDeviceToHost));
  else std::memcpy(h.data(), w_lower, nb * 8);
  std::vector<float> h32(nb);
  for (size_t q = 0; q < nb; ++q) {
    if (std::isnan(h[q])) return fail(MCDC_ERR_INVALID, "weight-window bound is NaN");
    h32[q] = (float)h[q];
  }
  if (!pr->ww64) {
    int rc;
    if ((rc = dalloc(pr, &pr->ww64, nb))) return rc;
    if ((rc = dalloc(pr, &pr->ww32, nb))) return rc;
  }
  CK(cudaMemcpy(pr->ww64, h.data(), nb * 8, cudaMemcpyHostToDevice));
  pr->ww_table_valid = true;
  CK(cudaMemcpy(pr->ww32, h32.data(), nb * 4, cudaMemcpyHostToDevice));
  pr->P.ww_lower = pr->ww64;
  pr->P.ww_lower32 = pr->ww32;
  pr->P.ww_net64 = nullptr;
  pr->P.ww_net32 = nullptr;
  pr->P.ww_netfrag = nullptr;
  pr->P.ww_upper = upper_ratio;
  pr->P.ww_survival = survival_ratio;
  pr->P.ww_upper32 = (float)upper_ratio;
  pr->P.ww_survival32 = (float)survival_ratio;
  pr->P.ww_nmax = nmax;
  if (int rc = set_track_kernel_impl(pr, false, true)) return rc;
  return ensure_overflow(pr);
}

int mcdc_set_network_windows(struct mcdc_problem *pr, const float *params, int32_t n_in,
                              int32_t hidden, double shift, double scale, double top,
                              double floor_lp, double source_wl, double upper_ratio,
                              double survival_ratio, int32_t nmax) {
  g_err.clear();
  if (!pr) return fail(MCDC_ERR_INVALID, "problem is NULL");
  if (params == nullptr) return mcdc_set_weight_windows(pr, nullptr, 0.0, 0.0, 0);
  pr->p_version += 1;
  if (pr->P.pc_target > 0)
    return fail(MCDC_ERR_INVALID, "weight windows and population control do not combine");
  if (hidden < 1 || hidden > 64) return fail(MCDC_ERR_INVALID, "hidden width must be 1..64");
  if (pr->tally_mode != MCDC_TALLY_GLOBAL)
    return fail(MCDC_ERR_INVALID, "per-event windows need the global tally (tally_mode)");
  if (pr->P.G > 16) return fail(MCDC_ERR_INVALID, "per-event windows take at most 16 groups");  // inputs 4 + G fit the kernel's 20
  if (!(upper_ratio > survival_ratio && survival_ratio > 1.0) || nmax < 2 || nmax > 1024)
    return fail(MCDC_ERR_INVALID, "need 1 < survival_ratio < upper_ratio and 2 <= nmax <= 1024");
  if (!(source_wl > 0.0) || !std::isfinite(shift) || !std::isfinite(scale) ||
      !std::isfinite(top) || !std::isfinite(floor_lp))
    return fail(MCDC_ERR_INVALID, "window constants must be finite (source_wl > 0)");
  if (n_in != 3 && n_in != 4 + pr->P.G)
    return fail(MCDC_ERR_INVALID, "n_in must be 3 (position) or 4 + groups (position, time, group)");
  CK(cudaSetDevice(pr->device));
  const int in = n_in;
  // W1[hidden][in], b1[hidden], W2[hidden][hidden], b2[hidden], W3[hidden], b3
  const size_t n = (size_t)hidden * in + hidden + (size_t)hidden * hidden + 2 * (size_t)hidden + 1;
  std::vector<float> h32(n);
  if (is_device_ptr(params)) CK(cudaMemcpy(h32.data(), params, n * 4, cudaMemcpyDeviceToHost));
  else std::memcpy(h32.data(), params, n * 4);
  std::vector<double> h64(n);
  for (size_t q = 0; q < n; ++q) {
    if (!std::isfinite(h32[q])) return fail(MCDC_ERR_INVALID, "network parameter is not finite");
    h64[q] = (double)h32[q];
  }
  if (!pr->key.f64) {
    // the FP32 modes hold W1 / 2, W2 / 2 and W3 in binary16
    const size_t w1 = (size_t)hidden * in, b1 = w1 + hidden, w2 = b1 + (size_t)hidden * hidden,
                 w3 = w2 + hidden;
    for (size_t q = 0; q < w3 + hidden; ++q) {
      const bool weight = q < w1 || (q >= b1 && q < w2) || q >= w3;
      const float lim = q >= w3 ? 65504.0f : 131008.0f;
      if (weight && std::fabs(h32[q]) >= lim)
        return fail(MCDC_ERR_INVALID, "network weight beyond the binary16 range of the FP32 modes");
    }
  }
  if (pr->net_cap < n) {
    int rc;
    if ((rc = dalloc(pr, &pr->net64, n))) return rc;
    if ((rc = dalloc(pr, &pr->net32, n))) return rc;
    pr->net_cap = n;
  }
  if (!pr->netfrag) {
    if (int rc = dalloc(pr, &pr->netfrag, (size_t)kNetFragWords)) return rc;
  }
  const std::vector<uint32_t> frag = net_fragments(h32.data(), in, hidden);
  CK(cudaMemcpy(pr->net64, h64.data(), n * 8, cudaMemcpyHostToDevice));
  CK(cudaMemcpy(pr->net32, h32.data(), n * 4, cudaMemcpyHostToDevice));
  CK(cudaMemcpy(pr->netfrag, frag.data(), (size_t)kNetFragBytes, cudaMemcpyHostToDevice));
  // the network kernel first: if its launch shape fails, nothing changes
  // (the kernel of the windows already set, table or network, stays)
  const bool prev_net = pr->key.net, prev_ww = pr->P.ww_lower != nullptr;
  if (int rc = set_track_kernel_impl(pr, true, false)) {
    const std::string msg = g_err;
    set_track_kernel_impl(pr, prev_net, prev_ww);
    return fail(rc, msg);
  }
  DevProblem &P = pr->P;
  P.ww_lower = nullptr;
  P.ww_lower32 = nullptr;
  P.ww_net64 = pr->net64;
  P.ww_net32 = pr->net32;
  P.ww_netfrag = pr->netfrag;
  P.ww_net_b3 = h32[n - 1];
  for (int a = 0; a < 3; ++a) {
    const bool b = P.bounded[a] != 0;
    P.net_cell[a] = b ? (float)(2.0 / P.n[a]) : 0.0f;
    P.net_off[a] = b ? (float)(2.0 / (P.n[a] * P.width[a])) : 0.0f;
  }
  P.ww_net_in = in;
  P.ww_net_h = hidden;
  P.ww_net_shift = shift;
  P.ww_net_scale = scale;
  P.ww_net_top = top;
  P.ww_net_floor = floor_lp;
  P.ww_net_wl0 = source_wl;
  P.ww_upper = upper_ratio;
  P.ww_survival = survival_ratio;
  P.ww_net_shift32 = (float)shift;
  P.ww_net_scale32 = (float)scale;
  P.ww_net_top32 = (float)top;
  P.ww_net_floor32 = (float)floor_lp;
  P.ww_net_wl0_32 = (float)source_wl;
  P.ww_upper32 = (float)upper_ratio;
  P.ww_survival32 = (float)survival_ratio;
  P.ww_nmax = nmax;
  return ensure_overflow(pr);
}

int mcdc_get_weight_windows(const struct mcdc_problem *pr, double *w_lower) {
  g_err.clear();
  if (!pr || !w_lower) return fail(MCDC_ERR_INVALID, "problem and w_lower are required");
  if (!pr->ww_table_valid || !pr->ww64) return fail(MCDC_ERR_INVALID, "no window table yet");
  CK(cudaSetDevice(pr->device));
  CK(cudaDeviceSynchronize());
  CK(cudaMemcpy(w_lower, pr->ww64, sizeof(double) * (size_t)pr->P.n_bins, cudaMemcpyDefault));
  return MCDC_OK;
}

int mcdc_network_window_lower(struct mcdc_problem *pr, const double *x, const double *t,
                              const int32_t *g, int64_t n, double *w_lower) {
  g_err.clear();
  if (!pr) return fail(MCDC_ERR_INVALID, "problem is NULL");
  if (pr->P.ww_net64 == nullptr) return fail(MCDC_ERR_INVALID, "no network windows are set");
  if (n < 0) return fail(MCDC_ERR_INVALID, "n must be >= 0");
  if (n == 0) return MCDC_OK;
  if (!x || !t || !g || !w_lower) return fail(MCDC_ERR_INVALID, "x, t, g and w_lower are required");
  CK(cudaSetDevice(pr->device));
  // device copies of host arrays (a diagnostic entry point, not a hot path)
  const size_t un = (size_t)n;
  std::vector<void *> tmp;
  auto dev_in = [&](const void *src, size_t bytes, const void **out) -> cudaError_t {
    if (is_device_ptr(src)) { *out = src; return cudaSuccess; }
    void *d = nullptr;
    cudaError_t e = cudaMalloc(&d, bytes);
    if (e != cudaSuccess) return e;
    tmp.push_back(d);
    *out = d;
    return cudaMemcpy(d, src, bytes, cudaMemcpyHostToDevice);
  };
  const void *dx = nullptr, *dt = nullptr, *dg = nullptr;
  void *dout = w_lower;
  cudaError_t e = dev_in(x, 24 * un, &dx);
  if (e == cudaSuccess) e = dev_in(t, 8 * un, &dt);
  if (e == cudaSuccess) e = dev_in(g, 4 * un, &dg);
  const bool host_out = !is_device_ptr(w_lower);
  if (e == cudaSuccess && host_out) {
    e = cudaMalloc(&dout, 8 * un);
    if (e == cudaSuccess) tmp.push_back(dout);
  }
  if (e == cudaSuccess)
    e = launch_net_lower(pr->key, nullptr, pr->P, (const double *)dx, (const double *)dt,
                         (const int32_t *)dg, (long long)n, (double *)dout, pr->sms);
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e == cudaSuccess && host_out) e = cudaMemcpy(w_lower, dout, 8 * un, cudaMemcpyDeviceToHost);
  for (void *d : tmp) cudaFree(d);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(e == cudaErrorMemoryAllocation ? MCDC_ERR_OOM : MCDC_ERR_CUDA,
                std::string("window evaluation: ") + cudaGetErrorString(e));
  }
  return MCDC_OK;
}

int mcdc_run_ex(struct mcdc_problem *pr, const mcdc_run_args *a, mcdc_stats *stats) {
  NvtxRange nvtx("mcdc_run_ex");
  g_err.clear();
  if (!pr || !a) return fail(MCDC_ERR_INVALID, "problem and args are required");
  if (a->n_histories == 0) return fail(MCDC_ERR_INVALID, "n_histories must be > 0");
  CK(cudaSetDevice(pr->device));
  cudaStream_t s = (cudaStream_t)a->stream;
  const DevProblem &P = pr->P;
  int B = a->n_batches > 0 ? a->n_batches : default_batches(pr, a->n_histories);
  if (B < 2 || (uint64_t)B > a->n_histories)
    return fail(MCDC_ERR_INVALID, "need 2 <= n_batches <= n_histories");
  if (int rc = ensure_overflow(pr)) return rc;
  if (int rc = ensure_work_slots(pr, pr->tally_mode == MCDC_TALLY_GLOBAL ? B : 1)) return rc;

  const size_t nb = (size_t)P.n_bins, nt = (size_t)P.n_tally;
  const bool comb = P.estimator == MCDC_EST_COMBINED;
  const bool mean_dev = is_device_ptr(a->mean_out), rel_dev = is_device_ptr(a->relerr_out);
  const bool s1_dev = is_device_ptr(a->sum1_out), s2_dev = is_device_ptr(a->sum2_out);
  double *const sum12_out = comb ? a->sum12_out : nullptr;
  double *const parts_out = comb ? a->parts_out : nullptr;
  const bool s12_dev = is_device_ptr(sum12_out), parts_dev = is_device_ptr(parts_out);
  if (parts_out && !parts_dev && !pr->parts_tmp) {
    int rc;
    if ((rc = dalloc(pr, &pr->parts_tmp, 5 * nb))) return rc;
  }
  const bool rec_dev = is_device_ptr(a->records);
  if (a->records && a->n_records == 0) return fail(MCDC_ERR_INVALID, "records given with n_records == 0");
  if (a->records && P.pc_target > 0)
    return fail(MCDC_ERR_INVALID, "no per-history records under population control (histories mix)");
  if ((a->mean_out && !mean_dev) || (a->relerr_out && !rel_dev)) {
    if (!pr->mean_tmp) {
      int rc;
      if ((rc = dalloc(pr, &pr->mean_tmp, nb))) return rc;
      if ((rc = dalloc(pr, &pr->rel_tmp, nb))) return rc;
    }
  }
  Record *rec_buf = nullptr;
  uint64_t n_rec = a->records ? std::min<uint64_t>(a->n_records, a->n_histories) : 0;
  if (a->records) {
    if (rec_dev) {
      rec_buf = (Record *)a->records;
    } else {
      if (pr->rec_cap < n_rec) {
        int rc;
        if ((rc = dalloc(pr, &pr->rec_tmp, (size_t)n_rec))) return rc;
        pr->rec_cap = n_rec;
      }
      rec_buf = pr->rec_tmp;
    }
  }

  CK(cudaEventRecord(pr->ev0, s));
  CK(cudaMemsetAsync(pr->sum1, 0, nt * 8, s));
  CK(cudaMemsetAsync(pr->sum2, 0, nt * 8, s));
  if (comb) CK(cudaMemsetAsync(pr->sum12, 0, nb * 8, s));
  CK(cudaMemsetAsync(pr->region, 0, 8 * sizeof(double), s));
  CK(cudaMemsetAsync(pr->stats, 0, sizeof(Stats), s));
  CK(cudaMemsetAsync(pr->error, 0, 4 * sizeof(int32_t), s));
  CK(cudaMemsetAsync(pr->work, 0, sizeof(unsigned long long) * pr->work_slots, s));
  CK(cudaMemsetAsync(pr->children, 0, sizeof(unsigned long long), s));

  RunArgs A{};
  A.n_hist = a->n_histories;
  A.offset = a->hist_offset;
  A.seed = a->seed;
  A.rk = round_keys(a->seed);
  A.n_batches = B;
  A.sum1 = pr->sum1;
  A.sum2 = pr->sum2;
  A.sum12 = pr->sum12;
  A.region = pr->region;
  A.stats = pr->stats;
  A.records = rec_buf;
  A.n_records = n_rec;
  A.error = pr->error;
  A.overflow = pr->overflow;
  A.overflow_cap = pr->overflow_cap;
  A.overflow_tail = pr->opt.overflow_tail;
  A.warp_aggregate = pr->warp_aggregate;
  A.tally = pr->tally;
  if (pr->opt.max_children >= 0) {
    A.children_made = pr->children;
    // default: 4096 children per history, at least 2^27 -- 8x what learned
    // windows on a 30-mean-free-path absorber make, so only a runaway map
    // reaches it, and the bound grows with the run
    A.children_budget = pr->opt.max_children > 0
                            ? (unsigned long long)pr->opt.max_children
                            : std::max<unsigned long long>(1ull << 27, 4096ull * a->n_histories);
  }
  A.batch_q = a->n_histories / (uint64_t)B;
  A.batch_r = a->n_histories % (uint64_t)B;
  if (a->n_histories <= 0xFFFFFFFFull) {
    A.div_q1.set((uint32_t)(A.batch_q + 1));
    A.div_q.set((uint32_t)std::max<uint64_t>(1, A.batch_q));
  }

  CK(cudaEventRecord(pr->ev1, s));
  // a run that returned early (a failed launch, the spill-pass limit) left
  // scores in the batch tally or the slices, which a fold would otherwise
  // zero: clear them before this run scores
  if (pr->tally_dirty) {
    CK(cudaMemsetAsync(pr->tally, 0, nt * 8, s));
    pr->tally_dirty = false;
  }
  if (pr->slices_dirty && pr->pc_tally) {
    CK(cudaMemsetAsync(pr->pc_tally, 0, (size_t)pr->slice_bytes * (size_t)pr->pc_tally_bins, s));
    CK(cudaMemsetAsync(pr->slice_rb, 0, sizeof(double) * 2 * (size_t)(pr->pc_tally_bins / std::max<long long>(1, P.n_tally)), s));
    pr->slices_dirty = false;
  }
  if (pr->tally_mode == MCDC_TALLY_SHARED) {
    A.work = pr->work;
    A.batch = 0;
    A.chunk = 0;
    CK(launch_track(pr->key, pr->grid, pr->block, pr->smem, s, P, A, pr->L));
  } else if (P.pc_target > 0) {
    // population control: every batch is a time-stepped simulation with its
    // own tally slice; one launch runs one step of all batches, then the
    // census bank is combed batch by batch and the next step runs it
    const int M = P.pc_target;
    const uint64_t N = a->n_histories;
    if (N > 0x7fffffffull || (uint64_t)B * (uint64_t)M > 0x7fffffffull)
      return fail(MCDC_ERR_INVALID, "population control needs n_histories and n_batches x pc_target < 2^31");
    if (int rc = ensure_pc(pr, (int)std::max<uint64_t>(N, (uint64_t)B * M), (long long)B * M, B))
      return rc;
    A.work = pr->work;
    A.batch = 0;
    use_slices(pr, A);
    A.tally_per_batch = 1;
    A.chunk = (int)std::max<uint64_t>(32, std::min<uint64_t>(pr->S, N / ((uint64_t)pr->grid * 4) + 1));
    A.spill_in = nullptr;
    A.spill_out = nullptr;
    A.census_out = pr->pc_bank;
    A.census_count = pr->pc_cnt;
    A.census_cap = (unsigned long long)pr->pc_cap;
    // every particle of a step is in that step's time bin: score it into a
    // CTA-private shared tally over (estimator, batch, cell, group) when that
    // fits beside the pool, else straight into the slices
    // After a comb, each warp also stages its next 32 births from the combed
    // bank in shared memory (bulk async copies overlapping the flights).
    // Both are used only where they keep the CTAs per SM.
    Layout Ls = pr->L;
    int smem_pc = pr->smem;
    {
      const long long bins = (long long)(P.estimator == MCDC_EST_COMBINED ? 2 : 1) * B *
                             P.n_cells * P.G;
      const long long bytes = (bins * (pr->key.f64 ? 8 : 4) + 15) & ~15ll;
      const long long stage = (long long)pr->block * slot_bytes(pr->key.f64, pr->dim, pr->key.local);
      const long long base = (long long)Ls.tables_bytes + Ls.bank_bytes + 64;
      auto fits = [&](long long total) {
        return total <= pr->dyn_max &&
               track_occupancy(pr->key, pr->block, (int)total) >= pr->ctas_per_sm;
      };
      if (fits(base + bytes + stage)) {
        A.step_tally = 1;
        A.prefetch = 1;
      } else if (fits(base + bytes)) {
        A.step_tally = 1;
      } else if (fits(base + stage)) {
        A.prefetch = 1;
      }
      if (A.step_tally) { Ls.tally_bytes = bytes; A.step_bins = (int)bins; }
      Ls.total = (int)(base + (A.step_tally ? bytes : 0) + (A.prefetch ? stage : 0));
      smem_pc = Ls.total;
    }
    // every banked particle lands at its position in the step's input (the
    // histories, then the combed bank): its census weight marks it
    A.census_w = pr->pc_w;
    int32_t *live[2] = {pr->pc_live, pr->pc_live + B};
    int32_t *n_live[2] = {pr->pc_live + 2 * B, pr->pc_live + 2 * B + 1};
    long long n_in = (long long)N;
    pr->slices_dirty = true;
    for (int step = 0;; ++step) {
      CK(cudaMemsetAsync(pr->pc_cnt, 0, sizeof(unsigned long long), s));
      CK(cudaMemsetAsync(pr->pc_w, 0, sizeof(double) * (size_t)n_in, s));
      A.step_tbin = step;
      CK(launch_track(pr->key, pr->grid, pr->block, smem_pc, s, P, A, Ls));
      if (step >= P.T - 1) break;
      // no host round trip between steps: when nothing was banked the comb
      // finds zero weight in every batch and the next step's launch finds
      // an empty combed bank, so the remaining steps cost a few empty launches
      NvtxRange nvtx_comb("comb");
      CombArgs c{};
      c.bank = pr->pc_bank;
      c.bank_cap = pr->pc_cap;
      c.out_cap = pr->pc_combed_cap;
      c.dim = pr->dim;
      c.w = pr->pc_w;
      c.n_in = (int)n_in;
      c.first_step = step == 0;
      c.live_in = live[(step + 1) & 1];
      c.n_live_in = n_live[(step + 1) & 1];
      c.live_out = live[step & 1];
      c.n_live_out = n_live[step & 1];
      c.out = pr->pc_combed;
      c.out_count = pr->pc_cnt + 1;
      c.banked = pr->pc_cnt;
      c.M = M;
      c.offset = a->hist_offset;
      c.n_hist = N;
      c.B = B;
      c.step = step;
      c.rk = A.rk;
      c.key = pr->pc_key;
      c.S = pr->pc_S;
      c.seg = pr->pc_seg;
      c.segd = pr->pc_segd;
      c.temp = pr->pc_temp;
      c.temp_bytes = pr->pc_temp_bytes;
      c.stats = pr->stats;
      c.error = pr->error;
      CK(comb_bank(pr->key, s, c));
      CK(cudaMemsetAsync(pr->pc_cnt + 2, 0, sizeof(unsigned long long), s));
      A.spill_in = pr->pc_combed;
      A.spill_in_count = pr->pc_cnt + 1;
      A.spill_in_cursor = pr->pc_cnt + 2;
      A.spill_cap = (unsigned long long)pr->pc_combed_cap;
      n_in = (long long)B * M;        // the next input: one chunk of M per combed batch
    }
    CK(fold_slices(pr, s, P, nt, B));
    pr->slices_dirty = false;
  } else {
    const bool spill = ww_on(P) && pr->spill[0] != nullptr;
    // every batch in one launch, one tally slice per batch, when the slices
    // fit in 8 GiB: weight-window runs would otherwise leave most warps idle
    // while a handful work through a batch's split families, and analog runs
    // pay a launch tail per batch (one launch: +5 % on the 60^3 channel,
    // +9 % on the deep box); otherwise one launch and one fold per batch
    // (options.slice_bytes_max moves the 8 GiB cap; negative: never).  When
    // the slices cannot be allocated the run falls back to the per-batch
    // launches, which need only the one batch tally.
    const double cap = pr->opt.slice_bytes_max > 0 ? (double)pr->opt.slice_bytes_max
                                                   : 8.0 * 1073741824.0;
    const double entry = pr->key.f64 ? 8.0 : 4.0;
    bool merged = pr->opt.slice_bytes_max >= 0 && (double)B * (double)nt * entry <= cap;
    if (merged) {
      if (int rc = ensure_slices(pr, B)) {
        if (rc != MCDC_ERR_OOM) return rc;
        cudaGetLastError();
        g_err.clear();
        merged = false;
      }
    }
    if (merged) pr->slices_dirty = true;
    else pr->tally_dirty = true;
    for (int b = 0; b < (merged ? 1 : B); ++b) {
      A.work = pr->work + b;
      A.batch = b;
      if (merged) {
        use_slices(pr, A);
      } else {
        A.tally = pr->tally;
        A.tally32 = nullptr;
      }
      A.tally_per_batch = merged ? 1 : 0;
      const uint64_t nb_hist = merged ? a->n_histories : a->n_histories / B + 1;
      A.chunk = (int)std::max<uint64_t>(32, std::min<uint64_t>(pr->S, nb_hist / ((uint64_t)pr->grid * 4) + 1));
      A.spill_in = nullptr;
      A.spill_out = nullptr;
      if (spill) {
        CK(cudaMemsetAsync(pr->spill_cnt, 0, 4 * sizeof(unsigned long long), s));
        A.spill_out = pr->spill[0];
        A.spill_out_count = pr->spill_cnt + 0;
        A.spill_cap = pr->spill_cap;
      }
      CK(launch_track(pr->key, pr->grid, pr->block, pr->smem, s, P, A, pr->L));
      // passes over the spilled children, ping-ponging between the banks,
      // until a pass spills nothing
      for (int pass = 1; spill; ++pass) {
        const int in = (pass - 1) & 1, out = pass & 1;
        CK(cudaMemcpyAsync(pr->h_spill, pr->spill_cnt + in, sizeof(unsigned long long),
                           cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        if (*pr->h_spill == 0) break;
        if (pass == 100000)
          return fail(MCDC_ERR_BANK_OVERFLOW, "split children still pending after 100000 spill passes");
        CK(cudaMemsetAsync(pr->spill_cnt + out, 0, sizeof(unsigned long long), s));
        CK(cudaMemsetAsync(pr->spill_cnt + 2, 0, sizeof(unsigned long long), s));
        A.spill_in = pr->spill[in];
        A.spill_in_count = pr->spill_cnt + in;
        A.spill_in_cursor = pr->spill_cnt + 2;
        A.spill_out = pr->spill[out];
        A.spill_out_count = pr->spill_cnt + out;
        CK(launch_track(pr->key, pr->grid, pr->block, pr->smem, s, P, A, pr->L));
      }
      if (merged) {
        CK(fold_slices(pr, s, P, nt, B));
      } else {
        CK(launch_fold(s, P, pr->tally, pr->sum1, pr->sum2, pr->sum12, pr->region_batch,
                       pr->region, pr->sms));
      }
    }
    pr->slices_dirty = false;
    pr->tally_dirty = false;
  }
  CK(cudaEventRecord(pr->ev2, s));

  // outputs
  double *mean_d = a->mean_out ? (mean_dev ? a->mean_out : pr->mean_tmp) : nullptr;
  double *rel_d = a->relerr_out ? (rel_dev ? a->relerr_out : pr->rel_tmp) : nullptr;
  double *parts_d = parts_out ? (parts_dev ? parts_out : pr->parts_tmp) : nullptr;
  if (comb) {
    if (mean_d || rel_d || parts_d)
      CK(launch_finalize_combined(s, (int64_t)nb, pr->sum1, pr->sum2, pr->sum12, a->n_histories,
                                  B, P.volume, mean_d, rel_d, parts_d, pr->sms));
  } else if (mean_d || rel_d) {
    CK(launch_finalize(s, (int64_t)nb, pr->sum1, pr->sum2, a->n_histories, B, P.volume, mean_d,
                       rel_d, pr->sms));
  }
  const cudaMemcpyKind d2h = cudaMemcpyDeviceToHost, d2d = cudaMemcpyDeviceToDevice;
  if (a->mean_out && !mean_dev)
    CK(cudaMemcpyAsync(a->mean_out, pr->mean_tmp, nb * 8, d2h, s));
  if (a->relerr_out && !rel_dev)
    CK(cudaMemcpyAsync(a->relerr_out, pr->rel_tmp, nb * 8, d2h, s));
  if (parts_out && !parts_dev)
    CK(cudaMemcpyAsync(parts_out, pr->parts_tmp, 5 * nb * 8, d2h, s));
  if (a->sum1_out) CK(cudaMemcpyAsync(a->sum1_out, pr->sum1, nt * 8, s1_dev ? d2d : d2h, s));
  if (a->sum2_out) CK(cudaMemcpyAsync(a->sum2_out, pr->sum2, nt * 8, s2_dev ? d2d : d2h, s));
  if (sum12_out) CK(cudaMemcpyAsync(sum12_out, pr->sum12, nb * 8, s12_dev ? d2d : d2h, s));
  if (a->records && !rec_dev)
    CK(cudaMemcpyAsync(a->records, rec_buf, n_rec * sizeof(Record), d2h, s));
  CK(cudaMemcpyAsync(pr->h_stats, pr->stats, sizeof(Stats), d2h, s));
  CK(cudaMemcpyAsync(pr->h_error, pr->error, 4 * sizeof(int32_t), d2h, s));
  double region_h[5] = {0, 0, 0, 0, 0};
  const bool want_region = a->scalar_out || (comb && a->scalar_parts_out);
  const bool need_sync = (s == nullptr) || stats || want_region || (a->mean_out && !mean_dev) ||
                         (a->relerr_out && !rel_dev) || (a->sum1_out && !s1_dev) ||
                         (a->sum2_out && !s2_dev) || (a->records && !rec_dev) ||
                         (sum12_out && !s12_dev) || (parts_out && !parts_dev);
  if (want_region) CK(cudaMemcpyAsync(region_h, pr->region, 5 * sizeof(double), d2h, s));
  if (!need_sync) return MCDC_OK;
  CK(cudaStreamSynchronize(s));
  if (comb && want_region) {
    double m, rel, al;
    combine_scalar(region_h, a->n_histories, B, P.volume, &m, &rel, &al);
    if (a->scalar_out) { a->scalar_out[0] = m; a->scalar_out[1] = rel; }
    if (double *sp = a->scalar_parts_out) {
      scalar_moments(region_h[0], region_h[1], a->n_histories, B, P.volume, &sp[0], &sp[1]);
      scalar_moments(region_h[2], region_h[3], a->n_histories, B, P.volume, &sp[2], &sp[3]);
      sp[4] = al;
    }
  } else if (a->scalar_out) {
    scalar_moments(region_h[0], region_h[1], a->n_histories, B, P.volume, &a->scalar_out[0],
                   &a->scalar_out[1]);
  }
  if (stats) {
    const Stats &h = *pr->h_stats;
    stats->histories = h.histories; stats->segments = h.segments;
    stats->collisions = h.collisions; stats->crossings = h.crossings; stats->census = h.census;
    stats->absorbed = h.absorbed; stats->leaked = h.leaked; stats->censused = h.censused;
    stats->splits = h.splits; stats->children = h.children;
    stats->splits_dropped = h.splits_dropped;
    stats->pc_combs = h.pc_combs; stats->pc_in = h.pc_in; stats->pc_out = h.pc_out;
    stats->w_pc_in = h.w_pc_in; stats->w_pc_out = h.w_pc_out;
    stats->roulette_killed = h.roulette_killed; stats->roulette_survived = h.roulette_survived;
    stats->w_source = h.w_source; stats->w_absorbed = h.w_absorbed;
    stats->w_leaked = h.w_leaked; stats->w_censused = h.w_censused;
    if (!weights_summed(P)) {   // analog: every weight is 1
      stats->w_source = (double)h.histories;
      stats->w_absorbed = (double)h.absorbed;
      stats->w_leaked = (double)h.leaked;
      stats->w_censused = (double)h.censused;
    }
    float k_ms = 0.f, t_ms = 0.f;
    cudaEventElapsedTime(&k_ms, pr->ev1, pr->ev2);
    cudaEventElapsedTime(&t_ms, pr->ev0, pr->ev2);
    stats->kernel_ms = k_ms;
    stats->total_ms = t_ms;
    stats->block_size = pr->block;
    stats->bank_per_cta = pr->S;
    stats->ctas_per_sm = pr->ctas_per_sm;
    stats->tally_mode = pr->tally_mode;
    stats->n_batches = B;
    stats->warp_aggregate = pr->warp_aggregate;
  }
  if (*pr->h_error & ERRBIT_CHECK) return fail(MCDC_ERR_CHECK, check_message(pr->h_error));
  if (*pr->h_error & ERRBIT_OVERFLOW)
    return fail(MCDC_ERR_BANK_OVERFLOW, "split children overflowed the warp stacks or the device-wide spill bank");
  if (*pr->h_error & ERRBIT_TIMEOUT) return fail(MCDC_ERR_TIMEOUT, "a bounded device wait gave up");
  return MCDC_OK;
}

int mcdc_run(struct mcdc_problem *pr, uint64_t n_histories, uint64_t seed, double *tally_out) {
  mcdc_run_args a;
  std::memset(&a, 0, sizeof a);
  a.n_histories = n_histories;
  a.seed = seed;
  a.mean_out = tally_out;
  a.stream = nullptr;
  int rc = mcdc_run_ex(pr, &a, nullptr);
  if (rc == MCDC_OK) {
    cudaError_t e = cudaStreamSynchronize(nullptr);
    if (e != cudaSuccess) return fail(MCDC_ERR_CUDA, cudaGetErrorString(e));
  }
  return rc;
}

}  // extern "C"
