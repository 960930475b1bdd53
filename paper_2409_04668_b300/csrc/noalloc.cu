// noalloc.cu -- mcdc_run_noalloc: a run that allocates no device memory.
//
// Some callers cannot call cudaMalloc while they run transport: a code that
// has handed all device memory to its own pool allocator, a real-time loop
// where an allocation would stall the device, or a host that forbids
// allocation after start-up.  For them this entry point keeps the run's
// scratch (the per-batch claim counters, the global-mode batch tally, the
// region and error accumulators and the event counters) in one file-scope
// __device__ array of fixed size instead of buffers from cudaMalloc.  The
// problem tables come from mcdc_problem_create (done once, at set-up) and
// the caller passes the output buffers.
//
// Limits: at most kMaxBins tally bins when the problem uses the global
// tally, at most kMaxBatches batches; larger requests are rejected.
// Weight windows: the run draws split children from the same per-run budget
// as mcdc_run_ex (the problem's max_children option, by default 4096 per
// history and at least 2^27), counted in the fixed array, so windows that
// would split without end still end.  There is no device-wide spill bank
// here: a child that finds its warp's stack full is not made and its parent
// keeps the weight (unbiased, but in the global tally mode, whose warp
// stacks hold 64 children, such a run then differs from mcdc_run_ex, which
// spills those children to banks it allocates).  Every
// GPU that loads the library holds the array (about 1.1 MiB) until exit.
// All calls share it and it keeps the previous call's contents: each call
// clears what must start at zero, and calls that overlap on the GPU (on
// different streams, or from different threads) race on it.
#include <cstring>
#include <mutex>
#include <string>

#include "../../include/mcdc.h"
#include "launch.h"
#include "problem.h"
#include "tracker.cuh"

using namespace mcdc;

namespace {

constexpr long long kMaxBins = 1ll << 17;   // global-mode batch tally (1 MiB of doubles)
constexpr int kMaxBatches = 4096;           // one claim counter per batch
constexpr int kMaxDevices = 64;

struct Scratch {
  double tally[kMaxBins];
  unsigned long long work[kMaxBatches];
  double region[8];     // region sums and squares [0..4], batch partials [5..6]
  unsigned long long children;   // split children made so far (weight windows)
  Stats stats;
  int32_t error[4];
};

int fail(int code, const std::string &m) { return mcdc::set_error(code, m); }

bool on_device(const void *p) {
  if (!p) return false;
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

std::mutex g_mu;
Scratch *g_addr[kMaxDevices] = {};

}  // namespace

static __device__ __align__(256) Scratch mcdc_noalloc_scratch;

// Device address of the scratch array on `dev` (the current device), looked
// up once per device.  The name of the array in host code is only a host-side
// stand-in; kernels must be given this address.
static int scratch_address(int dev, Scratch **out) {
  if (dev < 0 || dev >= kMaxDevices) return fail(MCDC_ERR_INVALID, "device index out of range");
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_addr[dev]) {
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, mcdc_noalloc_scratch);
    if (e != cudaSuccess || p == nullptr)
      return fail(MCDC_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
    g_addr[dev] = (Scratch *)p;
  }
  *out = g_addr[dev];
  return MCDC_OK;
}

extern "C" int mcdc_run_noalloc(struct mcdc_problem *pr, uint64_t n_histories, uint64_t seed,
                                uint64_t hist_offset, int32_t n_batches, double *sum1,
                                double *sum2, double *mean, double *relerr, void *stream) {
  if (!pr) return fail(MCDC_ERR_INVALID, "problem is NULL");
  if (pr->P.pc_target > 0)
    return fail(MCDC_ERR_INVALID, "population control needs its bank buffers: use mcdc_run_ex");
  if (pr->P.estimator == MCDC_EST_COMBINED)
    return fail(MCDC_ERR_INVALID, "the combined estimator needs its second tally: use mcdc_run_ex");
  if (n_histories < 2) return fail(MCDC_ERR_INVALID, "n_histories must be >= 2");
  if (n_batches < 2 || (uint64_t)n_batches > n_histories)
    return fail(MCDC_ERR_INVALID, "need 2 <= n_batches <= n_histories");
  if (n_batches > kMaxBatches)
    return fail(MCDC_ERR_INVALID, "n_batches exceeds the allocation-free limit of 4096");
  const bool global = pr->tally_mode == MCDC_TALLY_GLOBAL;
  if (global && pr->P.n_bins > kMaxBins)
    return fail(MCDC_ERR_INVALID, "tally exceeds the allocation-free limit of 131072 bins "
                                  "(global tally mode)");
  if (ww_on(pr->P) && pr->overflow == nullptr)
    return fail(MCDC_ERR_INVALID, "weight windows set without an overflow stack");
  cudaError_t e = cudaSetDevice(pr->device);
  if (e != cudaSuccess) return fail(MCDC_ERR_CUDA, cudaGetErrorString(e));
  if (!on_device(sum1) || !on_device(sum2) || (mean && !on_device(mean)) ||
      (relerr && !on_device(relerr)))
    return fail(MCDC_ERR_INVALID, "outputs must be device pointers");
  Scratch *sc = nullptr;
  if (int rc = scratch_address(pr->device, &sc)) return rc;

  cudaStream_t s = (cudaStream_t)stream;
  const size_t nb = (size_t)pr->P.n_bins;
#define CKN(call)                                                                   \
  do {                                                                              \
    cudaError_t e_ = (call);                                                        \
    if (e_ != cudaSuccess) return fail(MCDC_ERR_CUDA, cudaGetErrorString(e_));      \
  } while (0)
  // clear what starts at zero: counters, accumulators, outputs, batch tally
  CKN(cudaMemsetAsync(sc->work, 0, sizeof(unsigned long long) * (global ? n_batches : 1), s));
  CKN(cudaMemsetAsync(sc->region, 0, sizeof(sc->region), s));
  CKN(cudaMemsetAsync(&sc->stats, 0, sizeof(Stats), s));
  CKN(cudaMemsetAsync(sc->error, 0, sizeof(sc->error), s));
  CKN(cudaMemsetAsync(&sc->children, 0, sizeof(sc->children), s));
  CKN(cudaMemsetAsync(sum1, 0, nb * 8, s));
  CKN(cudaMemsetAsync(sum2, 0, nb * 8, s));
  if (global) CKN(cudaMemsetAsync(sc->tally, 0, nb * 8, s));

  RunArgs A{};
  A.n_hist = n_histories;
  A.offset = hist_offset;
  A.seed = seed;
  A.rk = round_keys(seed);
  A.n_batches = n_batches;
  A.sum1 = sum1;
  A.sum2 = sum2;
  A.region = sc->region;
  A.stats = &sc->stats;
  A.records = nullptr;
  A.n_records = 0;
  A.error = sc->error;
  A.overflow = pr->overflow;
  A.overflow_cap = pr->overflow_cap;
  A.overflow_tail = pr->opt.overflow_tail;
  A.warp_aggregate = pr->warp_aggregate;
  A.tally = global ? sc->tally : nullptr;
  if (pr->opt.max_children >= 0) {
    // the budget of mcdc_run_ex: the option, else 4096 children per history
    // and at least 2^27
    A.children_made = &sc->children;
    A.children_budget = pr->opt.max_children > 0
                            ? (unsigned long long)pr->opt.max_children
                            : std::max<unsigned long long>(1ull << 27, 4096ull * n_histories);
  }
  if (!global) {
    A.work = sc->work;
    CKN(launch_track(pr->key, pr->grid, pr->block, pr->smem, s, pr->P, A, pr->L));
  } else {
    for (int b = 0; b < n_batches; ++b) {
      A.work = sc->work + b;
      A.batch = b;
      const uint64_t per = n_histories / n_batches + 1;
      A.chunk = (int)std::max<uint64_t>(
          32, std::min<uint64_t>(pr->S, per / ((uint64_t)pr->grid * 4) + 1));
      CKN(launch_track(pr->key, pr->grid, pr->block, pr->smem, s, pr->P, A, pr->L));
      CKN(launch_fold(s, pr->P, sc->tally, sum1, sum2, nullptr, sc->region + 5, sc->region,
                      pr->sms));
    }
  }
  if (mean || relerr)
    CKN(launch_finalize(s, (int64_t)nb, sum1, sum2, n_histories, n_batches, pr->P.volume, mean,
                        relerr, pr->sms));
#undef CKN
  return MCDC_OK;
}
