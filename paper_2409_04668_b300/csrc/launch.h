// launch.h -- host-side entry points into the kernel translation units.
#pragma once
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>
#include <string>
#include "common.cuh"

namespace mcdc {

// NVTX range for the scope (shows the library's phases in Nsight timelines)
struct NvtxRange {
  explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange &) = delete;
  NvtxRange &operator=(const NvtxRange &) = delete;
};

// The cell box of the scalar region, tested per bin without 64-bit division.
struct RegionTest {
  bool whole, narrow;
  long long per_cell;
  __device__ explicit RegionTest(const DevProblem &P) {
    whole = P.region_lo[0] == 0 && P.region_lo[1] == 0 && P.region_lo[2] == 0 &&
            P.region_hi[0] >= P.n[0] && P.region_hi[1] >= P.n[1] && P.region_hi[2] >= P.n[2];
    narrow = P.n_bins < (1ll << 31);
    per_cell = (long long)P.G * P.T1;
  }
  __device__ bool operator()(const DevProblem &P, long long q) const {
    if (whole) return true;
    int ci, cj, ck;
    if (narrow) {
      const uint32_t cell = (uint32_t)q / (uint32_t)per_cell;
      const uint32_t row = cell / (uint32_t)P.n[0];
      ci = (int)(cell - row * (uint32_t)P.n[0]);
      ck = (int)(row / (uint32_t)P.n[1]);
      cj = (int)(row - (uint32_t)ck * (uint32_t)P.n[1]);
    } else {
      const long long cell = q / per_cell;
      ci = (int)(cell % P.n[0]);
      cj = (int)((cell / P.n[0]) % P.n[1]);
      ck = (int)(cell / ((long long)P.n[0] * P.n[1]));
    }
    return ci >= P.region_lo[0] && ci < P.region_hi[0] && cj >= P.region_lo[1] &&
           cj < P.region_hi[1] && ck >= P.region_lo[2] && ck < P.region_hi[2];
  }
};

struct Layout;

struct MultiArgs;

struct TrackKey {
  bool f64;     // FP64 everywhere
  bool local;   // FP32 cell-local positions (when !f64)
  bool multi = false;   // batched problems (work items over several problems)
  bool shared;
  int dim;   // 1 or 3
  bool net = false;     // per-event network windows (global tally, single problem)
  bool pc = false;      // population control (global tally, single problem)
  bool vr = false;      // weights vary: a window table is set, or implicit capture is on
};

// Launches the persistent tracker for one configuration (MA: batched mode only).
cudaError_t launch_track(const TrackKey &key, int grid, int block, int smem_bytes,
                         cudaStream_t stream, const DevProblem &P, const RunArgs &A,
                         const Layout &L, const MultiArgs *MA = nullptr);
// Raises the dynamic shared-memory limit of that instantiation.
cudaError_t prepare_track(const TrackKey &key, int smem_bytes);
// Registers per thread of that instantiation (for occupancy decisions).
int track_regs(const TrackKey &key);
// The window lower bounds at n given states (positions x[3 n], times, groups)
// through that precision's own evaluation (k_net_lower); all device pointers.
cudaError_t launch_net_lower(const TrackKey &key, cudaStream_t s, const DevProblem &P,
                             const double *x, const double *t, const int32_t *g, long long n,
                             double *out, int sms);
// Resident CTAs per SM for a block size and dynamic shared memory.
int track_occupancy(const TrackKey &key, int block, int smem_bytes);

// batch fold (global tally mode): sum1 += x, sum2 += x^2, region partial, x = 0;
// combined estimator: both halves of the tally and sum12 += x_track x_collision
// (sum12 unused otherwise); region_batch [2], region [5]
cudaError_t launch_fold(cudaStream_t s, const DevProblem &P, double *tally, double *sum1,
                        double *sum2, double *sum12, double *region_batch, double *region,
                        int sms);
// the same for an FP32 batch tally (the FP32 modes' slices), folded in FP64
cudaError_t launch_fold(cudaStream_t s, const DevProblem &P, float *tally, double *sum1,
                        double *sum2, double *sum12, double *region_batch, double *region,
                        int sms);
// all B tally slices of a one-launch run (slice b at tally + b nt) in one
// pass: per bin the batch values in batch order into sum1, sum2 (and sum12),
// the slices zeroed, each batch's region sum into rb[b] (rb[B + b]: the
// collision half; rb: 2 B zeroed doubles), then region[0..4] as B calls of
// launch_fold would leave it.  B <= 2048.
cudaError_t launch_fold_slices(cudaStream_t s, const DevProblem &P, double *tally, long long nt,
                               int B, double *sum1, double *sum2, double *sum12, double *rb,
                               double *region, int sms);
cudaError_t launch_fold_slices(cudaStream_t s, const DevProblem &P, float *tally, long long nt,
                               int B, double *sum1, double *sum2, double *sum12, double *rb,
                               double *region, int sms);
// mean and relative error from the batch sums (host-side formula mirrored)
cudaError_t launch_finalize(cudaStream_t s, int64_t n_bins, const double *sum1,
                            const double *sum2, uint64_t n_hist, int n_batches, double volume,
                            double *mean, double *relerr, int sms);
// combined estimator: minimum-variance combination of the two halves per bin;
// parts (or nullptr): [5][n_bins] track mean, relerr, collision mean, relerr, a
cudaError_t launch_finalize_combined(cudaStream_t s, int64_t n_bins, const double *sum1,
                                     const double *sum2, const double *sum12, uint64_t n_hist,
                                     int n_batches, double volume, double *mean, double *relerr,
                                     double *parts, int sms);
// mean and relative error of one scalar from its batch sums, on the host
void scalar_moments(double s1, double s2, uint64_t n_hist, int n_batches, double volume,
                    double *mean, double *relerr);
// the combination for one scalar (region[0..4] as in launch_fold), on the host
void combine_scalar(const double r[5], uint64_t n_hist, int n_batches, double volume,
                    double *mean, double *relerr, double *alpha);

// Records the calling thread's error message (read by mcdc_last_error).
int set_error(int code, const std::string &msg);
// message of a failed bounds check from a run's error words (checked build)
std::string check_message(const int32_t *words);
}  // namespace mcdc
struct mcdc_problem;
namespace mcdc {
// Allocates the per-warp overflow stacks once weight windows are on.
int ensure_overflow_for(mcdc_problem *pr);
// Selects the problem's tracker instantiation (per-event network windows, a
// window table -- or implicit capture --, or analog) and redoes its launch shape.
int set_track_kernel(mcdc_problem *pr, bool net, bool ww);
// Drops every cached batched-run plan that holds the problem with this uid
// (called when the problem is destroyed).
void batched_forget(uint64_t uid);
// The device's stream-ordered memory pool of problems (nullptr where pools
// are unavailable), for temporaries allocated and freed on a caller's stream.
cudaMemPool_t device_mem_pool(int dev);
// importance network (mlp.cu)
cudaError_t mlp_prepare();
int64_t mlp_param_count(int n_in);

}  // namespace mcdc
