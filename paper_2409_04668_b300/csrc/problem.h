// problem.h -- the library's private view of a problem handle: device
// tables, launch shape and the device buffers a run uses.
#pragma once
#include <vector>

#include "../../include/mcdc.h"
#include "launch.h"
#include "tracker.cuh"

struct mcdc_problem {
  uint64_t uid = 0;             // unique over the process (batched-run plans key on it)
  int user_aggregate = 0;       // the caller's warp_aggregate and ctas_per_sm (0: the tuner's)
  int user_cps = 0;
  int user_block = 0;           // the caller's block_size (0: the tuner's)
  uint64_t p_version = 0;       // bumped whenever P changes after create (windows):
                                // cached batched plans hold a copy of P
  int device = 0;
  int sms = 0;
  mcdc::DevProblem P{};
  mcdc_options opt{};
  // host copies needed later
  std::vector<double> edges;
  int dim = 3;
  mcdc::TrackKey key{};
  // launch shape
  int block = 256, S = 512, ctas_per_sm = 1, grid = 0, smem = 0;
  int dyn_max = 0;            // dynamic shared memory the tracker may use per CTA
  mcdc::Layout L{};
  int tally_mode = MCDC_TALLY_SHARED;
  int warp_aggregate = 0;
  int batch_per_cta = 2;      // shared tally: default batches = grid x this
  int overflow_cap = 0;
  // device memory
  std::vector<void *> allocs;        // cudaMalloc'ed, freed with cudaFree
  std::vector<void *> pool_allocs;   // from the device's memory pool (dalloc)
  double *sum1 = nullptr, *sum2 = nullptr, *tally = nullptr, *region = nullptr,
         *region_batch = nullptr, *mean_tmp = nullptr, *rel_tmp = nullptr;
  double *sum12 = nullptr;      // combined estimator: [n_bins]
  unsigned long long *children = nullptr;   // weight windows: children made in the run
  double *parts_tmp = nullptr;  // combined estimator: [5][n_bins] staging of host parts_out
  mcdc::Stats *stats = nullptr;
  int32_t *error = nullptr;
  unsigned long long *work = nullptr;   // [max batches] work counters
  int work_slots = 0;
  void *overflow = nullptr;
  void *spill[2] = {nullptr, nullptr};   // device-wide banks of spilled children
  unsigned long long *spill_cnt = nullptr; // [4]: counts of both banks, input cursor
  unsigned long long spill_cap = 0;
  unsigned long long *h_spill = nullptr;   // pinned copy of a count
  size_t overflow_bytes = 0;
  mcdc::Record *rec_tmp = nullptr;
  uint64_t rec_cap = 0;
  double *ww64 = nullptr;      // the last window table set or baked
  bool ww_table_valid = false;
  float *ww32 = nullptr;
  double *net64 = nullptr;      // per-event windows: network parameters
  float *net32 = nullptr;
  size_t net_cap = 0;
  uint32_t *netfrag = nullptr;  // the same network as binary16 mma.sync fragments (kNetFragWords)
  // population control: census bank (by input position), combed bank and
  // the comb's scratch
  int pc_cap = 0;                          // input positions the census bank holds
  long long pc_combed_cap = 0;             // particles the combed bank holds
  long long pc_tally_bins = 0;             // entries of the per-batch tally slices
  void *pc_tally = nullptr;                // [batches][n_tally]: FP64 in FP64 mode, FP32
                                           // in the FP32 modes (folded in FP64)
  int slice_bytes = 8;                     // bytes per slice entry (8 or 4)
  double *slice_rb = nullptr;              // [2 batches] per-batch region sums of the slices
  bool slices_dirty = false;               // a run left scores in the slices (returned early)
  bool tally_dirty = false;                // likewise for the batch tally
  int32_t *pc_key = nullptr, *pc_seg = nullptr, *pc_live = nullptr;
  double *pc_segd = nullptr;
  int pc_seg_cap = 0;
  void *pc_bank = nullptr, *pc_combed = nullptr;
  unsigned long long *pc_cnt = nullptr;    // [4]: banked count, combed count, cursor
  double *pc_w = nullptr, *pc_S = nullptr; // [cap] census weights, per-batch exclusive sums
  void *pc_temp = nullptr;
  size_t pc_temp_bytes = 0;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr, ev2 = nullptr;
  // host staging: words of one pinned block from a process-wide pool
  void *pinned = nullptr;
  mcdc::Stats *h_stats = nullptr;   // pinned
  int32_t *h_error = nullptr; // pinned
};
