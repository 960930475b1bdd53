// comb.h -- host entry points of the population-control comb (comb.cu).
#pragma once
#include <cstddef>
#include <cuda_runtime.h>

#include "launch.h"

namespace mcdc {

// One step's comb over all batches.  The step's input is laid out batch by
// batch: in the first step the histories (batch b at [batch_start(N, B, b),
// batch_start(N, B, b + 1))), after a comb one chunk of M particles per batch
// that still had particles, in batch order.  The tracker wrote every banked
// particle at its input position (bank, w); other positions hold weight 0.
struct CombArgs {
  const void *bank;             // banked particles by input position (pool layout, bank_cap slots)
  long long bank_cap;
  const double *w;              // [n_in] their weights, 0 where nothing was banked
  int n_in;                     // input positions of the step (N, or B x M after a comb)
  bool first_step;              // the input is the histories themselves
  const int32_t *live_in;       // [B] after a comb: batch of chunk c; [0] <- chunk count
  const int32_t *n_live_in;     //   (device; unused in the first step)
  int32_t *live_out;            // [B] batches combed by this step, in order
  int32_t *n_live_out;          // their count (device)
  void *out;                    // combed bank: chunk c (batch live_out[c]) at [c M, (c + 1) M)
  long long out_cap;            //   (pool layout, out_cap slots)
  int dim;                      // 1 or 3
  unsigned long long *out_count;   // set to M x n_live_out
  const unsigned long long *banked;  // particles the tracker banked this step (device)
  int M;                        // particles per batch after the comb
  uint64_t offset;              // first history id of the run
  uint64_t n_hist;              // histories in the run
  int B;                        // batches
  int step;                     // index of the time bin that just ended
  RoundKeys rk;
  int32_t *key;                 // [n_in] scratch: segment of each input position (the scan's keys)
  double *S;                    // [n_in] scratch: per-segment exclusive sums of w
  int32_t *seg;                 // [3 B] scratch: per segment first, end, output chunk (-1: none)
  double *segd;                 // [4 B] scratch: per segment W, xi, W / M, M / W
  void *temp;                   // CUB scratch
  size_t temp_bytes;
  Stats *stats;
  int32_t *error;               // the run's error words (bounds checks of the checked build)
};

// CUB scratch bytes for up to cap input positions.
size_t comb_temp_bytes(int cap);
// Scans and combs one step's bank (all on stream s).
cudaError_t comb_bank(const TrackKey &key, cudaStream_t s, const CombArgs &c);
// Bytes per slot of a particle bank in the pool layout of the run's precision.
size_t bank_slot_bytes(const TrackKey &key);

}  // namespace mcdc
