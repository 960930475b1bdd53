// comb.h -- host entry points of the population-control comb (comb.cu).
#pragma once
#include <cstddef>
#include <cuda_runtime.h>

#include "launch.h"

namespace mcdc {

struct CombArgs {
  const void *bank;             // census bank: n particles of the run's precision, all batches
  int n;                        // particles in the bank (>= 1)
  void *out;                    // combed bank: M per batch that had particles, batch by batch
  int M;                        // particles per batch after the comb
  unsigned long long *out_count;   // set to M x (batches that had particles)
  uint64_t offset;              // first history id of the run
  uint64_t n_hist;              // histories in the run
  int B;                        // batches
  int step;                     // index of the time bin that just ended
  RoundKeys rk;
  int key_bits;                 // 32 + bits of the run's history count
  unsigned long long *keys[2];  // [cap] sort keys in / out
  uint32_t *idx[2];             // [cap] bank positions in / out
  double *w, *S;                // [cap] weights in key order and their per-batch exclusive sums
  int32_t *bid;                 // [cap] batch of each particle in key order
  int32_t *seg;                 // [3 B]: first, end and output base of each batch's run
  void *temp;                   // CUB scratch
  size_t temp_bytes;
  Stats *stats;
};

// CUB scratch bytes for a bank of up to cap particles.
size_t comb_temp_bytes(int cap);
// Sorts, scans and combs one bank (all on stream s).
cudaError_t comb_bank(const TrackKey &key, cudaStream_t s, const CombArgs &c);
// Bytes of one particle record of the run's precision.
size_t part_bytes(const TrackKey &key);

}  // namespace mcdc
