// comb.cu -- population control: the comb of the census bank.
//
// Every batch is an independent time-stepped simulation, and one launch runs
// the current step of all of them.  Particles that reached an interior
// census edge sit in one bank in the order the warps appended them.  The comb
// orders them by (history id, serial) -- one radix sort of the 64-bit key
// (hid - offset) << 32 | serial; batches are contiguous history ranges, so
// this also groups them by batch -- and does not depend on scheduling.  Per
// batch it takes the exclusive prefix sum S of the weights in that order
// (W_b = S[end-1] + w[end-1]) and emits M particles: tooth k at
// (k + xi_b) W_b / M copies the particle whose interval [S_i, S_i + w_i)
// holds it, with weight W_b / M, a serial hashed from (parent serial, step,
// k) and a fresh counter.  xi_b comes from the block (key seed; counter
// 0xFFFFFFFC, step, first history id of the batch).
#include <cub/device/device_radix_sort.cuh>
#include <cub/device/device_scan.cuh>

#include "comb.h"
#include "tracker.cuh"

namespace mcdc {

template <class PT>
__global__ void k_comb_keys(const PT *__restrict__ bank, int n, uint64_t offset,
                            unsigned long long *__restrict__ keys, uint32_t *__restrict__ idx) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const PT &q = bank[i];
    keys[i] = ((unsigned long long)(q.hid - offset) << 32) | (unsigned long long)q.serial;
    idx[i] = (uint32_t)i;
  }
}

// weights and batch ids in key order; first and end of every batch's run
template <class PT>
__global__ void k_comb_gather(const PT *__restrict__ bank, const uint32_t *__restrict__ order,
                              int n, uint64_t offset, uint64_t n_hist, int B,
                              double *__restrict__ w, int32_t *__restrict__ bid,
                              int32_t *__restrict__ seg) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const PT &q = bank[order[i]];
    w[i] = (double)q.w;
    const int b = batch_of(n_hist, B, q.hid - offset);
    bid[i] = b;
    const int bp = i > 0 ? batch_of(n_hist, B, bank[order[i - 1]].hid - offset) : -1;
    const int bn = i < n - 1 ? batch_of(n_hist, B, bank[order[i + 1]].hid - offset) : -1;
    if (bp != b) seg[b] = i;               // first of batch b
    if (bn != b) seg[B + b] = i + 1;       // end of batch b
  }
}

// output base of every batch that has particles; comb statistics
template <class PT>
__global__ void k_comb_bases(const double *__restrict__ S, const double *__restrict__ w, int n,
                             int M, int B, int32_t *__restrict__ seg,
                             unsigned long long *out_count, Stats *stats) {
  using R = decltype(PT::w);
  int base = 0, combs = 0;
  double win = 0.0, wout = 0.0;
  for (int b = 0; b < B; ++b) {
    const int s0 = seg[b], s1 = seg[B + b];
    if (s1 > s0) {
      seg[2 * B + b] = base;
      base += M;
      combs += 1;
      const double W = S[s1 - 1] + w[s1 - 1];
      win += W;
      wout += (double)M * (double)(R)(W / (double)M);
    } else {
      seg[2 * B + b] = -1;
    }
  }
  *out_count = (unsigned long long)base;
  stats->pc_combs += (unsigned long long)combs;
  stats->pc_in += (unsigned long long)n;
  stats->pc_out += (unsigned long long)base;
  stats->w_pc_in += win;
  stats->w_pc_out += wout;
}

template <class PT>
__global__ void k_comb_teeth(const PT *__restrict__ bank, const uint32_t *__restrict__ order,
                             const double *__restrict__ S, const double *__restrict__ w,
                             const int32_t *__restrict__ seg, int M, int B, RoundKeys rk,
                             uint32_t step, uint64_t offset, uint64_t n_hist,
                             PT *__restrict__ out) {
  using R = decltype(PT::w);
  const long long total = (long long)B * M;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    const int b = (int)(t / M), k = (int)(t % M);
    const int base = seg[2 * B + b];
    if (base < 0) continue;                       // the batch has no particle left
    const int s0 = seg[b], s1 = seg[B + b];
    const double W = S[s1 - 1] + w[s1 - 1];
    const uint64_t h0 = offset + batch_start(n_hist, B, b);
    const U4 r = philox4x32_10_rk(0xFFFFFFFCu, step, (uint32_t)h0, (uint32_t)(h0 >> 32), rk);
    const double xi = u01_f64(r.a, r.b);
    const double wn = W / (double)M;
    const double tooth = ((double)k + xi) * wn;
    int lo = s0, hi = s1 - 1;                     // the last i with S[i] <= tooth
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (S[mid] <= tooth) lo = mid; else hi = mid - 1;
    }
    PT q = bank[order[lo]];
    const U4 h = philox4x32_10_rk(0xFFFFFFFDu, q.serial, step, (uint32_t)k, rk);
    q.serial = h.a;
    q.ctr = 0;
    q.tau = -1.0f;            // FP32 modes: every copy draws its own optical depth
    q.w = (R)wn;
    out[base + k] = q;
  }
}

size_t comb_temp_bytes(int cap) {
  size_t a = 0, b = 0;
  cub::DeviceRadixSort::SortPairs(nullptr, a, (const unsigned long long *)nullptr,
                                  (unsigned long long *)nullptr, (const uint32_t *)nullptr,
                                  (uint32_t *)nullptr, cap, 0, 64);
  cub::DeviceScan::ExclusiveSumByKey(nullptr, b, (const int32_t *)nullptr,
                                     (const double *)nullptr, (double *)nullptr, cap);
  return a > b ? a : b;
}

template <class PT>
static cudaError_t comb_impl(cudaStream_t s, const CombArgs &c) {
  const PT *bank = reinterpret_cast<const PT *>(c.bank);
  const int threads = 256;
  const int blocks_n = (int)std::min<long long>((c.n + threads - 1) / threads, 4096);
  k_comb_keys<PT><<<blocks_n, threads, 0, s>>>(bank, c.n, c.offset, c.keys[0], c.idx[0]);
  size_t tb = c.temp_bytes;
  cudaError_t e = cub::DeviceRadixSort::SortPairs(c.temp, tb, c.keys[0], c.keys[1], c.idx[0],
                                                  c.idx[1], c.n, 0, c.key_bits, s);
  if (e != cudaSuccess) return e;
  e = cudaMemsetAsync(c.seg, 0, sizeof(int32_t) * 3 * (size_t)c.B, s);
  if (e != cudaSuccess) return e;
  k_comb_gather<PT><<<blocks_n, threads, 0, s>>>(bank, c.idx[1], c.n, c.offset, c.n_hist, c.B,
                                                 c.w, c.bid, c.seg);
  tb = c.temp_bytes;
  e = cub::DeviceScan::ExclusiveSumByKey(c.temp, tb, c.bid, c.w, c.S, c.n,
                                         ::cuda::std::equal_to<>(), s);
  if (e != cudaSuccess) return e;
  k_comb_bases<PT><<<1, 1, 0, s>>>(c.S, c.w, c.n, c.M, c.B, c.seg, c.out_count, c.stats);
  const long long teeth = (long long)c.B * c.M;
  const int blocks_t = (int)std::min<long long>((teeth + threads - 1) / threads, 8192);
  k_comb_teeth<PT><<<blocks_t, threads, 0, s>>>(bank, c.idx[1], c.S, c.w, c.seg, c.M, c.B, c.rk,
                                                (uint32_t)c.step, c.offset, c.n_hist,
                                                reinterpret_cast<PT *>(c.out));
  return cudaGetLastError();
}

cudaError_t comb_bank(const TrackKey &key, cudaStream_t s, const CombArgs &c) {
  if (key.f64) return comb_impl<PartOf<PrecF64>>(s, c);
  if (key.local) return comb_impl<PartOf<PrecF32L>>(s, c);
  return comb_impl<PartOf<PrecF32>>(s, c);
}

size_t part_bytes(const TrackKey &key) {
  if (key.f64) return sizeof(PartOf<PrecF64>);
  if (key.local) return sizeof(PartOf<PrecF32L>);
  return sizeof(PartOf<PrecF32>);
}

}  // namespace mcdc
