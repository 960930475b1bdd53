// comb.cu -- population control: the comb of a batch's census bank.
//
// Particles that reached an interior census edge sit in the bank in the
// order the warps appended them.  The comb first orders them by (history id,
// serial) -- one radix sort of the 64-bit key (hid - h0) << 32 | serial -- so
// that the result does not depend on scheduling, takes the exclusive prefix
// sum S of their weights in that order (W = S[n-1] + w[n-1]), and emits M
// particles: tooth k at (k + xi) W / M copies the particle whose interval
// [S_i, S_i + w_i) holds it, with weight W / M, a serial hashed from (parent
// serial, step, k) and a fresh counter.  xi comes from the block (key seed;
// counter 0xFFFFFFFC, step, first history id of the batch).
#include <cub/device/device_radix_sort.cuh>
#include <cub/device/device_scan.cuh>

#include "comb.h"
#include "tracker.cuh"

namespace mcdc {

template <class PT>
__global__ void k_comb_keys(const PT *__restrict__ bank, int n, uint64_t h0,
                            unsigned long long *__restrict__ keys, uint32_t *__restrict__ idx) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const PT &q = bank[i];
    keys[i] = ((unsigned long long)(q.hid - h0) << 32) | (unsigned long long)q.serial;
    idx[i] = (uint32_t)i;
  }
}

template <class PT>
__global__ void k_comb_weights(const PT *__restrict__ bank, const uint32_t *__restrict__ order,
                               int n, double *__restrict__ w) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    w[i] = (double)bank[order[i]].w;
}

template <class PT>
__global__ void k_comb_teeth(const PT *__restrict__ bank, const uint32_t *__restrict__ order,
                             const double *__restrict__ S, const double *__restrict__ w, int n,
                             int M, RoundKeys rk, uint32_t step, uint64_t h0, PT *__restrict__ out,
                             unsigned long long *out_count, Stats *stats) {
  using R = decltype(PT::w);
  const double W = S[n - 1] + w[n - 1];
  const U4 r = philox4x32_10_rk(0xFFFFFFFCu, step, (uint32_t)h0, (uint32_t)(h0 >> 32), rk);
  const double xi = u01_f64(r.a, r.b);
  const double wn = W / (double)M;
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < M; k += gridDim.x * blockDim.x) {
    const double tooth = ((double)k + xi) * wn;
    int lo = 0, hi = n - 1;            // the last i with S[i] <= tooth
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (S[mid] <= tooth) lo = mid; else hi = mid - 1;
    }
    PT q = bank[order[lo]];
    const U4 h = philox4x32_10_rk(0xFFFFFFFDu, q.serial, step, (uint32_t)k, rk);
    q.serial = h.a;
    q.ctr = 0;
    q.w = (R)wn;
    out[k] = q;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    *out_count = (unsigned long long)M;
    atomicAdd(&stats->pc_combs, 1ull);
    atomicAdd(&stats->pc_in, (unsigned long long)n);
    atomicAdd(&stats->pc_out, (unsigned long long)M);
    atomicAdd(&stats->w_pc_in, W);
    atomicAdd(&stats->w_pc_out, (double)M * (double)(R)wn);
  }
}

size_t comb_temp_bytes(int cap) {
  size_t a = 0, b = 0;
  cub::DeviceRadixSort::SortPairs(nullptr, a, (const unsigned long long *)nullptr,
                                  (unsigned long long *)nullptr, (const uint32_t *)nullptr,
                                  (uint32_t *)nullptr, cap, 0, 64);
  cub::DeviceScan::ExclusiveSum(nullptr, b, (const double *)nullptr, (double *)nullptr, cap);
  return a > b ? a : b;
}

template <class PT>
static cudaError_t comb_impl(cudaStream_t s, const CombArgs &c) {
  const PT *bank = reinterpret_cast<const PT *>(c.bank);
  const int threads = 256;
  const int blocks_n = (int)std::min<long long>((c.n + threads - 1) / threads, 4096);
  k_comb_keys<PT><<<blocks_n, threads, 0, s>>>(bank, c.n, c.h0, c.keys[0], c.idx[0]);
  size_t tb = c.temp_bytes;
  cudaError_t e = cub::DeviceRadixSort::SortPairs(c.temp, tb, c.keys[0], c.keys[1], c.idx[0],
                                                  c.idx[1], c.n, 0, c.key_bits, s);
  if (e != cudaSuccess) return e;
  k_comb_weights<PT><<<blocks_n, threads, 0, s>>>(bank, c.idx[1], c.n, c.w);
  tb = c.temp_bytes;
  e = cub::DeviceScan::ExclusiveSum(c.temp, tb, c.w, c.S, c.n, s);
  if (e != cudaSuccess) return e;
  const int blocks_m = (int)std::min<long long>((c.M + threads - 1) / threads, 4096);
  k_comb_teeth<PT><<<blocks_m, threads, 0, s>>>(bank, c.idx[1], c.S, c.w, c.n, c.M, c.rk,
                                                (uint32_t)c.step, c.h0,
                                                reinterpret_cast<PT *>(c.out), c.out_count,
                                                c.stats);
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
