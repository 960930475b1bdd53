// comb.cu -- population control: the comb of the census bank.
//
// Every batch is an independent time-stepped simulation, and one launch runs
// the current step of all of them.  A particle that reaches an interior
// census edge is written at its position in the step's input (nothing splits
// under population control, so every input yields at most one), which keeps
// the bank in the order the step ran its particles -- history order in the
// first step, tooth order after a comb -- without a sort and independently of
// scheduling.  Positions whose particle ended hold weight 0.  The input is
// laid out batch by batch, so a segmented exclusive scan gives every batch's
// cumulative weights S (W_b = S[end-1] + w[end-1]); the comb then emits M
// particles per batch: tooth k at T_k = (k + xi_b) W_b / M copies the last
// particle i with S_i <= T_k, with weight W_b / M, a serial hashed from
// (parent serial, step, k) and a fresh counter.  xi_b comes from the block
// (key seed; counter 0xFFFFFFFC, step, first history id of the batch).  One
// thread per banked particle finds its teeth, a contiguous range because T_k
// does not decrease with k, and writes them.
#include <cub/device/device_scan.cuh>

#include "comb.h"
#include "tracker.cuh"

namespace mcdc {

// segment (batch in the first step, chunk of M afterwards) of every input position
__global__ void k_comb_keys(int n, bool first_step, uint64_t n_hist, int B, int M,
                            int32_t *__restrict__ key) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    key[i] = first_step ? batch_of(n_hist, B, (uint64_t)i) : i / M;
}

// Per segment: its range, total weight, xi and tooth spacing; the output
// chunk of every segment that has weight; comb statistics.
template <class PR>
__global__ void k_comb_bases(CombArgs c) {
  using R = typename PR::R;
  const int nseg = c.first_step ? c.B : *c.n_live_in;
  int chunks = 0;
  double win = 0.0, wout = 0.0;
  for (int q = 0; q < c.B; ++q) {
    c.seg[2 * c.B + q] = -1;
    if (q >= nseg) continue;
    const int b = c.first_step ? q : c.live_in[q];
    const int s0 = c.first_step ? (int)batch_start(c.n_hist, c.B, b) : q * c.M;
    const int s1 = c.first_step ? (int)batch_start(c.n_hist, c.B, b + 1) : (q + 1) * c.M;
    const double W = s1 > s0 ? c.S[s1 - 1] + c.w[s1 - 1] : 0.0;
    if (!(W > 0.0)) continue;
    const uint64_t h0 = c.offset + batch_start(c.n_hist, c.B, b);
    const U4 r = philox4x32_10_rk(0xFFFFFFFCu, (uint32_t)c.step, (uint32_t)h0,
                                  (uint32_t)(h0 >> 32), c.rk);
    c.seg[q] = s0;
    c.seg[c.B + q] = s1;
    c.seg[2 * c.B + q] = chunks;
    c.segd[q] = W;
    c.segd[c.B + q] = u01_f64(r.a, r.b);
    c.segd[2 * c.B + q] = W / (double)c.M;
    c.segd[3 * c.B + q] = (double)c.M / W;
    c.live_out[chunks] = b;
    chunks += 1;
    win += W;
    wout += (double)c.M * (double)(R)(W / (double)c.M);
  }
  *c.n_live_out = chunks;
  *c.out_count = (unsigned long long)chunks * (unsigned long long)c.M;
  c.stats->pc_combs += (unsigned long long)chunks;
  c.stats->pc_in += *c.banked;
  c.stats->pc_out += (unsigned long long)chunks * (unsigned long long)c.M;
  c.stats->w_pc_in += win;
  c.stats->w_pc_out += wout;
}

__device__ __forceinline__ double comb_tooth(int k, double xi, double wn) {
  return ((double)k + xi) * wn;
}

// First k in [0, M] with T_k >= s (M if none).  The estimate e = s M / W - xi
// is within ~8 u max(M, 1) of the exact boundary in units of teeth (u = 2^-53:
// the rounding of e, of M / W and of T_k itself), at most 2e-6 for M < 2^31,
// so a ceiling whose distance from e exceeds 1e-5 is the answer; closer cases
// are settled by evaluating T_k as defined.  (FP64 arithmetic is scarce on
// this GPU: the fast path costs a handful of FP64 operations, a division
// several times that.)
__device__ __forceinline__ int first_tooth_at_or_after(double s, double xi, double wn,
                                                      double inv, int M) {
  const double e = fma(s, inv, -xi);
  const double ce = ceil(e);
  if (ce <= 0.0) {
    if (e < -1e-5) return 0;
  } else if (ce >= (double)M) {
    if (e > (double)M - 1.0 + 1e-5) return M;
  } else if (ce - e > 1e-5 && ce - e < 1.0 - 1e-5) {
    return (int)ce;
  }
  int k = ce < 0.0 ? 0 : (ce > (double)M ? M : (int)ce);
  while (k > 0 && comb_tooth(k - 1, xi, wn) >= s) --k;
  while (k < M && comb_tooth(k, xi, wn) < s) ++k;
  return k;
}

// Banked particle i owns the teeth with S_i <= T_k < S_j, j the next banked
// particle of its segment (all teeth from S_i on if there is none): the
// assignment "last particle with S <= T_k" made per tooth.  Each thread finds
// the first tooth at or after S_i and at or after S_j itself (a few FP64
// operations each), so no pass writes them out first.  Both banks have the
// pool's structure-of-arrays layout.
template <class PR, int DIM>
__global__ void k_comb_teeth(CombArgs c) {
  using R = typename PR::R;
  const Bank<PR> in = bank_view<PR>(const_cast<void *>(c.bank), c.bank_cap, DIM);
  const Bank<PR> out = bank_view<PR>(c.out, c.out_cap, DIM);
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < c.n_in; i += gridDim.x * blockDim.x) {
    if (!(c.w[i] > 0.0)) continue;
    const int q = c.first_step ? batch_of(c.n_hist, c.B, (uint64_t)i) : i / c.M;
    const int chunk = c.seg[2 * c.B + q];
    if (chunk < 0) continue;
    const int s1 = c.seg[c.B + q];
    const double xi = c.segd[c.B + q], wn = c.segd[2 * c.B + q], inv = c.segd[3 * c.B + q];
    const int k0 = first_tooth_at_or_after(c.S[i], xi, wn, inv, c.M);
    int j = i + 1;
    while (j < s1 && !(c.w[j] > 0.0)) ++j;
    const int k1 = j < s1 ? first_tooth_at_or_after(c.S[j], xi, wn, inv, c.M) : c.M;
    if (k1 <= k0) continue;
    if (!MCDC_CHK(c.error, CHK_COMB_IN, i < c.bank_cap, i)) continue;
    PartOf<PR> parent;
    in.load(i, parent, DIM);
    const R wc = (R)wn;
    for (int k = k0; k < k1; ++k) {
      PartOf<PR> p = parent;
      const U4 h = philox4x32_10_rk(0xFFFFFFFDu, p.serial, (uint32_t)c.step, (uint32_t)k, c.rk);
      p.serial = h.a;
      p.ctr = 0;
      p.tau = -1.0f;            // FP32 modes: every copy draws its own optical depth
      p.w = wc;
      if (!MCDC_CHK(c.error, CHK_COMB_OUT,
                    k >= 0 && (long long)chunk * c.M + k < c.out_cap, (long long)chunk * c.M + k))
        continue;
      out.store(chunk * c.M + k, p, DIM);
    }
  }
}

size_t comb_temp_bytes(int cap) {
  size_t b = 0;
  cub::DeviceScan::ExclusiveSumByKey(nullptr, b, (const int32_t *)nullptr,
                                     (const double *)nullptr, (double *)nullptr, cap);
  return b;
}

template <class PR>
static cudaError_t comb_impl(cudaStream_t s, const CombArgs &c) {
  const int threads = 256;
  const int blocks = (int)std::max<long long>(1, std::min<long long>((c.n_in + threads - 1) / threads, 8192));
  k_comb_keys<<<blocks, threads, 0, s>>>(c.n_in, c.first_step, c.n_hist, c.B, c.M, c.key);
  size_t tb = c.temp_bytes;
  cudaError_t e = cub::DeviceScan::ExclusiveSumByKey(c.temp, tb, c.key, c.w, c.S, c.n_in,
                                                     ::cuda::std::equal_to<>(), s);
  if (e != cudaSuccess) return e;
  k_comb_bases<PR><<<1, 1, 0, s>>>(c);
  if (c.dim == 3) k_comb_teeth<PR, 3><<<blocks, threads, 0, s>>>(c);
  else k_comb_teeth<PR, 1><<<blocks, threads, 0, s>>>(c);
  return cudaGetLastError();
}

cudaError_t comb_bank(const TrackKey &key, cudaStream_t s, const CombArgs &c) {
  if (key.f64) return comb_impl<PrecF64>(s, c);
  if (key.local) return comb_impl<PrecF32L>(s, c);
  return comb_impl<PrecF32>(s, c);
}

size_t bank_slot_bytes(const TrackKey &key) {
  return (size_t)slot_bytes(key.f64, key.dim, key.local);
}

}  // namespace mcdc
