// mlp.cu -- the learned importance proposal: a 3-layer perceptron
// in -> 64 -> 64 -> 1 (SiLU hidden layers) over (x, y, z, t, group one-hot)
// that predicts the log of the forward flux of every tally bin.  Weight
// windows follow the prediction (lower bound proportional to the predicted
// flux, a forward-flux importance reading), so particles are split on their
// way into regions the analog run hardly reaches and rouletted on their way
// back.
//
// Training and inference run on the fifth-generation tensor cores (tcgen05):
// BF16 weights and activations in shared memory, FP32 accumulators in
// tensor memory, FP32 master weights and Adam state.  Tiles of 128 samples:
// thread r of a 128-thread group owns sample r (tensor-memory lane r), one
// thread issues the MMAs, completion arrives on an mbarrier.
#include <cuda_bf16.h>
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/mcdc.h"
#include "launch.h"
#include "problem.h"
#include "tc.cuh"
#include <cub/device/device_scan.cuh>

namespace mcdc {
namespace {

constexpr int kH = 64;        // hidden width
constexpr int kIn = 16;       // padded input width (n_in <= 16)
constexpr int kS = 64;        // smallest minibatch

__host__ __device__ inline int64_t param_count(int n_in) {
  return (int64_t)kH * n_in + kH + (int64_t)kH * kH + kH + kH + 1;
}

struct Params {              // offsets into the flat FP32 parameter vector
  const float *W1, *b1, *W2, *b2, *W3, *b3;
};
__device__ __forceinline__ Params split(const float *p, int n_in) {
  Params q;
  q.W1 = p; q.b1 = q.W1 + kH * n_in; q.W2 = q.b1 + kH; q.b2 = q.W2 + kH * kH;
  q.W3 = q.b2 + kH; q.b3 = q.W3 + kH;
  return q;
}

// SiLU and its derivative with the fast exponential and divide: the network
// runs in BF16, far coarser than their few-ulp error
__device__ __forceinline__ float silu(float z) { return __fdividef(z, 1.0f + __expf(-z)); }
__device__ __forceinline__ float dsilu(float z) {
  const float s = __fdividef(1.0f, 1.0f + __expf(-z));
  return s * (1.0f + z * (1.0f - s));
}

}  // namespace

// ---- fifth-generation tensor cores (tcgen05): tiles of 128 samples -------
constexpr int kTM = 128;                  // samples per tile = MMA M = TMEM lanes
constexpr int kMbarTries = 1 << 22;       // bounded waits on MMA completion
// set when a wait on the tensor cores ran out (read back by the host)
__device__ int g_tc_timeout = 0;
// tries of the waits on MMA completion (mcdc_set_wait_limit); a wait that
// gives up leaves its MMA in flight, which the kernel still awaits (up to
// kMbarTries) before freeing its tensor memory
__device__ int g_tc_wait_limit = kMbarTries;

// shared memory of the tcgen05 forward pass (operands K-major, no swizzle)
struct TcFwd {
  __nv_bfloat16 W1[kH * kIn];             // B of layer 1: [out 64][in 16]
  __nv_bfloat16 W2[kH * kH];              // B of layer 2: [out 64][in 64]
  __nv_bfloat16 X[kTM * kIn];             // A of layer 1: [sample][in 16]
  __nv_bfloat16 H1[kTM * kH];             // A of layer 2: [sample][hidden]
  float b1[kH], b2[kH], W3[kH];
  uint64_t mbar;
  uint32_t tmem;
  int abort;
};

__device__ __forceinline__ void st_bf16(void *tile, uint32_t off, float v) {
  *reinterpret_cast<__nv_bfloat16 *>(reinterpret_cast<unsigned char *>(tile) + off) =
      __float2bfloat16(v);
}

// Prediction for samples [0, n) with tcgen05: per tile, Z1 = X W1^T and
// Z2 = H1 W2^T accumulate in tensor memory (columns [0, 64) and [64, 128));
// thread r of the CTA owns sample row r (its tensor-memory lane).
__global__ void __launch_bounds__(kTM) k_mlp_forward_tc(const float *__restrict__ p, int n_in,
                                                         const float *__restrict__ X, int64_t n,
                                                         float *__restrict__ out) {
  extern __shared__ __align__(128) unsigned char raw[];
  TcFwd &s = *reinterpret_cast<TcFwd *>(raw);
  const int tid = threadIdx.x, warp = tid >> 5;
  const Params q = split(p, n_in);
  for (int i = tid; i < kH * kIn; i += kTM) {
    const int r = i / kIn, c = i % kIn;
    st_bf16(s.W1, tc::kmaj(r, c, kIn), c < n_in ? q.W1[r * n_in + c] : 0.0f);
  }
  for (int i = tid; i < kH * kH; i += kTM) st_bf16(s.W2, tc::kmaj(i / kH, i % kH, kH), q.W2[i]);
  for (int i = tid; i < kH; i += kTM) { s.b1[i] = q.b1[i]; s.b2[i] = q.b2[i]; s.W3[i] = q.W3[i]; }
  const float b3 = p[param_count(n_in) - 1];
  if (warp == 0) tc::tmem_alloc(&s.tmem, 128);
  if (tid == 0) { tc::mbar_init(&s.mbar, 1); s.abort = 0; }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tm = s.tmem;
  const uint32_t lane_base = (uint32_t)(warp * 32) << 16;
  const uint32_t aX = tc::smem_u32(s.X), aW1 = tc::smem_u32(s.W1);
  const uint32_t aH1 = tc::smem_u32(s.H1), aW2 = tc::smem_u32(s.W2);
  uint32_t phase = 0;
  bool pending = false;
  for (int64_t base = (int64_t)blockIdx.x * kTM; base < n; base += (int64_t)gridDim.x * kTM) {
    const int64_t row = base + tid;
    float xr[kIn];                      // all loads first, then the stores
#pragma unroll
    for (int c = 0; c < kIn; ++c) xr[c] = (row < n && c < n_in) ? X[row * n_in + c] : 0.0f;
#pragma unroll
    for (int c = 0; c < kIn; ++c) st_bf16(s.X, tc::kmaj(tid, c, kIn), xr[c]);
    tc::fence_async_smem();
    __syncthreads();
    if (tid == 0) {
      tc::fence_after_sync();
      tc::mma(tm, tc::desc(aX, 128, 256), tc::desc(aW1, 128, 256), tc::idesc_bf16(kTM, kH), 0);
      tc::commit(&s.mbar);
    }
    pending = true;
    if (!tc::mbar_wait(&s.mbar, phase, g_tc_wait_limit)) { atomicOr(&g_tc_timeout, 1); s.abort = 1; }
    phase ^= 1u;
    __syncthreads();
    if (s.abort) break;
    pending = false;
    tc::fence_after_sync();
    float z[16];
#pragma unroll
    for (int q4 = 0; q4 < 4; ++q4) {
      tc::ld16(tm + lane_base + 16 * q4, z);
#pragma unroll
      for (int c = 0; c < 16; ++c) st_bf16(s.H1, tc::kmaj(tid, 16 * q4 + c, kH), silu(z[c] + s.b1[16 * q4 + c]));
    }
    tc::fence_before_sync();
    tc::fence_async_smem();
    __syncthreads();
    if (tid == 0) {
      tc::fence_after_sync();
#pragma unroll
      for (int kk = 0; kk < kH / 16; ++kk)
        tc::mma(tm + kH, tc::desc(aH1 + 256 * kk, 128, 1024), tc::desc(aW2 + 256 * kk, 128, 1024),
                tc::idesc_bf16(kTM, kH), kk > 0);
      tc::commit(&s.mbar);
    }
    pending = true;
    if (!tc::mbar_wait(&s.mbar, phase, g_tc_wait_limit)) { atomicOr(&g_tc_timeout, 1); s.abort = 1; }
    phase ^= 1u;
    __syncthreads();
    if (s.abort) break;
    pending = false;
    tc::fence_after_sync();
    float y = b3;
#pragma unroll
    for (int q4 = 0; q4 < 4; ++q4) {
      tc::ld16(tm + lane_base + kH + 16 * q4, z);
#pragma unroll
      for (int c = 0; c < 16; ++c) y += silu(z[c] + s.b2[16 * q4 + c]) * s.W3[16 * q4 + c];
    }
    if (row < n) out[row] = y;
    tc::fence_before_sync();
    __syncthreads();
  }
  // an MMA still in flight after a timed-out wait gets one more bounded wait
  if (pending) tc::mbar_wait(&s.mbar, phase ^ 1u, kMbarTries);
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) {
    tc::fence_after_sync();
    tc::tmem_free(tm, 128);
  }
}

// shared memory of the tcgen05 gradient kernel (no swizzle).  A CTA runs two
// independent tile pipelines (two groups of 4 warps); each has its own
// operand tiles, tensor-memory columns, mbarrier and barrier.  Every tile is
// stored sample-major ([sample][column], the K-major layout of an A operand
// whose K is the column): the forward and dH1 products read them as K-major
// A operands, the weight-gradient products (whose K is the sample) read the
// same bytes as MN-major operands, so no transposed copy is written.
constexpr int kNB = 80;    // columns of H1: hidden (64), ones (64), zero padding
constexpr int kNX = 32;    // columns of X: features (<= 16), ones (16), zero padding
constexpr int kGroups = 2;
struct TcTile {
  __nv_bfloat16 X[kTM * kNX];             // [sample][feature | 1 | 0]
  __nv_bfloat16 D[kTM * kTM];             // [sample][o | 0]: D2, then D1 (dL/dz1)
  __nv_bfloat16 H1[kTM * kNB];            // [sample][hidden | 1 | 0]
  uint64_t mbar;
  int abort;
  int pad;
};
struct TcGrad {
  TcTile t[kGroups];                      // first: every operand read of the tiles
                                          // stays inside this structure
  __nv_bfloat16 W1[kH * kIn];             // B of Z1:  [out][in]
  __nv_bfloat16 W2[kH * kH];              // B of Z2:  [out][in]
  __nv_bfloat16 W2T[kH * kH];             // B of dH1: [in][out]
  float b1[kH], b2[kH], W3[kH];
  float red[kGroups * 4][kH + 2];         // per-warp sums of gW3, gb3, loss
  float xch[kH * (kH + 18)];              // pipeline 1's weight gradients for pipeline 0
  uint32_t tmem;
  int pad[3];
};

// eight consecutive BF16 values (one 16-byte core-matrix row) in one store
__device__ __forceinline__ void st_bf16x8(void *tile, uint32_t off, const float *v) {
  uint32_t w[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const __nv_bfloat162 h = __floats2bfloat162_rn(v[2 * k], v[2 * k + 1]);
    w[k] = *reinterpret_cast<const uint32_t *>(&h);
  }
  *reinterpret_cast<uint4 *>(reinterpret_cast<unsigned char *>(tile) + off) =
      make_uint4(w[0], w[1], w[2], w[3]);
}

__device__ __forceinline__ void group_sync(int g) {
  asm volatile("bar.sync %0, %1;\n" : : "r"(1 + g), "r"(kTM) : "memory");
}

// Writes the BF16 weight operands (W1, W2, W2^T) and the FP32 biases and
// output weights of the parameter vector p into shared memory (all threads
// of the CTA); returns b3.  Loads bypass L1 (cache at L2 only): in the fused
// training kernel other CTAs rewrite p between steps.
// The loads of a thread are all issued before its shared-memory stores (the
// stores go through generic addresses, which the compiler cannot separate
// from the loads, so interleaving them would cost an L2 round trip each).
// Needs blockDim.x == kGroups * kTM.
__device__ __forceinline__ float load_weights(TcGrad &s, const float *__restrict__ p, int n_in) {
  constexpr int nt = kGroups * kTM;
  constexpr int n1 = kH * kIn / nt, n2 = kH * kH / nt;
  const int tid = threadIdx.x;
  const Params q = split(p, n_in);
  float w1[n1], w2[n2], bb[3];
#pragma unroll
  for (int j = 0; j < n1; ++j) {
    const int i = tid + j * nt, rr = i / kIn, c = i % kIn;
    w1[j] = c < n_in ? __ldcg(q.W1 + rr * n_in + c) : 0.0f;
  }
#pragma unroll
  for (int j = 0; j < n2; ++j) w2[j] = __ldcg(q.W2 + tid + j * nt);
  const int tb = tid & (kH - 1);
  bb[0] = __ldcg(q.b1 + tb);
  bb[1] = __ldcg(q.b2 + tb);
  bb[2] = __ldcg(q.W3 + tb);
  const float b3 = __ldcg(p + param_count(n_in) - 1);
#pragma unroll
  for (int j = 0; j < n1; ++j) {
    const int i = tid + j * nt;
    st_bf16(s.W1, tc::kmaj(i / kIn, i % kIn, kIn), w1[j]);
  }
#pragma unroll
  for (int j = 0; j < n2; ++j) {
    const int i = tid + j * nt, rr = i / kH, c = i % kH;
    st_bf16(s.W2, tc::kmaj(rr, c, kH), w2[j]);
    st_bf16(s.W2T, tc::kmaj(c, rr, kH), w2[j]);
  }
  if (tid < kH) { s.b1[tid] = bb[0]; s.b2[tid] = bb[1]; s.W3[tid] = bb[2]; }
  return b3;
}

// constant columns of a group's tiles: the ones of X (column 16) and H1
// (column 64) that carry the bias gradients, and the zero padding of X, H1
// and D; thread r of the group writes row r
__device__ __forceinline__ void init_tile_constants(TcTile &t, int r) {
  float z[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) z[k] = k == 0 ? 1.0f : 0.0f;
  st_bf16x8(t.X, tc::kmaj(r, 16, kNX), z);
  st_bf16x8(t.H1, tc::kmaj(r, kH, kNB), z);
  z[0] = 0.0f;
  st_bf16x8(t.X, tc::kmaj(r, 24, kNX), z);
  st_bf16x8(t.H1, tc::kmaj(r, kH + 8, kNB), z);
#pragma unroll
  for (int c = kH; c < kTM; c += 8) st_bf16x8(t.D, tc::kmaj(r, c, kTM), z);
}

// State of one tile pipeline (a group of 128 threads) across its tiles.
struct TileState {
  uint32_t phase;          // parity of the group's mbarrier
  bool pending;            // an MMA chain was committed and not yet waited for
  bool started;            // the weight-gradient accumulators hold a tile
  float loss, gb3;         // this thread's sample: loss and d loss / d b3 so far
};

// One tile of 128 samples (thread r of group g owns sample `row`, valid if
// row < n) through forward and backward: Z1 = X W1^T, Z2 = H1 W2^T,
// dH1 = D2 W2, and the weight gradients over the tile's samples,
// [dW2 | gb2] += D2^T [H1 | 1] and [dW1 | gb1] += D1^T [X | 1], accumulated
// in tensor memory across the group's tiles (ts.started); gW3 and gb3 build
// up in registers.  The weight-gradient products take D (M = output unit,
// padded to 128), H1 and X (N = input unit, with the ones column) as
// MN-major operands over K = the tile's samples.  Tensor memory (512
// columns), group g: Z1 in [128 g, 128 g + 64), Z2 and later dH1 in
// [128 g + 64, 128 g + 128), the gradient accumulators in [256 + 112 g,
// 256 + 112 g + 80) (rows o < 64 hold dW2 (cols 0-63) and gb2 (col 64)) and
// [256 + 112 g + 80, 256 + 112 g + 112) (rows i < 64 hold dW1 (cols < n_in)
// and gb1 (col 16)).  Returns false if a wait on the tensor cores gave up.
__device__ __forceinline__ bool grad_tile(TcGrad &s, TcTile &t, int g, int r, uint32_t tm,
                                          uint32_t lb, const float *__restrict__ Xs,
                                          const float *__restrict__ Ys,
                                          const float *__restrict__ Ws, int n_in, int64_t n,
                                          int64_t row, float b3, float inv_wsum, TileState &ts,
                                          float (&gw3)[kH]) {
  const uint32_t cZ1 = 128u * g, cZ2 = cZ1 + 64, cW2 = 256u + 112u * g, cW1 = cW2 + 80;
  const uint32_t aX = tc::smem_u32(t.X), aW1 = tc::smem_u32(s.W1), aH1 = tc::smem_u32(t.H1);
  const uint32_t aW2 = tc::smem_u32(s.W2), aW2T = tc::smem_u32(s.W2T), aD = tc::smem_u32(t.D);
  // byte strides of the sample-major tiles: 8-sample groups (the K groups of
  // the MN-major reads) and 8-column groups
  constexpr uint32_t sX = kNX / 8 * 128, sH = kNB / 8 * 128, sD = kTM / 8 * 128;
  auto wait_mma = [&]() {
    ts.pending = true;
    if (!tc::mbar_wait(&t.mbar, ts.phase, g_tc_wait_limit)) { atomicOr(&g_tc_timeout, 1); t.abort = 1; }
    ts.phase ^= 1u;
    group_sync(g);
    if (!t.abort) ts.pending = false;
    tc::fence_after_sync();
    return !t.abort;
  };
  const bool valid = row < n;
  const float yv = valid ? Ys[row] : 0.0f, wv = valid ? Ws[row] : 0.0f;
  {
    float xr[kIn];                    // all loads first, then the stores
#pragma unroll
    for (int c = 0; c < kIn; ++c) xr[c] = (valid && c < n_in) ? Xs[row * n_in + c] : 0.0f;
    st_bf16x8(t.X, tc::kmaj(r, 0, kNX), xr);
    st_bf16x8(t.X, tc::kmaj(r, 8, kNX), xr + 8);
  }
  tc::fence_async_smem();
  group_sync(g);
  if (r == 0) {
    tc::fence_after_sync();
    tc::mma(tm + cZ1, tc::desc(aX, 128, sX), tc::desc(aW1, 128, 256), tc::idesc_bf16(kTM, kH), 0);
    tc::commit(&t.mbar);
  }
  if (!wait_mma()) return false;
  // layer 1: H1
  float v[16], u[16];
#pragma unroll 1
  for (int q4 = 0; q4 < 4; ++q4) {
    tc::ld16(tm + lb + cZ1 + 16 * q4, v);
#pragma unroll
    for (int c = 0; c < 16; ++c) u[c] = silu(v[c] + s.b1[16 * q4 + c]);
    st_bf16x8(t.H1, tc::kmaj(r, 16 * q4, kNB), u);
    st_bf16x8(t.H1, tc::kmaj(r, 16 * q4 + 8, kNB), u + 8);
  }
  tc::fence_before_sync();
  tc::fence_async_smem();
  group_sync(g);
  if (r == 0) {
    tc::fence_after_sync();
#pragma unroll
    for (int kk = 0; kk < kH / 16; ++kk)
      tc::mma(tm + cZ2, tc::desc(aH1 + 256 * kk, 128, sH), tc::desc(aW2 + 256 * kk, 128, 1024),
              tc::idesc_bf16(kTM, kH), kk > 0);
    tc::commit(&t.mbar);
  }
  if (!wait_mma()) return false;
  // layer 2 and the output: f, the loss, dL/df; then dL/dz2 and gW3
  float f = b3;
#pragma unroll 1
  for (int q4 = 0; q4 < 4; ++q4) {
    tc::ld16(tm + lb + cZ2 + 16 * q4, v);
#pragma unroll
    for (int c = 0; c < 16; ++c) f += silu(v[c] + s.b2[16 * q4 + c]) * s.W3[16 * q4 + c];
  }
  const float e = f - yv;
  const float dy = 2.0f * wv * e * inv_wsum;
  ts.loss += wv * e * e * inv_wsum;
  ts.gb3 += dy;
#pragma unroll
  for (int q4 = 0; q4 < 4; ++q4) {
    tc::ld16(tm + lb + cZ2 + 16 * q4, v);
#pragma unroll
    for (int c = 0; c < 16; ++c) {
      const int o = 16 * q4 + c;
      const float z2 = v[c] + s.b2[o];
      gw3[o] += dy * silu(z2);
      u[c] = dy * s.W3[o] * dsilu(z2);
    }
    st_bf16x8(t.D, tc::kmaj(r, 16 * q4, kTM), u);
    st_bf16x8(t.D, tc::kmaj(r, 16 * q4 + 8, kTM), u + 8);
  }
  tc::fence_before_sync();
  tc::fence_async_smem();
  group_sync(g);
  if (r == 0) {
    tc::fence_after_sync();
#pragma unroll
    for (int kk = 0; kk < kH / 16; ++kk)           // dH1 = D2 W2 (over Z2's columns)
      tc::mma(tm + cZ2, tc::desc(aD + 256 * kk, 128, sD), tc::desc(aW2T + 256 * kk, 128, 1024),
              tc::idesc_bf16(kTM, kH), kk > 0);
#pragma unroll
    for (int kk = 0; kk < kTM / 16; ++kk)          // [dW2 | gb2] += D2^T [H1 | 1]
      tc::mma(tm + cW2, tc::desc(aD + 2 * sD * kk, sD, 128), tc::desc(aH1 + 2 * sH * kk, sH, 128),
              tc::idesc_bf16(kTM, kNB) | tc::kMnMajorA | tc::kMnMajorB,
              (ts.started || kk > 0) ? 1u : 0u);
    tc::commit(&t.mbar);
  }
  if (!wait_mma()) return false;
  // dL/dz1 = dH1 * silu'(z1) -> D (D2 is no longer read)
#pragma unroll 1
  for (int q4 = 0; q4 < 4; ++q4) {
    tc::ld16(tm + lb + cZ2 + 16 * q4, v);
    tc::ld16(tm + lb + cZ1 + 16 * q4, u);
#pragma unroll
    for (int c = 0; c < 16; ++c) v[c] *= dsilu(u[c] + s.b1[16 * q4 + c]);
    st_bf16x8(t.D, tc::kmaj(r, 16 * q4, kTM), v);
    st_bf16x8(t.D, tc::kmaj(r, 16 * q4 + 8, kTM), v + 8);
  }
  tc::fence_before_sync();
  tc::fence_async_smem();
  group_sync(g);
  if (r == 0) {
    tc::fence_after_sync();
#pragma unroll
    for (int kk = 0; kk < kTM / 16; ++kk)          // [dW1 | gb1] += D1^T [X | 1]
      tc::mma(tm + cW1, tc::desc(aD + 2 * sD * kk, sD, 128), tc::desc(aX + 2 * sX * kk, sX, 128),
              tc::idesc_bf16(kTM, kNX) | tc::kMnMajorA | tc::kMnMajorB,
              (ts.started || kk > 0) ? 1u : 0u);
    tc::commit(&t.mbar);
  }
  ts.started = true;
  return wait_mma();
}

// gW3, gb3 and the loss of the CTA's tiles: warp sums of the per-thread
// values into s.red (the caller synchronises before reading it).  gW3 goes
// through a butterfly reduce-scatter: at each of the five levels every lane
// keeps half of its values and adds the partner's copy of that half, so 62
// shuffles leave lane l with the warp sums of outputs 2 l and 2 l + 1.
__device__ __forceinline__ void reduce_output_grads(TcGrad &s, const TileState &ts,
                                                    float (&gw3)[kH]) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
  for (int d = 16, half = 32; d >= 1; d >>= 1, half >>= 1) {
    const bool upper = (lane & d) != 0;
#pragma unroll
    for (int j = 0; j < half; ++j) {
      const float send = upper ? gw3[j] : gw3[j + half];
      const float keep = upper ? gw3[j + half] : gw3[j];
      gw3[j] = keep + __shfl_xor_sync(0xffffffffu, send, d);
    }
  }
  s.red[warp][2 * lane] = gw3[0];
  s.red[warp][2 * lane + 1] = gw3[1];
  float gb3 = ts.gb3, loss = ts.loss;
  for (int d = 16; d > 0; d >>= 1) {
    gb3 += __shfl_xor_sync(0xffffffffu, gb3, d);
    loss += __shfl_xor_sync(0xffffffffu, loss, d);
  }
  if (lane == 0) { s.red[warp][kH] = gb3; s.red[warp][kH + 1] = loss; }
}

// Loss sum_i w_i (f(x_i) - y_i)^2 / wsum over samples [0, n) and its gradient
// (added into grad, zeroed by the caller) with tcgen05, 128 samples per tile and
// two tile pipelines per CTA (grad_tile); the accumulators are added into
// grad with atomics at the end.
__global__ void __launch_bounds__(kGroups * kTM) k_mlp_grad_tc(
    const float *__restrict__ p, int n_in, const float *__restrict__ X,
    const float *__restrict__ Y, const float *__restrict__ Wt, int64_t n, int64_t first,
    float inv_wsum, float *__restrict__ grad, double *__restrict__ loss) {
  extern __shared__ __align__(128) unsigned char raw[];
  TcGrad &s = *reinterpret_cast<TcGrad *>(raw);
  const int tid = threadIdx.x, warp = tid >> 5;
  const int g = tid / kTM, r = tid % kTM;         // group and sample row
  TcTile &t = s.t[g];
  const float b3 = load_weights(s, p, n_in);
  init_tile_constants(t, r);
  if (warp == 0) tc::tmem_alloc(&s.tmem, 512);
  if (r == 0) { tc::mbar_init(&t.mbar, 1); t.abort = 0; }
  tc::fence_async_smem();
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tm = s.tmem;
  const uint32_t lb = (uint32_t)((warp & 3) * 32) << 16;   // this warp's lanes
  const uint32_t cW2 = 256u + 112u * g, cW1 = cW2 + 80;
  TileState ts{0u, false, false, 0.0f, 0.0f};
  float gw3[kH];
#pragma unroll
  for (int o = 0; o < kH; ++o) gw3[o] = 0.0f;
  for (int64_t base = ((int64_t)blockIdx.x * kGroups + g) * kTM; base < n;
       base += (int64_t)gridDim.x * kGroups * kTM)
    if (!grad_tile(s, t, g, r, tm, lb, X + first * n_in, Y + first, Wt + first, n_in, n,
                   base + r, b3, inv_wsum, ts, gw3))
      break;
  if (ts.pending) tc::mbar_wait(&t.mbar, ts.phase ^ 1u, kMbarTries);
  reduce_output_grads(s, ts, gw3);
  __syncthreads();
  const bool ok = !s.t[0].abort && !s.t[1].abort;
  float *gW1 = grad, *gb1 = gW1 + kH * n_in, *gW2 = gb1 + kH, *gb2 = gW2 + kH * kH;
  float *gW3 = gb2 + kH, *gb3 = gW3 + kH;
  if (ok && tid < kH + 2) {
    float a = 0.0f;
    for (int w = 0; w < kGroups * 4; ++w) a += s.red[w][tid];
    if (tid < kH) atomicAdd(&gW3[tid], a);
    else if (tid == kH) atomicAdd(gb3, a);
    else atomicAdd(loss, (double)a);
  }
  if (ok && ts.started && (warp & 3) < 2) {
    // this group's accumulators: lanes 0-63 are warps 0, 1 of the group
    tc::fence_after_sync();
    const int o = r;                                  // 0..63
    float v[16];
#pragma unroll
    for (int q4 = 0; q4 < 5; ++q4) {                  // columns 0-79 of DT BH
      tc::ld16(tm + lb + cW2 + 16 * q4, v);
#pragma unroll
      for (int c = 0; c < 16; ++c) {
        const int col = 16 * q4 + c;
        if (col < kH) atomicAdd(&gW2[o * kH + col], v[c]);
        else if (col == kH) atomicAdd(&gb2[o], v[c]);
      }
    }
    tc::ld16(tm + lb + cW1, v);
#pragma unroll
    for (int c = 0; c < 16; ++c)
      if (c < n_in) atomicAdd(&gW1[o * n_in + c], v[c]);
    tc::ld16(tm + lb + cW1 + 16, v);
    atomicAdd(&gb1[o], v[0]);
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) {
    tc::fence_after_sync();
    tc::tmem_free(tm, 512);
  }
}

// ---- a whole fit in one launch ----------------------------------------------

// Arguments of k_mlp_train_tc.
struct TrainArgs {
  const float *X, *Y, *W;        // compacted samples [n][n_in], targets, weights
  int64_t n_samples;             // minibatch b: samples [b batch, min(n, (b + 1) batch))
  int batch;
  const float *inv_wsum;         // [n_steps] 1 / its weight sum
  int n_in, n_steps, epochs;
  int np, np_pad;                // parameters; row length of part (multiple of 4)
  float *p, *m, *v;              // FP32 master weights, Adam moments
  float *part;                   // [gridDim.x][np_pad] per-CTA gradients of a step
  double *losses;                // [2 n_steps]: loss per minibatch, first and last epoch
  unsigned long long *bar;       // grid-barrier arrivals (zero at launch)
  int *err;                      // set when a wait gives up; every CTA then leaves
  float lr, lr_end;               // step size: lr at the first step, cosine down to lr_end
                                 // at the last (lr_end = lr: constant)
};

__device__ __forceinline__ unsigned long long ld_acquire_u64(const unsigned long long *p) {
  unsigned long long v;
  asm volatile("ld.acquire.gpu.global.u64 %0, [%1];\n" : "=l"(v) : "l"(p) : "memory");
  return v;
}

// Barrier over the CTAs of a cooperative launch (all co-resident): every CTA
// adds one arrival, then waits until `target` arrivals (the k-th barrier of
// the launch waits for k x gridDim.x).  Bounded: a CTA gives up after `limit`
// polls (setting *err), and leaves at once once another CTA has given up.
// Returns false in both cases.
__device__ bool grid_barrier(unsigned long long *bar, int *err, unsigned long long target,
                             int limit) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    // release: the CTA's writes (ordered before this thread by the barrier
    // above) become visible before the arrival; acquire on the polls
    asm volatile("red.release.gpu.global.add.u64 [%0], %1;\n" : : "l"(bar), "l"(1ull) : "memory");
    int ok = 0;
    for (int i = 0; i < limit; ++i) {
      if (ld_acquire_u64(bar) >= target) { ok = 1; break; }
      if (*reinterpret_cast<volatile int *>(err)) break;
      if (i > 64) __nanosleep(32);
    }
    if (!ok) { atomicOr(err, 1); atomicOr(&g_tc_timeout, 1); }
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

// The whole training of a fit in one persistent cooperative launch: for every
// minibatch of every epoch, (1) every CTA converts the FP32 master weights to
// its BF16 operands, (2) each of its two tile pipelines runs its tiles of the
// minibatch (tile j of the step goes to pipeline j mod (2 x gridDim.x)) with
// the weight gradients accumulating in tensor memory, (3) the CTA writes its
// gradient to its row of `part` with plain stores, (4) grid barrier, (5) CTA c
// sums the rows of its slice of the parameters in CTA order and applies Adam
// to it, (6) grid barrier.  The sums have a fixed order, so a fit is
// reproducible bit for bit.  The algorithm is the one of the per-minibatch
// kernel (k_mlp_grad_tc) and Adam (Kingma & Ba) on FP32 master weights;
// only the per-minibatch launches and the gradient atomics are gone.
__global__ void __launch_bounds__(kGroups * kTM) k_mlp_train_tc(const TrainArgs A) {
  extern __shared__ __align__(128) unsigned char raw[];
  TcGrad &s = *reinterpret_cast<TcGrad *>(raw);
  __shared__ float s_acc[kGroups * kTM];
  const int tid = threadIdx.x, warp = tid >> 5;
  const int g = tid / kTM, r = tid % kTM;
  const int G = gridDim.x, n_in = A.n_in;
  TcTile &t = s.t[g];
  init_tile_constants(t, r);
  if (warp == 0) tc::tmem_alloc(&s.tmem, 512);
  if (r == 0) { tc::mbar_init(&t.mbar, 1); t.abort = 0; }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tm = s.tmem;
  const uint32_t lb = (uint32_t)((warp & 3) * 32) << 16;
  const uint32_t cW2 = 256u + 112u * g, cW1 = cW2 + 80;
  // parameter offsets (flat layout W1, b1, W2, b2, W3, b3)
  const int oW1 = 0, ob1 = kH * n_in, oW2 = ob1 + kH, ob2 = oW2 + kH * kH, oW3 = ob2 + kH,
            ob3 = oW3 + kH;
  // this CTA's slice of the parameters for the reduction and Adam
  const int PS = (A.np + G - 1) / G;
  const int slice0 = blockIdx.x * PS, nslice = max(0, min(PS, A.np - slice0));
  float *my_part = A.part + (size_t)blockIdx.x * A.np_pad;
  TileState ts{0u, false, false, 0.0f, 0.0f};
  const int total = A.epochs * A.n_steps;
  unsigned long long arrivals = 0;
  for (int k = 0; k < total; ++k) {
    const int b = k % A.n_steps, ep = k / A.n_steps;
    // (1) operands from the master weights (the previous step's Adam)
    const float b3 = load_weights(s, A.p, n_in);
    tc::fence_async_smem();
    __syncthreads();
    // (2) this pipeline's tiles of minibatch b
    ts.started = false;
    ts.loss = 0.0f;
    ts.gb3 = 0.0f;
    float gw3[kH];
#pragma unroll
    for (int o = 0; o < kH; ++o) gw3[o] = 0.0f;
    const int64_t f0 = (int64_t)b * A.batch, cnt = min((int64_t)A.batch, A.n_samples - f0);
    const float inv = A.inv_wsum[b];
    for (int64_t base = ((int64_t)blockIdx.x * kGroups + g) * kTM; base < cnt;
         base += (int64_t)G * kGroups * kTM)
      if (!grad_tile(s, t, g, r, tm, lb, A.X + f0 * n_in, A.Y + f0, A.W + f0, n_in, cnt,
                     base + r, b3, inv, ts, gw3))
        break;
    // (3) the CTA's gradient: gW3, gb3 (and the loss) from registers, the
    // rest from both pipelines' tensor-memory accumulators; pipeline 1 hands
    // its part to pipeline 0 through shared memory
    reduce_output_grads(s, ts, gw3);
    __syncthreads();
    if (s.t[0].abort || s.t[1].abort) {
      if (tid == 0) atomicOr(A.err, 1);
      break;
    }
    if (tid <= kH) {
      float a = 0.0f;
      for (int w = 0; w < kGroups * 4; ++w) a += s.red[w][tid];
      my_part[tid < kH ? oW3 + tid : ob3] = a;
    } else if (tid == kH + 1 && (ep == 0 || ep == A.epochs - 1)) {
      float a = 0.0f;
      for (int w = 0; w < kGroups * 4; ++w) a += s.red[w][kH + 1];
      atomicAdd(&A.losses[(ep == 0 ? 0 : A.n_steps) + b], (double)a);
    }
    // row o of a pipeline's accumulators: dW2[o][0..63], gb2[o] (column 64),
    // dW1[o][0..15], gb1[o] (column 16 of the second block) -> 82 values
    constexpr int kX = kH + 18;
    float *xo = s.xch + (size_t)r * kX;
    if ((warp & 3) < 2) {
      float v[16];
      tc::fence_after_sync();
      if (g == 1) {
#pragma unroll
        for (int q4 = 0; q4 < 5; ++q4) {
          if (ts.started) tc::ld16(tm + lb + cW2 + 16 * q4, v);
#pragma unroll
          for (int c = 0; c < 16; ++c)
            if (16 * q4 + c <= kH) xo[16 * q4 + c] = ts.started ? v[c] : 0.0f;
        }
        if (ts.started) tc::ld16(tm + lb + cW1, v);
#pragma unroll
        for (int c = 0; c < 16; ++c) xo[kH + 1 + c] = ts.started ? v[c] : 0.0f;
        if (ts.started) tc::ld16(tm + lb + cW1 + 16, v);
        xo[kH + 17] = ts.started ? v[0] : 0.0f;
      }
    }
    tc::fence_before_sync();
    __syncthreads();
    if (g == 0 && (warp & 3) < 2) {
      float v[16];
      tc::fence_after_sync();
      const int o = r;
#pragma unroll
      for (int q4 = 0; q4 < 4; ++q4) {              // dW2 row o: four float4 per block
        if (ts.started) tc::ld16(tm + lb + cW2 + 16 * q4, v);
        float4 *dst = reinterpret_cast<float4 *>(my_part + oW2 + o * kH + 16 * q4);
#pragma unroll
        for (int c = 0; c < 16; c += 4)
          dst[c / 4] = make_float4((ts.started ? v[c] : 0.0f) + xo[16 * q4 + c],
                                   (ts.started ? v[c + 1] : 0.0f) + xo[16 * q4 + c + 1],
                                   (ts.started ? v[c + 2] : 0.0f) + xo[16 * q4 + c + 2],
                                   (ts.started ? v[c + 3] : 0.0f) + xo[16 * q4 + c + 3]);
      }
      if (ts.started) tc::ld16(tm + lb + cW2 + 64, v);
      my_part[ob2 + o] = (ts.started ? v[0] : 0.0f) + xo[kH];
      if (ts.started) tc::ld16(tm + lb + cW1, v);
#pragma unroll
      for (int c = 0; c < 16; ++c)
        if (c < n_in) my_part[oW1 + o * n_in + c] = (ts.started ? v[c] : 0.0f) + xo[kH + 1 + c];
      if (ts.started) tc::ld16(tm + lb + cW1 + 16, v);
      my_part[ob1 + o] = (ts.started ? v[0] : 0.0f) + xo[kH + 17];
    }
    tc::fence_before_sync();
    // (4) every CTA's gradient is in part
    arrivals += (unsigned long long)G;
    if (!grid_barrier(A.bar, A.err, arrivals, g_tc_wait_limit)) break;
    tc::fence_after_sync();
    // (5) sum over CTAs (fixed order) and Adam on this CTA's slice
    {
      const float b1 = 0.9f, b2 = 0.999f;
      const float c1 = 1.f - powf(b1, (float)(k + 1)), c2 = 1.f - powf(b2, (float)(k + 1));
      const int k_last = A.epochs * A.n_steps - 1;
      const float lr = A.lr_end + 0.5f * (A.lr - A.lr_end) *
                                      (1.0f + cospif(k_last > 0 ? (float)k / (float)k_last : 0.0f));
      const int nt = kGroups * kTM;
      for (int c0 = 0; c0 < nslice; c0 += nt) {
        const int nc = min(nt, nslice - c0);
        const int R = max(1, nt / nc);             // threads per parameter
        float acc = 0.0f;
        if (tid < nc * R) {
          // this thread's CTAs rr, rr + R, ... in order, up to 24 loads in flight
          const int pl = tid / R, rr = tid % R;
          const float *col = A.part + slice0 + c0 + pl;
          for (int src = rr; src < G; src += 24 * R) {
            float buf[24];
#pragma unroll
            for (int j = 0; j < 24; ++j)
              buf[j] = src + j * R < G ? __ldcg(col + (size_t)(src + j * R) * A.np_pad) : 0.0f;
#pragma unroll
            for (int j = 0; j < 24; ++j) acc += buf[j];
          }
        }
        s_acc[tid] = acc;
        __syncthreads();
        if (tid < nc) {
          float gi = 0.0f;
          for (int rr = 0; rr < R; ++rr) gi += s_acc[tid * R + rr];
          const int i = slice0 + c0 + tid;
          const float mi = b1 * A.m[i] + (1.f - b1) * gi;
          const float vi = b2 * A.v[i] + (1.f - b2) * gi * gi;
          A.m[i] = mi;
          A.v[i] = vi;
          A.p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + 1e-8f);
        }
        __syncthreads();
      }
    }
    // (6) every slice is updated
    arrivals += (unsigned long long)G;
    if (!grid_barrier(A.bar, A.err, arrivals, g_tc_wait_limit)) break;
  }
  if (ts.pending) tc::mbar_wait(&t.mbar, ts.phase ^ 1u, kMbarTries);
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) {
    tc::fence_after_sync();
    tc::tmem_free(tm, 512);
  }
}

// ---- host side -------------------------------------------------------------

size_t mlp_smem_bytes() { return sizeof(TcGrad); }

cudaError_t mlp_prepare() {
  cudaError_t e = cudaFuncSetAttribute(k_mlp_grad_tc, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)sizeof(TcGrad));
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(k_mlp_train_tc, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)sizeof(TcGrad));
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(k_mlp_forward_tc, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)sizeof(TcFwd));
}

cudaError_t launch_mlp_grad(cudaStream_t st, int sms, const float *p, int n_in, const float *X,
                            const float *Y, const float *W, int64_t n, int64_t first,
                            float inv_wsum, float *grad, double *loss) {
  const int64_t tiles = (n + kTM - 1) / kTM;
  const int grid = (int)std::max<int64_t>(1, std::min<int64_t>((tiles + kGroups - 1) / kGroups, (int64_t)sms));
  k_mlp_grad_tc<<<grid, kGroups * kTM, sizeof(TcGrad), st>>>(p, n_in, X, Y, W, n, first, inv_wsum, grad, loss);
  return cudaGetLastError();
}

cudaError_t launch_mlp_forward(cudaStream_t st, int sms, const float *p, int n_in, const float *X,
                               int64_t n, float *out) {
  const int64_t tiles = (n + kTM - 1) / kTM;
  const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(tiles, (int64_t)sms * 2));
  k_mlp_forward_tc<<<grid, kTM, sizeof(TcFwd), st>>>(p, n_in, X, n, out);
  return cudaGetLastError();
}

int64_t mlp_param_count(int n_in) { return param_count(n_in); }

// ---- training data from a pilot tally --------------------------------------

// Sample s holds tally bin perm(s) = (s * stride) mod n_bins (stride coprime
// with n_bins), so consecutive minibatches mix the whole mesh.  Features:
// cell centre and bin-centre time scaled to [-1, 1], then the group one-hot.
// Target: log of the pilot mean; weight 1 / (1 + relerr^2), 0 where the pilot
// never scored.
__global__ void k_make_samples(const DevProblem P, int n_in, uint64_t stride,
                               const double *__restrict__ mean, const double *__restrict__ rel,
                               float *__restrict__ X, float *__restrict__ Y,
                               float *__restrict__ W, double *__restrict__ moments) {
  double sw = 0.0, swt = 0.0, swt2 = 0.0;
  const int64_t nb = P.n_bins;
  for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < nb;
       s += (int64_t)gridDim.x * blockDim.x) {
    const int64_t b = (int64_t)(((unsigned __int128)s * stride) % (unsigned __int128)nb);
    const int tb = (int)(b % P.T1);
    const int g = (int)((b / P.T1) % P.G);
    const int64_t cell = b / ((int64_t)P.T1 * P.G);
    const int ci = (int)(cell % P.n[0]);
    const int cj = (int)((cell / P.n[0]) % P.n[1]);
    const int ck = (int)(cell / ((int64_t)P.n[0] * P.n[1]));
    float *x = X + s * n_in;
    const int idx[3] = {ci, cj, ck};
    for (int a = 0; a < 3; ++a)
      x[a] = P.bounded[a] ? (float)(2.0 * (idx[a] + 0.5) / P.n[a] - 1.0) : 0.0f;
    x[3] = P.T > 0 ? (float)(2.0 * (tb + 0.5) / P.T - 1.0) : 0.0f;
    for (int k = 4; k < n_in; ++k) x[k] = (k - 4 == g) ? 1.0f : 0.0f;
    const double m = mean ? mean[b] : 0.0;
    if (m > 0.0) {
      const double r = rel ? rel[b] : 0.0;
      const double w = 1.0 / (1.0 + r * r);
      const double t = log(m);
      Y[s] = (float)t;
      W[s] = (float)w;
      sw += w; swt += w * t; swt2 += w * t * t;
    } else {
      Y[s] = 0.0f;
      W[s] = 0.0f;
    }
  }
  for (int o = 16; o > 0; o >>= 1) {
    sw += __shfl_xor_sync(0xffffffffu, sw, o);
    swt += __shfl_xor_sync(0xffffffffu, swt, o);
    swt2 += __shfl_xor_sync(0xffffffffu, swt2, o);
  }
  if ((threadIdx.x & 31) == 0) {
    atomicAdd(&moments[0], sw);
    atomicAdd(&moments[1], swt);
    atomicAdd(&moments[2], swt2);
  }
}

// targets to zero mean and unit variance (weighted); moments[3..4] keep the
// shift and scale for the bake
__global__ void k_normalize_targets(int64_t n, float *__restrict__ Y, const float *__restrict__ W,
                                    double *__restrict__ moments) {
  const double sw = moments[0] > 0.0 ? moments[0] : 1.0;
  const double mu = moments[1] / sw;
  const double var = moments[2] / sw - mu * mu;
  const double sd = var > 1e-12 ? sqrt(var) : 1.0;
  if (blockIdx.x == 0 && threadIdx.x == 0) { moments[3] = mu; moments[4] = sd; }
  for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < n;
       s += (int64_t)gridDim.x * blockDim.x)
    if (W[s] > 0.0f) Y[s] = (float)((Y[s] - mu) / sd);
}

// Samples of the spatial distillation: one per cell, the position inputs of
// its centre (as k_make_samples) and the log of its window in a table that
// depends on the cell alone (time and group folded); unit weights
__global__ void k_distill_samples(const DevProblem P, const double *__restrict__ ww64,
                                  float *__restrict__ X, float *__restrict__ Y,
                                  float *__restrict__ W, double *__restrict__ moments) {
  double sw = 0.0, swt = 0.0, swt2 = 0.0;
  const int64_t nc = P.n_cells, per_cell = (int64_t)P.G * P.T1;
  for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < nc;
       c += (int64_t)gridDim.x * blockDim.x) {
    const int idx[3] = {(int)(c % P.n[0]), (int)((c / P.n[0]) % P.n[1]),
                        (int)(c / ((int64_t)P.n[0] * P.n[1]))};
    for (int a = 0; a < 3; ++a)
      X[c * 3 + a] = P.bounded[a] ? (float)(2.0 * (idx[a] + 0.5) / P.n[a] - 1.0) : 0.0f;
    const double t = log(ww64[c * per_cell]);
    Y[c] = (float)t;
    W[c] = 1.0f;
    sw += 1.0; swt += t; swt2 += t * t;
  }
  for (int o = 16; o > 0; o >>= 1) {
    sw += __shfl_xor_sync(0xffffffffu, sw, o);
    swt += __shfl_xor_sync(0xffffffffu, swt, o);
    swt2 += __shfl_xor_sync(0xffffffffu, swt2, o);
  }
  if ((threadIdx.x & 31) == 0) {
    atomicAdd(&moments[0], sw);
    atomicAdd(&moments[1], swt);
    atomicAdd(&moments[2], swt2);
  }
}

// 1 / (sum of the weights of minibatch b), one block per minibatch (FP64 sums)
__global__ void k_minibatch_inv(int64_t n, int batch, const float *__restrict__ W,
                                float *__restrict__ inv) {
  __shared__ double part[32];
  const int64_t f0 = (int64_t)blockIdx.x * batch;
  const int64_t f1 = f0 + batch < n ? f0 + batch : n;
  double a = 0.0;
  for (int64_t i = f0 + threadIdx.x; i < f1; i += blockDim.x) a += W[i];
  for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
  if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = a;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += part[w];
    inv[blockIdx.x] = t > 0.0 ? (float)(1.0 / t) : 0.0f;
  }
}

// the scored samples only (weight > 0), in their order: flags, then a gather
// at the exclusive prefix sum of the flags
__global__ void k_sample_flags(int64_t n, const float *__restrict__ W, int32_t *__restrict__ flag) {
  for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < n;
       s += (int64_t)gridDim.x * blockDim.x)
    flag[s] = W[s] > 0.0f ? 1 : 0;
}
__global__ void k_sample_gather(int64_t n, int n_in, const float *__restrict__ X,
                                const float *__restrict__ Y, const float *__restrict__ W,
                                const int32_t *__restrict__ flag, const int32_t *__restrict__ pos,
                                float *__restrict__ Xc, float *__restrict__ Yc,
                                float *__restrict__ Wc) {
  for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < n;
       s += (int64_t)gridDim.x * blockDim.x) {
    if (!flag[s]) continue;
    const int64_t d = pos[s];
    for (int k = 0; k < n_in; ++k) Xc[d * n_in + k] = X[s * n_in + k];
    Yc[d] = Y[s];
    Wc[d] = W[s];
  }
}

// largest prediction (denormalised log flux) over bins, as ordered bits of a
// non-negative offset: predictions are shifted by +1e4 so they stay positive
__global__ void k_pred_max(int64_t n, const float *__restrict__ pred,
                           const double *__restrict__ moments, unsigned long long *__restrict__ mx) {
  double best = -1e300;
  for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < n;
       s += (int64_t)gridDim.x * blockDim.x)
    best = fmax(best, (double)pred[s] * moments[4] + moments[3]);
  for (int o = 16; o > 0; o >>= 1) best = fmax(best, __shfl_xor_sync(0xffffffffu, best, o));
  if ((threadIdx.x & 31) == 0 && best > -1e300) {
    const double shifted = fmax(0.0, best + 1e4);
    atomicMax(mx, (unsigned long long)__double_as_longlong(shifted));
  }
}

// smallest prediction over the bins the pilot scored (same ordered-bits trick)
__global__ void k_pred_min_scored(int64_t n, const float *__restrict__ pred,
                                  const float *__restrict__ W, const double *__restrict__ moments,
                                  unsigned long long *__restrict__ mn) {
  double best = 1e300;
  for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < n;
       s += (int64_t)gridDim.x * blockDim.x)
    if (W[s] > 0.0f) best = fmin(best, (double)pred[s] * moments[4] + moments[3]);
  for (int o = 16; o > 0; o >>= 1) best = fmin(best, __shfl_xor_sync(0xffffffffu, best, o));
  if ((threadIdx.x & 31) == 0 && best < 1e300) {
    const double shifted = fmax(0.0, best + 1e4);
    atomicMin(mn, (unsigned long long)__double_as_longlong(shifted));
  }
}

// weight-window lower bounds: w_L = wl0 * exp(log phi - max log phi), but no
// lower than a tenth of the least-scored bin's value and no lower than
// min_ratio: where the pilot never scored, the network extrapolates, and a
// window far below the true flux would split every arriving particle again
// and again
__global__ void k_ww_from_pred(const DevProblem P, uint64_t stride, const float *__restrict__ pred,
                               const double *__restrict__ moments,
                               const unsigned long long *__restrict__ mx,
                               const unsigned long long *__restrict__ mn, double wl0,
                               double min_ratio, double *__restrict__ ww64,
                               float *__restrict__ ww32) {
  const double top = __longlong_as_double((long long)*mx) - 1e4;
  const double low = __longlong_as_double((long long)*mn) - 1e4;
  const double floor_lp = fmax(low - 2.302585092994046, top + log(min_ratio));
  const int64_t nb = P.n_bins;
  for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < nb;
       s += (int64_t)gridDim.x * blockDim.x) {
    const int64_t b = (int64_t)(((unsigned __int128)s * stride) % (unsigned __int128)nb);
    const double lp = fmax((double)pred[s] * moments[4] + moments[3], floor_lp);
    const double w = wl0 * exp(fmin(0.0, lp - top));
    ww64[b] = w;
    ww32[b] = (float)w;
  }
}

// largest predicted log importance over the bins of the cells the source box
// touches (ordered-bits trick as above)
__global__ void k_pred_src_max(const DevProblem P, uint64_t stride, const float *__restrict__ pred,
                               const double *__restrict__ moments,
                               unsigned long long *__restrict__ mx) {
  int lo[3], hi[3];
  for (int a = 0; a < 3; ++a) {
    if (!P.bounded[a]) { lo[a] = hi[a] = 0; continue; }
    lo[a] = max(0, min(P.n[a] - 1, (int)floor((P.src_lo[a] - P.origin[a]) / P.width[a])));
    hi[a] = max(0, min(P.n[a] - 1, (int)floor((P.src_hi[a] - P.origin[a]) / P.width[a])));
  }
  const int64_t nb = P.n_bins, per_cell = (int64_t)P.G * P.T1;
  double best = -1e300;
  for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < nb;
       s += (int64_t)gridDim.x * blockDim.x) {
    const int64_t b = (int64_t)(((unsigned __int128)s * stride) % (unsigned __int128)nb);
    const int64_t cell = b / per_cell;
    const int i = (int)(cell % P.n[0]), j = (int)((cell / P.n[0]) % P.n[1]);
    const int k = (int)(cell / ((int64_t)P.n[0] * P.n[1]));
    if (i >= lo[0] && i <= hi[0] && j >= lo[1] && j <= hi[1] && k >= lo[2] && k <= hi[2])
      best = fmax(best, (double)pred[s] * moments[4] + moments[3]);
  }
  for (int o = 16; o > 0; o >>= 1) best = fmax(best, __shfl_xor_sync(0xffffffffu, best, o));
  if ((threadIdx.x & 31) == 0 && best > -1e300)
    atomicMax(mx, (unsigned long long)__double_as_longlong(fmax(0.0, best + 1e4)));
}

// importance (adjoint) windows: w_L = wl0 * I(source) / I, with I kept above
// a tenth of the least-scored bin's value and above min_ratio * max I, and
// w_L never below wl0 * I(source) / max I
__global__ void k_ww_from_importance(const DevProblem P, uint64_t stride,
                                     const float *__restrict__ pred,
                                     const double *__restrict__ moments,
                                     const unsigned long long *__restrict__ mx, double wl0,
                                     double min_ratio, double *__restrict__ ww64,
                                     float *__restrict__ ww32) {
  const double top = __longlong_as_double((long long)mx[0]) - 1e4;
  const double low = __longlong_as_double((long long)mx[1]) - 1e4;
  const double src = __longlong_as_double((long long)mx[2]) - 1e4;
  const double floor_lp = fmax(low - 2.302585092994046, top + log(min_ratio));
  const int64_t nb = P.n_bins;
  for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < nb;
       s += (int64_t)gridDim.x * blockDim.x) {
    const int64_t b = (int64_t)(((unsigned __int128)s * stride) % (unsigned __int128)nb);
    const double lp = fmin(fmax((double)pred[s] * moments[4] + moments[3], floor_lp), top);
    const double w = wl0 * exp(fmin(src - lp, 700.0));
    ww64[b] = w;
    ww32[b] = (float)fmin(w, 3.0e38);
  }
}

// one window per (cell, group) -- the largest over its time bins -- or per
// cell, the largest over its groups and time bins (importance windows: the
// smallest, i.e. the largest importance)
__global__ void k_ww_collapse(const DevProblem P, bool over_groups, bool over_time, bool smallest,
                              double *__restrict__ ww64, float *__restrict__ ww32) {
  const int G = over_groups ? P.G : 1;        // groups folded into one window
  const int T = over_time ? P.T1 : 1;         // time bins folded into one window
  const int64_t n = P.n_bins / ((int64_t)G * T);
  for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < n;
       c += (int64_t)gridDim.x * blockDim.x) {
    // c enumerates (cell, kept group, kept time bin); bin = (cell G + g) T1 + t
    const int64_t cell = over_groups ? c / (over_time ? 1 : P.T1) : c / ((int64_t)P.G * (over_time ? 1 : P.T1));
    const int g0 = over_groups ? 0 : (int)((c / (over_time ? 1 : P.T1)) % P.G);
    const int t0 = over_time ? 0 : (int)(c % P.T1);
    double m = smallest ? 1e308 : 0.0;
    for (int g = 0; g < G; ++g)
      for (int t = 0; t < T; ++t) {
        const double w = ww64[(cell * P.G + g0 + g) * P.T1 + t0 + t];
        m = smallest ? fmin(m, w) : fmax(m, w);
      }
    for (int g = 0; g < G; ++g)
      for (int t = 0; t < T; ++t) {
        ww64[(cell * P.G + g0 + g) * P.T1 + t0 + t] = m;
        ww32[(cell * P.G + g0 + g) * P.T1 + t0 + t] = (float)fmin(m, 3.0e38);
      }
  }
}

namespace {
uint64_t gcd64(uint64_t a, uint64_t b) {
  while (b) { const uint64_t r = a % b; a = b; b = r; }
  return a;
}
// a stride near n * 0.618 that is coprime with n
uint64_t coprime_stride(uint64_t n) {
  if (n <= 2) return 1;
  uint64_t s = (uint64_t)((double)n * 0.6180339887498949) | 1ull;
  while (gcd64(s, n) != 1) s += 2;
  return s % n ? s % n : 1;
}
}  // namespace

}  // namespace mcdc

// ---- C-ABI -----------------------------------------------------------------
using namespace mcdc;

namespace {
int fail(int code, const std::string &m) { return mcdc::set_error(code, m); }

// MCDC_ERR_TIMEOUT if a tensor-core wait gave up since the last check
int tc_status() {
  int v = 0;
  if (cudaMemcpyFromSymbol(&v, g_tc_timeout, sizeof(int)) != cudaSuccess) {
    cudaGetLastError();
    return fail(MCDC_ERR_CUDA, "reading the tensor-core status failed");
  }
  if (v) {
    const int zero = 0;
    cudaMemcpyToSymbol(g_tc_timeout, &zero, sizeof(int));
    return fail(MCDC_ERR_TIMEOUT, "a wait on the tensor cores ran out (importance network)");
  }
  return MCDC_OK;
}

bool on_dev(const void *p) {
  if (!p) return false;
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) { cudaGetLastError(); return false; }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// device copy of a host-or-device array (owned by the caller through *keep)
template <class T>
cudaError_t as_device(const T *p, size_t count, const T **out, void **keep) {
  *keep = nullptr;
  if (on_dev(p)) { *out = p; return cudaSuccess; }
  void *d = nullptr;
  cudaError_t e = cudaMalloc(&d, std::max<size_t>(count * sizeof(T), 16));
  if (e != cudaSuccess) return e;
  e = cudaMemcpy(d, p, count * sizeof(T), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) { cudaFree(d); return e; }
  *keep = d;
  *out = (const T *)d;
  return cudaSuccess;
}

// Temporaries of one call from a stream-ordered pool (plain cudaMalloc where
// there is none), freed in the stream's order when the object goes away.
struct PoolBufs {
  cudaMemPool_t pool;
  cudaStream_t s;
  std::vector<void *> v;
  template <class T>
  cudaError_t get(T **p, size_t count) {
    void *q = nullptr;
    const size_t bytes = std::max<size_t>(count * sizeof(T), 16);
    const cudaError_t e = pool ? cudaMallocFromPoolAsync(&q, bytes, pool, s) : cudaMalloc(&q, bytes);
    if (e == cudaSuccess) { v.push_back(q); *p = (T *)q; }
    return e;
  }
  ~PoolBufs() { for (void *q : v) { if (pool) cudaFreeAsync(q, s); else cudaFree(q); } }
};

struct Frees {
  std::vector<void *> v;
  ~Frees() { for (void *p : v) if (p) cudaFree(p); }
  void *add(void *p) { v.push_back(p); return p; }
};

int device_sms() {
  int dev = 0, sms = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return sms;
}

#define CKM(call)                                                                        \
  do {                                                                                   \
    cudaError_t e_ = (call);                                                             \
    if (e_ != cudaSuccess)                                                               \
      return fail(e_ == cudaErrorMemoryAllocation ? MCDC_ERR_OOM : MCDC_ERR_CUDA,        \
                  std::string(#call) + ": " + cudaGetErrorString(e_));                   \
  } while (0)
// The whole training in one cooperative launch (k_mlp_train_tc) on stream st:
// n_steps minibatches of `batch` consecutive samples (1 / weight sums in
// d_inv), epochs passes, Adam on prm (n_in inputs; np_pad-padded), m, v;
// losses [2 n_steps] zeroed by the caller.  One CTA per SM at most, and no
// more than the two tile pipelines per CTA that cover a minibatch in one
// round.  Waits for the launch.
int train_fused(PoolBufs &tmp, cudaStream_t st, int sms, const float *Xc, const float *Yc,
                const float *Wc, int64_t n_samples, int n_in, int epochs, int batch, float lr,
                const float *d_inv, int n_steps, float *prm, float *m, float *v, double *losses,
                double *loss_first, double *loss_last, int32_t *steps, float lr_end) {
  *loss_first = *loss_last = 0.0;
  *steps = 0;
  if (n_steps <= 0) return MCDC_OK;
  const int64_t np = mlp_param_count(n_in);
  const int np_pad = (int)((np + 3) & ~3ll);
  CKM(mlp_prepare());
  int occ = 0;
  CKM(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_mlp_train_tc, kGroups * kTM,
                                                     sizeof(TcGrad)));
  if (occ < 1) return fail(MCDC_ERR_CUDA, "the training kernel does not fit on an SM");
  const int64_t tiles = (batch + kTM - 1) / kTM;
  const int grid = (int)std::max<int64_t>(
      1, std::min<int64_t>((int64_t)sms * occ, (tiles + kGroups - 1) / kGroups));
  int32_t *d_err;
  float *part;
  unsigned long long *d_bar;
  CKM(tmp.get(&part, (size_t)grid * np_pad));
  CKM(tmp.get(&d_bar, 1));
  CKM(tmp.get(&d_err, 1));
  CKM(cudaMemsetAsync(d_bar, 0, sizeof(unsigned long long), st));
  CKM(cudaMemsetAsync(d_err, 0, sizeof(int32_t), st));
  TrainArgs ta{};
  ta.X = Xc; ta.Y = Yc; ta.W = Wc;
  ta.n_samples = n_samples; ta.batch = batch; ta.inv_wsum = d_inv;
  ta.n_in = n_in; ta.n_steps = n_steps; ta.epochs = epochs;
  ta.np = (int)np; ta.np_pad = np_pad;
  ta.p = prm; ta.m = m; ta.v = v;
  ta.part = part; ta.losses = losses; ta.bar = d_bar; ta.err = d_err;
  ta.lr = lr;
  ta.lr_end = lr_end;
  void *kargs[] = {&ta};
  CKM(cudaLaunchCooperativeKernel((const void *)k_mlp_train_tc, dim3(grid), dim3(kGroups * kTM),
                                  kargs, sizeof(TcGrad), st));
  std::vector<double> hl(2 * (size_t)n_steps);
  int32_t herr = 0;
  CKM(cudaMemcpyAsync(hl.data(), losses, sizeof(double) * 2 * n_steps, cudaMemcpyDeviceToHost, st));
  CKM(cudaMemcpyAsync(&herr, d_err, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
  CKM(cudaStreamSynchronize(st));
  if (herr) {
    tc_status();
    return fail(MCDC_ERR_TIMEOUT, "a wait in the training kernel ran out (importance network)");
  }
  double s0 = 0.0, s1 = 0.0;
  for (int b = 0; b < n_steps; ++b) { s0 += hl[b]; s1 += hl[n_steps + b]; }
  *loss_first = s0 / n_steps;
  *loss_last = epochs > 1 ? s1 / n_steps : *loss_first;
  *steps = n_steps * epochs;
  return MCDC_OK;
}

}  // namespace

extern "C" int64_t mcdc_mlp_param_count(int32_t n_in) {
  if (n_in < 1 || n_in > kIn) return -1;
  return mlp_param_count(n_in);
}

extern "C" int mcdc_mlp_forward(const float *params, int32_t n_in, const float *X, int64_t n,
                                float *out) {
  if (n_in < 1 || n_in > kIn) return fail(MCDC_ERR_INVALID, "n_in must be in 1..16");
  if (n < 0 || !params || !X || !out) return fail(MCDC_ERR_INVALID, "bad arguments");
  if (n == 0) return MCDC_OK;
  Frees fr;
  const float *dp, *dx;
  void *k1, *k2;
  CKM(as_device(params, (size_t)mlp_param_count(n_in), &dp, &k1)); fr.add(k1);
  CKM(as_device(X, (size_t)n * n_in, &dx, &k2)); fr.add(k2);
  float *dout = out;
  if (!on_dev(out)) { CKM(cudaMalloc(&dout, n * sizeof(float))); fr.add(dout); }
  CKM(mlp_prepare());
  CKM(launch_mlp_forward(nullptr, device_sms(), dp, n_in, dx, n, dout));
  if (dout != out) CKM(cudaMemcpy(out, dout, n * sizeof(float), cudaMemcpyDeviceToHost));
  CKM(cudaDeviceSynchronize());
  return tc_status();
}

extern "C" int mcdc_mlp_loss_grad(const float *params, int32_t n_in, const float *X,
                                  const float *y, const float *w, int64_t n, float *grad,
                                  double *loss) {
  if (n_in < 1 || n_in > kIn) return fail(MCDC_ERR_INVALID, "n_in must be in 1..16");
  if (n <= 0 || !params || !X || !y || !w || !grad) return fail(MCDC_ERR_INVALID, "bad arguments");
  const int64_t np = mlp_param_count(n_in);
  Frees fr;
  const float *dp, *dx, *dy, *dw;
  void *k;
  CKM(as_device(params, (size_t)np, &dp, &k)); fr.add(k);
  CKM(as_device(X, (size_t)n * n_in, &dx, &k)); fr.add(k);
  CKM(as_device(y, (size_t)n, &dy, &k)); fr.add(k);
  CKM(as_device(w, (size_t)n, &dw, &k)); fr.add(k);
  std::vector<float> hw(n);
  CKM(cudaMemcpy(hw.data(), dw, n * sizeof(float), on_dev(w) ? cudaMemcpyDeviceToHost : cudaMemcpyHostToHost));
  double wsum = 0.0;
  for (float v : hw) wsum += v;
  if (!(wsum > 0.0)) return fail(MCDC_ERR_INVALID, "sample weights sum to zero");
  float *dg = nullptr;
  double *dl = nullptr;
  CKM(cudaMalloc(&dg, np * sizeof(float))); fr.add(dg);
  CKM(cudaMalloc(&dl, sizeof(double))); fr.add(dl);
  CKM(cudaMemset(dg, 0, np * sizeof(float)));
  CKM(cudaMemset(dl, 0, sizeof(double)));
  CKM(mlp_prepare());
  CKM(launch_mlp_grad(nullptr, device_sms(), dp, n_in, dx, dy, dw, n, 0, (float)(1.0 / wsum), dg, dl));
  CKM(cudaMemcpy(grad, dg, np * sizeof(float), on_dev(grad) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost));
  double lh = 0.0;
  CKM(cudaMemcpy(&lh, dl, sizeof(double), cudaMemcpyDeviceToHost));
  if (loss) *loss = lh;
  return tc_status();
}

extern "C" int mcdc_mlp_train(float *params, int32_t n_in, const float *X, const float *y,
                              const float *w, int64_t n, int32_t epochs, int32_t batch,
                              double lr, double *loss_first, double *loss_last) {
  if (n_in < 1 || n_in > kIn) return fail(MCDC_ERR_INVALID, "n_in must be in 1..16");
  if (n <= 0 || !params || !X || !y || !w || epochs < 1 || batch < kS || !(lr > 0.0) ||
      n > 0x7fffffffll)
    return fail(MCDC_ERR_INVALID, "bad arguments");
  const int64_t np = mlp_param_count(n_in);
  int dev = 0;
  CKM(cudaGetDevice(&dev));
  cudaStream_t st;
  CKM(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
  struct StreamGone {
    cudaStream_t s;
    ~StreamGone() { cudaStreamSynchronize(s); cudaStreamDestroy(s); }
  } sg{st};
  PoolBufs tmp{device_mem_pool(dev), st, {}};
  float *dX, *dY, *dW, *prm, *m, *v, *d_inv;
  double *losses;
  const int n_steps = (int)((n + batch - 1) / batch);
  CKM(tmp.get(&dX, (size_t)n * n_in));
  CKM(tmp.get(&dY, (size_t)n));
  CKM(tmp.get(&dW, (size_t)n));
  CKM(tmp.get(&prm, (size_t)((np + 3) & ~3ll)));
  CKM(tmp.get(&m, (size_t)np));
  CKM(tmp.get(&v, (size_t)np));
  CKM(tmp.get(&d_inv, (size_t)n_steps));
  CKM(tmp.get(&losses, 2 * (size_t)n_steps));
  CKM(cudaMemcpyAsync(dX, X, sizeof(float) * n * n_in, cudaMemcpyDefault, st));
  CKM(cudaMemcpyAsync(dY, y, sizeof(float) * n, cudaMemcpyDefault, st));
  CKM(cudaMemcpyAsync(dW, w, sizeof(float) * n, cudaMemcpyDefault, st));
  CKM(cudaMemcpyAsync(prm, params, sizeof(float) * np, cudaMemcpyDefault, st));
  CKM(cudaMemsetAsync(m, 0, sizeof(float) * np, st));
  CKM(cudaMemsetAsync(v, 0, sizeof(float) * np, st));
  CKM(cudaMemsetAsync(losses, 0, sizeof(double) * 2 * n_steps, st));
  k_minibatch_inv<<<n_steps, 256, 0, st>>>(n, batch, dW, d_inv);
  CKM(cudaGetLastError());
  std::vector<float> hinv(n_steps);
  CKM(cudaMemcpyAsync(hinv.data(), d_inv, sizeof(float) * n_steps, cudaMemcpyDeviceToHost, st));
  CKM(cudaStreamSynchronize(st));
  for (float x : hinv)
    if (!(x > 0.0f)) return fail(MCDC_ERR_INVALID, "a minibatch has zero weight sum");
  double lf, ll;
  int32_t steps;
  if (int rc = train_fused(tmp, st, device_sms(), dX, dY, dW, n, n_in, epochs, batch, (float)lr,
                           d_inv, n_steps, prm, m, v, losses, &lf, &ll, &steps, (float)lr))
    return rc;
  CKM(cudaMemcpyAsync(params, prm, sizeof(float) * np, cudaMemcpyDefault, st));
  CKM(cudaStreamSynchronize(st));
  if (loss_first) *loss_first = lf;
  if (loss_last) *loss_last = ll;
  return MCDC_OK;
}

extern "C" int mcdc_set_wait_limit(int32_t tries) {
  const int v = tries < 0 ? kMbarTries : tries;
  if (cudaMemcpyToSymbol(g_tc_wait_limit, &v, sizeof(int)) != cudaSuccess) {
    cudaGetLastError();
    return fail(MCDC_ERR_CUDA, "setting the wait limit failed");
  }
  return MCDC_OK;
}

extern "C" void mcdc_default_mlp_options(mcdc_mlp_options *o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->epochs = 40;
  o->batch = 65536;
  o->lr = 2e-3;
  o->seed = 1;
  o->source_wl = 0.5;
  o->upper_ratio = 5.0;
  o->survival_ratio = 2.5;
  o->nmax = 16;
  o->min_ratio = 1e-8;
}

// Initial parameters for n_in inputs: U(-1/sqrt(fan_in), 1/sqrt(fan_in))
// weights (splitmix64 uniforms from the seed), zero biases.  active < kH:
// hidden units active.. of both layers start at zero in every weight and
// bias, and stay zero under training (their activations are SiLU(0) = 0 and
// every gradient through them vanishes), so the network has `active` units.
std::vector<float> init_params(int n_in, uint64_t seed, int active = kH) {
  std::vector<float> h((size_t)mlp_param_count(n_in), 0.0f);
  uint64_t sd = seed * 0x9E3779B97F4A7C15ull + 12345;
  auto unif = [&]() {   // splitmix64 -> (0, 1)
    sd += 0x9E3779B97F4A7C15ull;
    uint64_t z = sd;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z ^= z >> 31;
    return ((z >> 11) + 0.5) * 0x1.0p-53;
  };
  const float a1 = 1.0f / std::sqrt((float)n_in), a2 = 1.0f / std::sqrt((float)kH);
  int64_t off = 0;
  for (int64_t i = 0; i < (int64_t)kH * n_in; ++i) h[off + i] = (float)((2 * unif() - 1) * a1);
  off += (int64_t)kH * n_in + kH;
  for (int64_t i = 0; i < (int64_t)kH * kH; ++i) h[off + i] = (float)((2 * unif() - 1) * a2);
  off += (int64_t)kH * kH + kH;
  for (int64_t i = 0; i < kH; ++i) h[off + i] = (float)((2 * unif() - 1) * a2);
  if (active < kH) {
    float *W1 = h.data(), *W2 = W1 + (size_t)kH * n_in + kH, *W3 = W2 + (size_t)kH * kH + kH;
    for (int j = active; j < kH; ++j) {
      for (int k = 0; k < n_in; ++k) W1[j * n_in + k] = 0.0f;
      for (int k = 0; k < kH; ++k) W2[j * kH + k] = W2[k * kH + j] = 0.0f;
      W3[j] = 0.0f;
    }
  }
  return h;
}

// The first `active` hidden units of a kH-wide parameter vector as a network
// of that width (layout of mcdc_mlp_forward)
std::vector<float> narrow_params(const std::vector<float> &p, int n_in, int active) {
  std::vector<float> q;
  const float *W1 = p.data(), *b1 = W1 + (size_t)kH * n_in, *W2 = b1 + kH, *b2 = W2 + (size_t)kH * kH;
  const float *W3 = b2 + kH, *b3 = W3 + kH;
  for (int j = 0; j < active; ++j)
    for (int k = 0; k < n_in; ++k) q.push_back(W1[j * n_in + k]);
  for (int j = 0; j < active; ++j) q.push_back(b1[j]);
  for (int j = 0; j < active; ++j)
    for (int k = 0; k < active; ++k) q.push_back(W2[j * kH + k]);
  for (int j = 0; j < active; ++j) q.push_back(b2[j]);
  for (int j = 0; j < active; ++j) q.push_back(W3[j]);
  q.push_back(b3[0]);
  return q;
}

extern "C" int mcdc_train_importance(struct mcdc_problem *pr, const double *pilot_mean,
                                     const double *pilot_relerr, const mcdc_mlp_options *opt,
                                     mcdc_mlp_report *rep) {
  NvtxRange nvtx("mcdc_train_importance");
  if (!pr || !pilot_mean) return fail(MCDC_ERR_INVALID, "problem and pilot tally are required");
  if (pr->P.pc_target > 0)
    return fail(MCDC_ERR_INVALID, "weight windows and population control do not combine");
  mcdc_mlp_options o;
  if (opt) o = *opt; else mcdc_default_mlp_options(&o);
  if (o.epochs < 1 || o.batch < kS || !(o.lr > 0.0) || !(o.source_wl > 0.0) ||
      o.distill_steps < 0 || o.distill_hidden < 0 || o.distill_hidden > kH)
    return fail(MCDC_ERR_INVALID, "need epochs >= 1, batch >= 64, lr > 0, source_wl > 0, "
                                  "distill_steps >= 0, 0 <= distill_hidden <= 64");
  if (o.per_event && (o.adjoint || pr->tally_mode != MCDC_TALLY_GLOBAL))
    return fail(MCDC_ERR_INVALID, "per-event windows need a forward pilot and the global tally");
  const DevProblem &P = pr->P;
  const int n_in = 4 + P.G;
  if (n_in > kIn) return fail(MCDC_ERR_INVALID, "the importance network takes at most 12 groups");
  CKM(cudaSetDevice(pr->device));
  const int64_t nb = P.n_bins, np = mlp_param_count(n_in);
  Frees fr;
  const double *dmean, *drel = nullptr;
  void *k;
  CKM(as_device(pilot_mean, (size_t)nb, &dmean, &k)); fr.add(k);
  if (pilot_relerr) { CKM(as_device(pilot_relerr, (size_t)nb, &drel, &k)); fr.add(k); }
  cudaEvent_t e0, e1, e2;
  CKM(cudaEventCreate(&e0)); CKM(cudaEventCreate(&e1)); CKM(cudaEventCreate(&e2));
  cudaStream_t st;
  CKM(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
  struct Cleanup {
    cudaStream_t s; cudaEvent_t a, b, c;
    ~Cleanup() {
      cudaEventDestroy(a); cudaEventDestroy(b); cudaEventDestroy(c);
      cudaStreamDestroy(s);
    }
  } cl{st, e0, e1, e2};
  // temporaries from the device's stream-ordered pool on the training
  // stream (freed in stream order when the call returns), so repeated fits
  // pay no driver allocation
  PoolBufs tmp{device_mem_pool(pr->device), st, {}};
  float *X, *Y, *W, *pred, *prm, *m, *v;
  double *mom, *losses;
  unsigned long long *mx;
  const int np_pad = (int)((np + 3) & ~3ll);
  CKM(tmp.get(&X, (size_t)nb * n_in));
  CKM(tmp.get(&Y, (size_t)nb));
  CKM(tmp.get(&W, (size_t)nb));
  CKM(tmp.get(&pred, (size_t)nb));
  CKM(tmp.get(&prm, (size_t)np_pad));
  CKM(tmp.get(&m, (size_t)np));
  CKM(tmp.get(&v, (size_t)np));
  CKM(tmp.get(&mom, 8));
  CKM(tmp.get(&mx, 3));
  const int64_t steps_per_epoch = (nb + o.batch - 1) / o.batch;
  CKM(tmp.get(&losses, (size_t)steps_per_epoch * 2));

  std::vector<float> h = init_params(n_in, o.seed);
  const int sms = pr->sms;
  const uint64_t stride = coprime_stride((uint64_t)nb);
  CKM(mlp_prepare());
  CKM(cudaEventRecord(e0, st));
  CKM(cudaMemcpyAsync(prm, h.data(), sizeof(float) * np, cudaMemcpyHostToDevice, st));
  CKM(cudaMemsetAsync(m, 0, sizeof(float) * np, st));
  CKM(cudaMemsetAsync(v, 0, sizeof(float) * np, st));
  CKM(cudaMemsetAsync(mom, 0, sizeof(double) * 8, st));
  CKM(cudaMemsetAsync(losses, 0, sizeof(double) * steps_per_epoch * 2, st));
  const int blocks = sms * 8;
  k_make_samples<<<blocks, 256, 0, st>>>(P, n_in, stride, dmean, drel, X, Y, W, mom);
  CKM(cudaGetLastError());
  k_normalize_targets<<<blocks, 256, 0, st>>>(nb, Y, W, mom);
  CKM(cudaGetLastError());
  // training set: the scored bins only, compacted in sample order (the
  // others carry zero weight and would only cost time)
  int32_t *flag, *pos;
  float *Xc, *Yc, *Wc;
  void *scan_tmp = nullptr;
  size_t scan_bytes = 0;
  CKM(tmp.get(&flag, (size_t)nb));
  CKM(tmp.get(&pos, (size_t)nb));
  CKM(cub::DeviceScan::ExclusiveSum(nullptr, scan_bytes, flag, pos, nb, st));
  CKM(tmp.get((unsigned char **)&scan_tmp, scan_bytes));
  k_sample_flags<<<blocks, 256, 0, st>>>(nb, W, flag);
  CKM(cudaGetLastError());
  CKM(cub::DeviceScan::ExclusiveSum(scan_tmp, scan_bytes, flag, pos, nb, st));
  // one round trip: the target moments and the number of scored bins
  double hmom[8];
  int32_t last[2];
  CKM(cudaMemcpyAsync(hmom, mom, sizeof(hmom), cudaMemcpyDeviceToHost, st));
  CKM(cudaMemcpyAsync(&last[0], pos + nb - 1, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
  CKM(cudaMemcpyAsync(&last[1], flag + nb - 1, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
  CKM(cudaStreamSynchronize(st));
  if (!(hmom[0] > 0.0)) return fail(MCDC_ERR_INVALID, "the pilot tally scored no bin");
  const int64_t n_samples = (int64_t)last[0] + last[1];
  CKM(tmp.get(&Xc, (size_t)std::max<int64_t>(1, n_samples) * n_in));
  CKM(tmp.get(&Yc, (size_t)std::max<int64_t>(1, n_samples)));
  CKM(tmp.get(&Wc, (size_t)std::max<int64_t>(1, n_samples)));
  k_sample_gather<<<blocks, 256, 0, st>>>(nb, n_in, X, Y, W, flag, pos, Xc, Yc, Wc);
  CKM(cudaGetLastError());
  // minibatch b is samples [b batch, (b + 1) batch); every compacted sample
  // has positive weight, so every minibatch has a positive weight sum
  const int n_steps = (int)((n_samples + o.batch - 1) / o.batch);
  float *d_inv;
  CKM(tmp.get(&d_inv, (size_t)std::max(1, n_steps)));
  if (n_steps > 0) {
    k_minibatch_inv<<<n_steps, 256, 0, st>>>(n_samples, o.batch, Wc, d_inv);
    CKM(cudaGetLastError());
  }
  double loss_first = 0.0, loss_last = 0.0;
  int32_t steps = 0;
  if (int rc = train_fused(tmp, st, sms, Xc, Yc, Wc, n_samples, n_in, o.epochs, o.batch,
                           (float)o.lr, d_inv, n_steps, prm, m, v, losses, &loss_first,
                           &loss_last, &steps, (float)o.lr))
    return rc;
  CKM(cudaEventRecord(e1, st));
  // bake: predict every bin, weight windows proportional to the predicted flux
  CKM(launch_mlp_forward(st, sms, prm, n_in, X, nb, pred));
  CKM(cudaMemsetAsync(mx, 0, 3 * sizeof(unsigned long long), st));
  CKM(cudaMemsetAsync(mx + 1, 0xff, sizeof(unsigned long long), st));
  k_pred_max<<<blocks, 256, 0, st>>>(nb, pred, mom, mx);
  CKM(cudaGetLastError());
  k_pred_min_scored<<<blocks, 256, 0, st>>>(nb, pred, W, mom, mx + 1);
  CKM(cudaGetLastError());
  if (o.adjoint) {
    k_pred_src_max<<<blocks, 256, 0, st>>>(P, stride, pred, mom, mx + 2);
    CKM(cudaGetLastError());
  }
  const bool fold_g = !o.group_resolved && P.G > 1, fold_t = !o.time_resolved && P.T1 > 1;
  // windows of the cell alone (time and group folded, or absent)
  const bool spatial = (fold_g || P.G == 1) && (fold_t || P.T1 == 1);
  int32_t d_steps = 0;
  double d_loss = 0.0;
  if (o.per_event && !spatial) {
    // the network itself sets every window: the constants of the bake below
    // (top, floor) with the trained parameters, evaluated at each event
    unsigned long long hmx[2];
    CKM(cudaMemcpyAsync(hmx, mx, sizeof hmx, cudaMemcpyDeviceToHost, st));
    CKM(cudaEventRecord(e2, st));
    CKM(cudaStreamSynchronize(st));
    if (int rc = tc_status()) return rc;
    double top, low;
    std::memcpy(&top, &hmx[0], 8);
    std::memcpy(&low, &hmx[1], 8);
    top -= 1e4;
    low -= 1e4;
    const double floor_lp = std::fmax(low - 2.302585092994046,
                                      top + std::log(o.min_ratio > 0.0 ? o.min_ratio : 1e-8));
    if (int rc = mcdc_set_network_windows(pr, prm, n_in, kH, hmom[3], hmom[4], top, floor_lp,
                                          o.source_wl, o.upper_ratio, o.survival_ratio, o.nmax))
      return rc;
  } else {
    if (!pr->ww64) {
      void *a, *b;
      CKM(cudaMalloc(&a, sizeof(double) * nb));
      pr->allocs.push_back(a);
      CKM(cudaMalloc(&b, sizeof(float) * nb));
      pr->allocs.push_back(b);
      pr->ww64 = (double *)a;
      pr->ww32 = (float *)b;
    }
    if (o.adjoint)
      k_ww_from_importance<<<blocks, 256, 0, st>>>(P, stride, pred, mom, mx, o.source_wl,
                                                   o.min_ratio > 0.0 ? o.min_ratio : 1e-8, pr->ww64,
                                                   pr->ww32);
    else
      k_ww_from_pred<<<blocks, 256, 0, st>>>(P, stride, pred, mom, mx, mx + 1, o.source_wl,
                                             o.min_ratio > 0.0 ? o.min_ratio : 1e-8, pr->ww64,
                                             pr->ww32);
    CKM(cudaGetLastError());
    if (fold_g || fold_t) {
      k_ww_collapse<<<blocks, 256, 0, st>>>(P, fold_g, fold_t, o.adjoint != 0, pr->ww64, pr->ww32);
      CKM(cudaGetLastError());
    }
    pr->ww_table_valid = true;
    if (o.per_event) {
      // per-event windows of the cell-only table: a network of the position
      // alone is fitted to the log of the folded table, one sample per cell
      // centre, and evaluated at every window check (continuous in position,
      // folded in time and group like the table)
      const int64_t nc = P.n_cells;
      const int64_t np3 = mlp_param_count(3);
      float *X3, *Y3, *W3, *prm3, *m3, *v3, *inv3;
      double *mom3, *loss3;
      const int batch3 = (int)std::max<int64_t>(kS, std::min<int64_t>(o.batch, (nc + 7) / 8));
      const int steps3 = (int)((nc + batch3 - 1) / batch3);
      const int want3 = o.distill_steps > 0 ? o.distill_steps : 8000;
    const int epochs3 = std::max(1, (want3 + steps3 - 1) / steps3);
      CKM(tmp.get(&X3, (size_t)nc * 3));
      CKM(tmp.get(&Y3, (size_t)nc));
      CKM(tmp.get(&W3, (size_t)nc));
      CKM(tmp.get(&prm3, (size_t)((np3 + 3) & ~3ll)));
      CKM(tmp.get(&m3, (size_t)np3));
      CKM(tmp.get(&v3, (size_t)np3));
      CKM(tmp.get(&inv3, (size_t)steps3));
      CKM(tmp.get(&mom3, 8));
      CKM(tmp.get(&loss3, (size_t)steps3 * 2));
      const int h_d = o.distill_hidden > 0 ? o.distill_hidden : 16;
      const std::vector<float> h3 = init_params(3, o.seed + 1, h_d);
      CKM(cudaMemcpyAsync(prm3, h3.data(), sizeof(float) * np3, cudaMemcpyHostToDevice, st));
      CKM(cudaMemsetAsync(m3, 0, sizeof(float) * np3, st));
      CKM(cudaMemsetAsync(v3, 0, sizeof(float) * np3, st));
      CKM(cudaMemsetAsync(mom3, 0, sizeof(double) * 8, st));
      CKM(cudaMemsetAsync(loss3, 0, sizeof(double) * steps3 * 2, st));
      k_distill_samples<<<blocks, 256, 0, st>>>(P, pr->ww64, X3, Y3, W3, mom3);
      CKM(cudaGetLastError());
      k_normalize_targets<<<blocks, 256, 0, st>>>(nc, Y3, W3, mom3);
      CKM(cudaGetLastError());
      k_minibatch_inv<<<steps3, 256, 0, st>>>(nc, batch3, W3, inv3);
      CKM(cudaGetLastError());
      double d_first = 0.0;
      // the step size falls from lr to lr / 20 over the fit (cosine): the
      // table is a fixed target, fitted as closely as the steps allow
      if (int rc = train_fused(tmp, st, sms, X3, Y3, W3, nc, 3, epochs3, batch3, (float)o.lr, inv3,
                               steps3, prm3, m3, v3, loss3, &d_first, &d_loss, &d_steps,
                               (float)(o.lr / 20.0)))
        return rc;
      unsigned long long hmx[2];
      double hm3[8];
      CKM(cudaMemcpyAsync(hmx, mx, sizeof hmx, cudaMemcpyDeviceToHost, st));
      CKM(cudaMemcpyAsync(hm3, mom3, sizeof hm3, cudaMemcpyDeviceToHost, st));
      CKM(cudaEventRecord(e2, st));
      CKM(cudaStreamSynchronize(st));
      if (int rc = tc_status()) return rc;
      double top, low;
      std::memcpy(&top, &hmx[0], 8);
      std::memcpy(&low, &hmx[1], 8);
      top -= 1e4;
      low -= 1e4;
      // the table is source_wl exp(min(0, max(lp, floor_lp) - top)): its log
      // lies in [log source_wl + floor_lp - top, log source_wl], so w_L =
      // source_wl exp(min(0, max(y sd + mu, that floor) - log source_wl))
      const double floor_lp = std::fmax(low - 2.302585092994046,
                                        top + std::log(o.min_ratio > 0.0 ? o.min_ratio : 1e-8));
      const double lw0 = std::log(o.source_wl);
      std::vector<float> fit3(np3);
      CKM(cudaMemcpy(fit3.data(), prm3, sizeof(float) * np3, cudaMemcpyDeviceToHost));
      const std::vector<float> net3 = narrow_params(fit3, 3, h_d);
      if (int rc = mcdc_set_network_windows(pr, net3.data(), 3, h_d, hm3[3], hm3[4], lw0,
                                            lw0 + floor_lp - top, o.source_wl, o.upper_ratio,
                                            o.survival_ratio, o.nmax))
        return rc;
    } else {
      CKM(cudaEventRecord(e2, st));
      CKM(cudaStreamSynchronize(st));
      if (int rc = tc_status()) return rc;      // the windows are not switched on
      // switch the problem to weight windows (w_U, w_S ratios as given)
      pr->p_version += 1;
      pr->P.ww_lower = pr->ww64;
      pr->P.ww_lower32 = pr->ww32;
      pr->P.ww_net64 = nullptr;
      pr->P.ww_net32 = nullptr;
      pr->P.ww_netfrag = nullptr;
      pr->P.ww_upper = o.upper_ratio;
      pr->P.ww_survival = o.survival_ratio;
      pr->P.ww_upper32 = (float)o.upper_ratio;
      pr->P.ww_survival32 = (float)o.survival_ratio;
      pr->P.ww_nmax = o.nmax;
      if (int rc = mcdc::set_track_kernel(pr, false, true)) return rc;
      if (int rc = mcdc::ensure_overflow_for(pr)) return rc;
    }
  }
  if (rep) {
    float a = 0.f, b = 0.f;
    cudaEventElapsedTime(&a, e0, e1);
    cudaEventElapsedTime(&b, e1, e2);
    rep->samples = n_samples;
    rep->loss_first = loss_first;
    rep->loss_last = loss_last;
    rep->train_ms = a;
    rep->bake_ms = b;
    rep->steps = steps;
    rep->target_mean = hmom[1] / hmom[0];
    rep->distill_steps = d_steps;
    rep->distill_loss = d_loss;
  }
  return MCDC_OK;
}
