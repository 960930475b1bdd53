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
    for (int c = 0; c < kIn; ++c)
      st_bf16(s.X, tc::kmaj(tid, c, kIn), (row < n && c < n_in) ? X[row * n_in + c] : 0.0f);
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

// shared memory of the tcgen05 gradient kernel (operands K-major, no swizzle).
// A CTA runs two independent tile pipelines (two groups of 4 warps); each
// has its own operand tiles, tensor-memory columns, mbarrier and barrier.
constexpr int kNB = 80;    // rows of BH: H1^T (64), ones (1), zero padding
constexpr int kNX = 32;    // rows of XT: features (<= 16), ones (row 16), zero padding
constexpr int kGroups = 2;
struct TcTile {
  __nv_bfloat16 X[kTM * kIn];             // A of Z1:  [sample][in]
  __nv_bfloat16 XT[kNX * kTM];            // B of dW1: [feature | 1][sample]
  __nv_bfloat16 H1[kTM * kH];             // A of Z2:  [sample][hidden]
  __nv_bfloat16 BH[kNB * kTM];            // B of dW2: [H1^T | 1][sample]
  __nv_bfloat16 D2[kTM * kH];             // A of dH1: [sample][out]
  __nv_bfloat16 DT[kTM * kTM];            // A of dW2 / dW1: [D2^T | 0] then [D1^T | 0]
  uint64_t mbar;
  int abort;
  int pad;
};
struct TcGrad {
  __nv_bfloat16 W1[kH * kIn];             // B of Z1:  [out][in]
  __nv_bfloat16 W2[kH * kH];              // B of Z2:  [out][in]
  __nv_bfloat16 W2T[kH * kH];             // B of dH1: [in][out]
  float b1[kH], b2[kH], W3[kH];
  float red[kGroups * 4][kH + 2];         // per-warp sums of gW3, gb3, loss
  uint32_t tmem;
  int pad[3];
  TcTile t[kGroups];
};

__device__ __forceinline__ void group_sync(int g) {
  asm volatile("bar.sync %0, %1;\n" : : "r"(1 + g), "r"(kTM) : "memory");
}

// Loss sum_i w_i (f(x_i) - y_i)^2 / wsum over samples [0, n) and its gradient
// (added into grad, zeroed by the caller) with tcgen05, 128 samples per tile and
// two tiles in flight per CTA.  Tensor memory (512 columns), group g:
// Z1 in [128 g, 128 g + 64), Z2 and later dH1 in [128 g + 64, 128 g + 128),
// and its weight-gradient accumulators across tiles in [256 + 112 g,
// 256 + 112 g + 80) (DT x BH: rows o < 64 hold dW2 (cols 0-63) and gb2
// (col 64)) and [256 + 112 g + 80, 256 + 112 g + 112) (DT x XT: rows i < 64
// hold dW1 (cols < n_in) and gb1 (col 16)).  Thread r of a group owns
// sample row r of its tile (its tensor-memory lane); gW3 and gb3 build up in
// registers and are reduced once at the end.
__global__ void __launch_bounds__(kGroups * kTM) k_mlp_grad_tc(
    const float *__restrict__ p, int n_in, const float *__restrict__ X,
    const float *__restrict__ Y, const float *__restrict__ Wt, int64_t n, int64_t first,
    float inv_wsum, float *__restrict__ grad, double *__restrict__ loss) {
  extern __shared__ __align__(128) unsigned char raw[];
  TcGrad &s = *reinterpret_cast<TcGrad *>(raw);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int g = tid / kTM, r = tid % kTM;         // group and sample row
  TcTile &t = s.t[g];
  const Params q = split(p, n_in);
  for (int i = tid; i < kH * kIn; i += kGroups * kTM) {
    const int rr = i / kIn, c = i % kIn;
    st_bf16(s.W1, tc::kmaj(rr, c, kIn), c < n_in ? q.W1[rr * n_in + c] : 0.0f);
  }
  for (int i = tid; i < kH * kH; i += kGroups * kTM) {
    const int rr = i / kH, c = i % kH;
    st_bf16(s.W2, tc::kmaj(rr, c, kH), q.W2[i]);
    st_bf16(s.W2T, tc::kmaj(c, rr, kH), q.W2[i]);
  }
  for (int i = tid; i < kH; i += kGroups * kTM) { s.b1[i] = q.b1[i]; s.b2[i] = q.b2[i]; s.W3[i] = q.W3[i]; }
  // constant rows of this group's tiles: ones of XT (16) and BH (64), zero padding
  for (int rr = 0; rr < kNX; ++rr) st_bf16(t.XT, tc::kmaj(rr, r, kTM), rr == 16 ? 1.0f : 0.0f);
  st_bf16(t.BH, tc::kmaj(kH, r, kTM), 1.0f);
  for (int rr = kH + 1; rr < kNB; ++rr) st_bf16(t.BH, tc::kmaj(rr, r, kTM), 0.0f);
  for (int rr = kH; rr < kTM; ++rr) st_bf16(t.DT, tc::kmaj(rr, r, kTM), 0.0f);
  const float b3 = p[param_count(n_in) - 1];
  if (warp == 0) tc::tmem_alloc(&s.tmem, 512);
  if (r == 0) { tc::mbar_init(&t.mbar, 1); t.abort = 0; }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tm = s.tmem;
  const uint32_t lb = (uint32_t)((warp & 3) * 32) << 16;   // this warp's lanes
  const uint32_t cZ1 = 128u * g, cZ2 = cZ1 + 64, cW2 = 256u + 112u * g, cW1 = cW2 + 80;
  const uint32_t aX = tc::smem_u32(t.X), aW1 = tc::smem_u32(s.W1), aH1 = tc::smem_u32(t.H1);
  const uint32_t aW2 = tc::smem_u32(s.W2), aW2T = tc::smem_u32(s.W2T), aD2 = tc::smem_u32(t.D2);
  const uint32_t aDT = tc::smem_u32(t.DT), aBH = tc::smem_u32(t.BH), aXT = tc::smem_u32(t.XT);
  uint32_t phase = 0;
  bool pending = false, started = false;
  float my_loss = 0.0f, my_gb3 = 0.0f, gw3[kH];
#pragma unroll
  for (int o = 0; o < kH; ++o) gw3[o] = 0.0f;
  const float *Xs = X + first * n_in;
  const float *Ys = Y + first;
  const float *Ws = Wt + first;
  auto wait_mma = [&]() {
    pending = true;
    if (!tc::mbar_wait(&t.mbar, phase, g_tc_wait_limit)) { atomicOr(&g_tc_timeout, 1); t.abort = 1; }
    phase ^= 1u;
    group_sync(g);
    if (!t.abort) pending = false;
    tc::fence_after_sync();
    return !t.abort;
  };
  for (int64_t base = ((int64_t)blockIdx.x * kGroups + g) * kTM; base < n;
       base += (int64_t)gridDim.x * kGroups * kTM) {
    const int64_t row = base + r;
    const bool valid = row < n;
    const float yv = valid ? Ys[row] : 0.0f, wv = valid ? Ws[row] : 0.0f;
    for (int c = 0; c < kIn; ++c) {
      const float v = (valid && c < n_in) ? Xs[row * n_in + c] : 0.0f;
      st_bf16(t.X, tc::kmaj(r, c, kIn), v);
      if (c < n_in) st_bf16(t.XT, tc::kmaj(c, r, kTM), v);
    }
    tc::fence_async_smem();
    group_sync(g);
    if (r == 0) {
      tc::fence_after_sync();
      tc::mma(tm + cZ1, tc::desc(aX, 128, 256), tc::desc(aW1, 128, 256), tc::idesc_bf16(kTM, kH), 0);
      tc::commit(&t.mbar);
    }
    if (!wait_mma()) break;
    // layer 1: H1 and H1^T
    float v[16], u[16];
#pragma unroll 1
    for (int q4 = 0; q4 < 4; ++q4) {
      tc::ld16(tm + lb + cZ1 + 16 * q4, v);
#pragma unroll
      for (int c = 0; c < 16; ++c) {
        const int o = 16 * q4 + c;
        const float h = silu(v[c] + s.b1[o]);
        st_bf16(t.H1, tc::kmaj(r, o, kH), h);
        st_bf16(t.BH, tc::kmaj(o, r, kTM), h);
      }
    }
    tc::fence_before_sync();
    tc::fence_async_smem();
    group_sync(g);
    if (r == 0) {
      tc::fence_after_sync();
#pragma unroll
      for (int kk = 0; kk < kH / 16; ++kk)
        tc::mma(tm + cZ2, tc::desc(aH1 + 256 * kk, 128, 1024), tc::desc(aW2 + 256 * kk, 128, 1024),
                tc::idesc_bf16(kTM, kH), kk > 0);
      tc::commit(&t.mbar);
    }
    if (!wait_mma()) break;
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
    my_loss += wv * e * e * inv_wsum;
    my_gb3 += dy;
#pragma unroll
    for (int q4 = 0; q4 < 4; ++q4) {
      tc::ld16(tm + lb + cZ2 + 16 * q4, v);
#pragma unroll
      for (int c = 0; c < 16; ++c) {
        const int o = 16 * q4 + c;
        const float z2 = v[c] + s.b2[o];
        gw3[o] += dy * silu(z2);
        const float d2 = dy * s.W3[o] * dsilu(z2);
        st_bf16(t.D2, tc::kmaj(r, o, kH), d2);
        st_bf16(t.DT, tc::kmaj(o, r, kTM), d2);
      }
    }
    tc::fence_before_sync();
    tc::fence_async_smem();
    group_sync(g);
    if (r == 0) {
      tc::fence_after_sync();
#pragma unroll
      for (int kk = 0; kk < kH / 16; ++kk)           // dH1 = D2 W2 (over Z2's columns)
        tc::mma(tm + cZ2, tc::desc(aD2 + 256 * kk, 128, 1024), tc::desc(aW2T + 256 * kk, 128, 1024),
                tc::idesc_bf16(kTM, kH), kk > 0);
#pragma unroll
      for (int kk = 0; kk < kTM / 16; ++kk)          // [dW2 | gb2] += DT BH
        tc::mma(tm + cW2, tc::desc(aDT + 256 * kk, 128, 2048), tc::desc(aBH + 256 * kk, 128, 2048),
                tc::idesc_bf16(kTM, kNB), (started || kk > 0) ? 1u : 0u);
      tc::commit(&t.mbar);
    }
    if (!wait_mma()) break;
    // dL/dz1 = dH1 * silu'(z1) -> DT rows [0, 64)
#pragma unroll 1
    for (int q4 = 0; q4 < 4; ++q4) {
      tc::ld16(tm + lb + cZ2 + 16 * q4, v);
      tc::ld16(tm + lb + cZ1 + 16 * q4, u);
#pragma unroll
      for (int c = 0; c < 16; ++c) {
        const int i = 16 * q4 + c;
        st_bf16(t.DT, tc::kmaj(i, r, kTM), v[c] * dsilu(u[c] + s.b1[i]));
      }
    }
    tc::fence_before_sync();
    tc::fence_async_smem();
    group_sync(g);
    if (r == 0) {
      tc::fence_after_sync();
#pragma unroll
      for (int kk = 0; kk < kTM / 16; ++kk)          // [dW1 | gb1] += DT XT
        tc::mma(tm + cW1, tc::desc(aDT + 256 * kk, 128, 2048), tc::desc(aXT + 256 * kk, 128, 2048),
                tc::idesc_bf16(kTM, kNX), (started || kk > 0) ? 1u : 0u);
      tc::commit(&t.mbar);
    }
    started = true;
    if (!wait_mma()) break;
  }
  if (pending) tc::mbar_wait(&t.mbar, phase ^ 1u, kMbarTries);
  // gW3, gb3 and the loss: warp sums into shared memory, then one pass
#pragma unroll
  for (int o = 0; o < kH; ++o) {
    float a = gw3[o];
    for (int d = 16; d > 0; d >>= 1) a += __shfl_xor_sync(0xffffffffu, a, d);
    if (lane == 0) s.red[warp][o] = a;
  }
  for (int d = 16; d > 0; d >>= 1) {
    my_gb3 += __shfl_xor_sync(0xffffffffu, my_gb3, d);
    my_loss += __shfl_xor_sync(0xffffffffu, my_loss, d);
  }
  if (lane == 0) { s.red[warp][kH] = my_gb3; s.red[warp][kH + 1] = my_loss; }
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
  if (ok && started && (warp & 3) < 2) {
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

// Adam (Kingma & Ba): FP32 master weights and moments.
__global__ void k_adam(int64_t np, float *__restrict__ p, float *__restrict__ m,
                       float *__restrict__ v, const float *__restrict__ g, float lr, float b1,
                       float b2, float eps, float c1, float c2) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < np;
       i += (int64_t)gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
  }
}

// ---- host side -------------------------------------------------------------

size_t mlp_smem_bytes() { return sizeof(TcGrad); }

cudaError_t mlp_prepare() {
  cudaError_t e = cudaFuncSetAttribute(k_mlp_grad_tc, cudaFuncAttributeMaxDynamicSharedMemorySize,
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

cudaError_t launch_adam(cudaStream_t st, int64_t np, float *p, float *m, float *v, const float *g,
                        float lr, int64_t t) {
  const float b1 = 0.9f, b2 = 0.999f;
  const float c1 = 1.f - powf(b1, (float)t), c2 = 1.f - powf(b2, (float)t);
  k_adam<<<(int)((np + 255) / 256), 256, 0, st>>>(np, p, m, v, g, lr, b1, b2, 1e-8f, c1, c2);
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

__global__ void k_step_counter(int64_t *t) { *t += 1; }

// Adam whose step count lives on the device (so a captured epoch can be
// replayed): c1 = 1 - b1^t, c2 = 1 - b2^t.
__global__ void k_adam_dev(int64_t np, float *__restrict__ p, float *__restrict__ m,
                           float *__restrict__ v, const float *__restrict__ g, float lr,
                           const int64_t *__restrict__ t) {
  const float b1 = 0.9f, b2 = 0.999f;
  const float c1 = 1.f - powf(b1, (float)*t), c2 = 1.f - powf(b2, (float)*t);
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < np;
       i += (int64_t)gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + 1e-8f);
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

extern "C" int mcdc_train_importance(struct mcdc_problem *pr, const double *pilot_mean,
                                     const double *pilot_relerr, const mcdc_mlp_options *opt,
                                     mcdc_mlp_report *rep) {
  NvtxRange nvtx("mcdc_train_importance");
  if (!pr || !pilot_mean) return fail(MCDC_ERR_INVALID, "problem and pilot tally are required");
  if (pr->P.pc_target > 0)
    return fail(MCDC_ERR_INVALID, "weight windows and population control do not combine");
  mcdc_mlp_options o;
  if (opt) o = *opt; else mcdc_default_mlp_options(&o);
  if (o.epochs < 1 || o.batch < kS || !(o.lr > 0.0) || !(o.source_wl > 0.0))
    return fail(MCDC_ERR_INVALID, "need epochs >= 1, batch >= 64, lr > 0, source_wl > 0");
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
  float *X, *Y, *W, *pred, *prm, *m, *v, *g;
  double *mom, *losses;
  int64_t *tstep;
  unsigned long long *mx;
  CKM(cudaMalloc(&X, sizeof(float) * nb * n_in)); fr.add(X);
  CKM(cudaMalloc(&Y, sizeof(float) * nb)); fr.add(Y);
  CKM(cudaMalloc(&W, sizeof(float) * nb)); fr.add(W);
  CKM(cudaMalloc(&pred, sizeof(float) * nb)); fr.add(pred);
  CKM(cudaMalloc(&prm, sizeof(float) * np)); fr.add(prm);
  CKM(cudaMalloc(&m, sizeof(float) * np)); fr.add(m);
  CKM(cudaMalloc(&v, sizeof(float) * np)); fr.add(v);
  CKM(cudaMalloc(&g, sizeof(float) * np)); fr.add(g);
  CKM(cudaMalloc(&mom, sizeof(double) * 8)); fr.add(mom);
  CKM(cudaMalloc(&tstep, sizeof(int64_t))); fr.add(tstep);
  CKM(cudaMalloc(&mx, 3 * sizeof(unsigned long long))); fr.add(mx);
  const int64_t steps_per_epoch = (nb + o.batch - 1) / o.batch;
  CKM(cudaMalloc(&losses, sizeof(double) * steps_per_epoch * 2)); fr.add(losses);

  // parameters: U(-1/sqrt(fan_in), 1/sqrt(fan_in)) weights, zero biases
  std::vector<float> h(np, 0.0f);
  {
    uint64_t st = o.seed * 0x9E3779B97F4A7C15ull + 12345;
    auto unif = [&]() {   // splitmix64 -> (0, 1)
      st += 0x9E3779B97F4A7C15ull;
      uint64_t z = st;
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
  }
  cudaEvent_t e0, e1, e2;
  CKM(cudaEventCreate(&e0)); CKM(cudaEventCreate(&e1)); CKM(cudaEventCreate(&e2));
  cudaStream_t st;
  CKM(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
  struct Cleanup {
    cudaStream_t s; cudaEvent_t a, b, c; cudaGraph_t gr = nullptr; cudaGraphExec_t ex = nullptr;
    ~Cleanup() {
      if (ex) cudaGraphExecDestroy(ex);
      if (gr) cudaGraphDestroy(gr);
      cudaEventDestroy(a); cudaEventDestroy(b); cudaEventDestroy(c);
      cudaStreamDestroy(s);
    }
  } cl{st, e0, e1, e2};
  const int sms = pr->sms;
  const uint64_t stride = coprime_stride((uint64_t)nb);
  CKM(mlp_prepare());
  CKM(cudaEventRecord(e0, st));
  CKM(cudaMemcpyAsync(prm, h.data(), sizeof(float) * np, cudaMemcpyHostToDevice, st));
  CKM(cudaMemsetAsync(m, 0, sizeof(float) * np, st));
  CKM(cudaMemsetAsync(v, 0, sizeof(float) * np, st));
  CKM(cudaMemsetAsync(mom, 0, sizeof(double) * 8, st));
  CKM(cudaMemsetAsync(tstep, 0, sizeof(int64_t), st));
  CKM(cudaMemsetAsync(losses, 0, sizeof(double) * steps_per_epoch * 2, st));
  const int blocks = sms * 8;
  k_make_samples<<<blocks, 256, 0, st>>>(P, n_in, stride, dmean, drel, X, Y, W, mom);
  CKM(cudaGetLastError());
  k_normalize_targets<<<blocks, 256, 0, st>>>(nb, Y, W, mom);
  CKM(cudaGetLastError());
  double hmom[8];
  CKM(cudaMemcpyAsync(hmom, mom, sizeof(hmom), cudaMemcpyDeviceToHost, st));
  CKM(cudaStreamSynchronize(st));
  if (!(hmom[0] > 0.0)) return fail(MCDC_ERR_INVALID, "the pilot tally scored no bin");
  // training set: the scored bins only, compacted in sample order (the
  // others carry zero weight and would only cost time)
  int32_t *flag, *pos;
  float *Xc, *Yc, *Wc;
  void *scan_tmp = nullptr;
  size_t scan_bytes = 0;
  CKM(cudaMalloc(&flag, sizeof(int32_t) * nb)); fr.add(flag);
  CKM(cudaMalloc(&pos, sizeof(int32_t) * nb)); fr.add(pos);
  CKM(cub::DeviceScan::ExclusiveSum(nullptr, scan_bytes, flag, pos, nb, st));
  CKM(cudaMalloc(&scan_tmp, scan_bytes)); fr.add(scan_tmp);
  k_sample_flags<<<blocks, 256, 0, st>>>(nb, W, flag);
  CKM(cudaGetLastError());
  CKM(cub::DeviceScan::ExclusiveSum(scan_tmp, scan_bytes, flag, pos, nb, st));
  int32_t last[2];
  CKM(cudaMemcpyAsync(&last[0], pos + nb - 1, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
  CKM(cudaMemcpyAsync(&last[1], flag + nb - 1, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
  CKM(cudaStreamSynchronize(st));
  const int64_t n_samples = (int64_t)last[0] + last[1];
  CKM(cudaMalloc(&Xc, sizeof(float) * std::max<int64_t>(1, n_samples) * n_in)); fr.add(Xc);
  CKM(cudaMalloc(&Yc, sizeof(float) * std::max<int64_t>(1, n_samples))); fr.add(Yc);
  CKM(cudaMalloc(&Wc, sizeof(float) * std::max<int64_t>(1, n_samples))); fr.add(Wc);
  k_sample_gather<<<blocks, 256, 0, st>>>(nb, n_in, X, Y, W, flag, pos, Xc, Yc, Wc);
  CKM(cudaGetLastError());
  // per-minibatch weight sums (host side, from the device weights)
  const int64_t steps_used = (n_samples + o.batch - 1) / o.batch;
  std::vector<float> hw(std::max<int64_t>(1, n_samples));
  CKM(cudaMemcpyAsync(hw.data(), Wc, sizeof(float) * n_samples, cudaMemcpyDeviceToHost, st));
  CKM(cudaStreamSynchronize(st));
  std::vector<float> inv(steps_per_epoch, 0.0f);
  for (int64_t b = 0; b < steps_used; ++b) {
    double ws = 0.0;
    for (int64_t i = b * o.batch; i < std::min<int64_t>(n_samples, (b + 1) * o.batch); ++i)
      ws += hw[i];
    inv[b] = ws > 0.0 ? (float)(1.0 / ws) : 0.0f;
  }
  // one epoch as a CUDA graph: per minibatch zero the gradient, forward and
  // backward on the tensor cores, count the step, Adam
  CKM(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
  for (int64_t b = 0; b < steps_used; ++b) {
    if (inv[b] == 0.0f) continue;
    const int64_t first = b * o.batch, cnt = std::min<int64_t>(o.batch, n_samples - first);
    cudaMemsetAsync(g, 0, sizeof(float) * np, st);
    launch_mlp_grad(st, sms, prm, n_in, Xc, Yc, Wc, cnt, first, inv[b], g, losses + b);
    k_step_counter<<<1, 1, 0, st>>>(tstep);
    k_adam_dev<<<(int)((np + 255) / 256), 256, 0, st>>>(np, prm, m, v, g, (float)o.lr, tstep);
  }
  CKM(cudaStreamEndCapture(st, &cl.gr));
  CKM(cudaGraphInstantiate(&cl.ex, cl.gr, 0));
  double loss_first = 0.0, loss_last = 0.0;
  std::vector<double> hl(steps_per_epoch);
  int32_t steps = 0;
  for (int ep = 0; ep < o.epochs; ++ep) {
    CKM(cudaMemsetAsync(losses, 0, sizeof(double) * steps_per_epoch, st));
    CKM(cudaGraphLaunch(cl.ex, st));
    if (ep == 0 || ep == o.epochs - 1) {
      CKM(cudaMemcpyAsync(hl.data(), losses, sizeof(double) * steps_per_epoch, cudaMemcpyDeviceToHost, st));
      CKM(cudaStreamSynchronize(st));
      double s = 0.0, c = 0.0;
      for (int64_t b = 0; b < steps_per_epoch; ++b)
        if (inv[b] != 0.0f) { s += hl[b]; c += 1.0; }
      (ep == 0 ? loss_first : loss_last) = c > 0 ? s / c : 0.0;
    }
    for (int64_t b = 0; b < steps_per_epoch; ++b) steps += inv[b] != 0.0f;
  }
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
  if (o.per_event) {
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
    if (int rc = mcdc_set_network_windows(pr, prm, kH, hmom[3], hmom[4], top, floor_lp,
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
  const bool fold_g = !o.group_resolved && P.G > 1, fold_t = !o.time_resolved && P.T1 > 1;
  if (fold_g || fold_t) {
    k_ww_collapse<<<blocks, 256, 0, st>>>(P, fold_g, fold_t, o.adjoint != 0, pr->ww64, pr->ww32);
    CKM(cudaGetLastError());
  }
  CKM(cudaEventRecord(e2, st));
  CKM(cudaStreamSynchronize(st));
  if (int rc = tc_status()) return rc;      // the windows are not switched on
  // switch the problem to weight windows (w_U, w_S ratios as given)
  pr->P.ww_lower = pr->ww64;
  pr->P.ww_lower32 = pr->ww32;
  pr->P.ww_upper = o.upper_ratio;
  pr->P.ww_survival = o.survival_ratio;
  pr->P.ww_nmax = o.nmax;
  if (int rc = mcdc::ensure_overflow_for(pr)) return rc;
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
  }
  return MCDC_OK;
}
