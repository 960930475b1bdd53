// tracker.cuh -- persistent, event-based particle tracker.
//
// Every lane of a warp flies one particle held in registers; the warp's
// flights are one dense pass.  A flight ends at a collision, a mesh surface,
// a time census or the end of the history: surface and census events are
// resolved in place, collisions park the particle in the warp's pool in
// shared memory (a stack growing down), and once 32 are parked one dense
// collision pass absorbs or scatters them and pushes the survivors on the
// ready stack (growing up).  Empty lanes pop ready particles; when none are
// ready, one dense pass of up to 32 births (split children first, then new
// source histories) hands newborns to empty lanes by warp shuffle.  All
// queues are built with warp ballots and popc prefixes.  Cross-section
// tables sit in shared memory.  The tally is a CTA-private copy in shared
// memory holding one batch at a time (shared mode) or a device-wide batch
// tally, optionally one slice per batch (global mode).
//
// Per particle, the sequence of draws, distances and events is the same as
// in the one-history-at-a-time loop of the paper's "MC/DC on CPUs" section,
// so the FP64 instantiation (built without FMA contraction) reproduces a
// plain FP64 tracker event for event.
#pragma once
#include <cfloat>
#include <cmath>
#include <math_constants.h>
#include "common.cuh"
#include "tc.cuh"

namespace mcdc {

// Precision modes.  R: direction, distance, cross sections; TT: shared
// tally; Q: position and time.
struct PrecF64 {        // everything in FP64 (event-exact with an FP64 tracker)
  using R = double;
  using TT = double;
  using Q = double;
  static constexpr bool kF64 = true;
  static constexpr bool kLocal = false;
};
struct PrecF32 {        // FP32 split: FP64 position and time accumulated every flight
  using R = float;
  using TT = float;
  using Q = double;
  static constexpr bool kF64 = false;
  static constexpr bool kLocal = false;
};
struct PrecF32L {       // FP32 cell-local: offsets from exact FP64 faces and census edges
  using R = float;
  using TT = float;
  using Q = float;
  static constexpr bool kF64 = false;
  static constexpr bool kLocal = true;
};

template <class PR>
using PartOf = Part<typename PR::R, typename PR::Q>;

template <class R> __device__ __forceinline__ R rinf();
template <> __device__ __forceinline__ double rinf<double>() { return CUDART_INF; }
template <> __device__ __forceinline__ float rinf<float>() { return CUDART_INF_F; }

// shared-memory copies of the per-material tables
template <class R>
struct Tables {
  R *sigma_t, *scat, *cdf;   // [M*G], [M*G], [M*G*G]
  R *src_cdf;                // [G]
  double *speed;             // [G]
  R *inv_speed;              // [G] (FP32 path)
  float *speed32;            // [G]
  double *edges;             // [T+1]
  const double *ww;          // global
  const float *ww32;
};

// Pool of parked particles in shared memory: one array per group of fields,
// each element 8 or 16 bytes, so a particle moves in four to six vector
// accesses.  Cell indices, time bin and group are packed into 32-bit words.
template <class PR>
struct Bank {
  using R = typename PR::R;
  void *xt;           // FP64 position: double2 {x, t}; cell-local: float4 {x, y, z, t}
  double2 *yz;        // FP64 position, 3-D only: {y, z}
  void *d0;           // FP32: float4 {ux, uy, uz, w}; FP64: double2 {ux, uy}
  double2 *d1;        // FP64 only: {uz, w}
  uint4 *ids;         // {ctr, serial, hid low, hid high}
  uint4 *cell;        // {i | j << 16, k | tbin << 16, g, nseg}
  uint4 *cnt;         // {ncol, ncross, slot, optical depth (FP32 modes)}

  // with_slot: also the particle's input position (population control only;
  // other launches leave it out of their registers)
  __device__ __forceinline__ void load(int s, PartOf<PR> &p, int dim, bool with_slot = true) const {
    if constexpr (PR::kLocal) {
      const float4 a = reinterpret_cast<const float4 *>(xt)[s];
      p.x = a.x; p.y = a.y; p.z = a.z; p.t = a.w;
    } else {
      const double2 a = reinterpret_cast<const double2 *>(xt)[s];
      p.x = a.x; p.t = a.y;
      if (dim == 3) { const double2 b = yz[s]; p.y = b.x; p.z = b.y; } else { p.y = 0.0; p.z = 0.0; }
    }
    if constexpr (sizeof(R) == 4) {
      const float4 c = reinterpret_cast<const float4 *>(d0)[s];
      p.ux = c.x; p.uy = c.y; p.uz = c.z; p.w = c.w;
    } else {
      const double2 c0 = reinterpret_cast<const double2 *>(d0)[s];
      const double2 c1 = d1[s];
      p.ux = c0.x; p.uy = c0.y; p.uz = c1.x; p.w = c1.y;
    }
    const uint4 id = ids[s];
    p.ctr = id.x; p.serial = id.y; p.hid = (uint64_t)id.z | ((uint64_t)id.w << 32);
    const uint4 ce = cell[s];
    p.i = (int)(ce.x & 0xffffu); p.j = (int)(ce.x >> 16);
    p.k = (int)(ce.y & 0xffffu); p.tbin = (int)(ce.y >> 16);
    p.g = (int)ce.z; p.nseg = ce.w;
    const uint4 cn = cnt[s];
    p.ncol = cn.x; p.ncross = cn.y; p.slot = with_slot ? cn.z : 0u; p.tau = __uint_as_float(cn.w);
  }
  __device__ __forceinline__ void store(int s, const PartOf<PR> &p, int dim, bool with_slot = true) const {
    if constexpr (PR::kLocal) {
      reinterpret_cast<float4 *>(xt)[s] = make_float4(p.x, p.y, p.z, p.t);
    } else {
      reinterpret_cast<double2 *>(xt)[s] = make_double2(p.x, p.t);
      if (dim == 3) yz[s] = make_double2(p.y, p.z);
    }
    if constexpr (sizeof(R) == 4) {
      reinterpret_cast<float4 *>(d0)[s] = make_float4(p.ux, p.uy, p.uz, p.w);
    } else {
      reinterpret_cast<double2 *>(d0)[s] = make_double2(p.ux, p.uy);
      d1[s] = make_double2(p.uz, p.w);
    }
    ids[s] = make_uint4(p.ctr, p.serial, (uint32_t)p.hid, (uint32_t)(p.hid >> 32));
    cell[s] = make_uint4((uint32_t)p.i | ((uint32_t)p.j << 16), (uint32_t)p.k | ((uint32_t)p.tbin << 16),
                         (uint32_t)p.g, p.nseg);
    cnt[s] = make_uint4(p.ncol, p.ncross, with_slot ? p.slot : 0u, __float_as_uint(p.tau));
  }
};

// bytes of one pool slot (kept in sync with the carve in k_track)
__host__ __device__ inline int slot_bytes(bool f64, int dim, bool local) {
  return 16 + ((dim == 3 && !local) ? 16 : 0) + (f64 ? 32 : 16) + 16 + 16 + 16;
}

// The pool's structure-of-arrays layout over any memory: cap slots carved
// from base as xt, yz (3-D, not cell-local), d0, d1 (FP64), ids, cell, cnt,
// 16 bytes per slot each -- slot_bytes(...) x cap bytes in all.  Shared
// memory holds the warps' pools this way; device memory holds the banks that
// population control writes at scattered positions and copies in bulk (one
// 16-byte access per field group and slot, coalesced over consecutive slots).
template <class PR>
__device__ __forceinline__ Bank<PR> bank_view(void *base, long long cap, int dim) {
  Bank<PR> b;
  unsigned char *ptr = static_cast<unsigned char *>(base);
  b.xt = ptr; ptr += 16 * cap;
  if (dim == 3 && !PR::kLocal) { b.yz = (double2 *)ptr; ptr += 16 * cap; } else { b.yz = nullptr; }
  b.d0 = ptr; ptr += 16 * cap;
  if constexpr (PR::kF64) { b.d1 = (double2 *)ptr; ptr += 16 * cap; } else { b.d1 = nullptr; }
  b.ids = (uint4 *)ptr; ptr += 16 * cap;
  b.cell = (uint4 *)ptr; ptr += 16 * cap;
  b.cnt = (uint4 *)ptr;
  return b;
}

// particles a warp can park in shared memory besides the 32 in flight
constexpr int kPool = 96;
constexpr int kReserve = 256;   // population control: input positions a warp reserves at once

// shared-memory layout of one CTA
struct Layout {
  int M, G, T;           // table sizes the carve reserves (the largest problem of a batch)
  int S;                 // pool slots of the whole CTA (warps x kPool)
  int tables_bytes;
  long long tally_bytes; // 0 in global mode
  int bank_bytes;
  int total;
  int net_bytes;         // FP32 per-event network kernels: the fragment block and the
                         // warps' tiles (kNetFragBytes + warps x kNetWarpBytes)
};

// The warp-batched network evaluation of the FP32 modes reads the network
// from shared memory, arranged on the host in the order of the mma.sync
// m16n8k16 B fragments (F16 pairs; hidden padded to 64, inputs to 32) so that
// each lane loads its fragment as one 8-byte word:
//   W1 / 2 fragments [n-tile 8][k-step 2][lane 32][2 words]   words    0 .. 1023
//   W2 / 2 fragments [n-tile 8][k-step 4][lane 32][2 words]   words 1024 .. 3071
//   b1 / 2, b2 / 2 in FP32, 64 each                           words 3072 .. 3199
//   W3 fragments, output in column 0 of one n-tile:
//                    [k-step 4][lane 32][2 words]             words 3200 .. 3455
// (the halves make the hidden accumulators z / 2, the argument SiLU's tanh
// takes; scaling by 2^-1 is exact)
constexpr int kNetW1Frag = 0, kNetW2Frag = 1024, kNetB1 = 3072, kNetB2 = 3136, kNetW3Frag = 3200;
constexpr int kNetFragWords = 3456;
constexpr int kNetFragBytes = kNetFragWords * 4;     // 13824, a multiple of 16
// then per warp: its input tile, 32 rows of 32 F16 inputs padded to 80 bytes
// (the 8 rows of an ldmatrix phase fall in distinct banks), and the 32
// outputs of its rows
constexpr int kNetRowBytes = 80;
constexpr int kNetWarpBytes = 32 * kNetRowBytes + 32 * 4;
// threads per CTA of the network instantiations: at most 384, so that each
// thread may hold 168 registers (the evaluation's fragments and accumulators
// on top of the event loop's state) where 512 threads would cap it at 128
constexpr int kNetBlockMax = 384;

__host__ __device__ inline int align16(long long v) { return (int)((v + 15) & ~15ll); }

inline int tables_bytes_of(bool f64, int M, int G, int T) {
  const int r = f64 ? 8 : 4;
  long long b = 0;
  b += align16((long long)r * M * G) * 2;          // sigma_t, scat
  b += align16((long long)r * M * G * G);          // cdf
  b += align16((long long)r * G);                  // src cdf
  b += align16(8ll * G);                           // speed
  b += align16((long long)r * G);                  // inv speed
  b += align16(4ll * G);                           // speed (FP32)
  b += align16(8ll * (T + 1));                     // edges
  return (int)b;
}

// per-thread event counters, flushed once per CTA
struct LocalCount {
  uint32_t seg, col, cross, census;
};

// ---------------------------------------------------------------------------
// geometry helpers (FP64 in both precisions)
// face coordinate origin + k * width, read from a table built on the host
// with the same two roundings
__device__ __forceinline__ double face_of(const DevProblem &P, int a, int idx, bool up) {
  const int k = up ? idx + 1 : idx;
  return __ldg(P.faces[a] + k);
}

__device__ __forceinline__ int loc2index(const DevProblem &P, int a, double x) {
  if (!P.bounded[a]) return 0;
  const double f = floor((x - P.origin[a]) / P.width[a]);
  int i = (int)f;
  if (f < 0.0) i = 0;
  if (f > (double)(P.n[a] - 1)) i = P.n[a] - 1;
  return i;
}

template <class R>
__device__ __forceinline__ int sample_cdf(const R *cdf, int n, R xi) {
  for (int k = 0; k < n; ++k)
    if (xi <= cdf[k]) return k;
  return n - 1;
}

template <int DIM>
__device__ __forceinline__ int cell_index(const DevProblem &P, int i, int j, int k) {
  if (DIM == 1) return i;
  return (k * P.n[1] + j) * P.n[0] + i;
}

__device__ __forceinline__ int bin_index(const DevProblem &P, int cell, int g, int tbin) {
  return (cell * P.G + g) * P.T1 + (P.T > 0 ? tbin : 0);
}

// ---------------------------------------------------------------------------
// records and termination bookkeeping
struct EndSink {
  double *w_end;        // shared [4]: source, absorbed, leaked, censused
  uint32_t *n_end;      // shared [9]: absorbed, leaked, censused, roulette kill, survive, splits,
                        // children, histories, children not made (no room)
};

template <class PR, int DIM>
__device__ __forceinline__ void finish(const DevProblem &P, const RunArgs &A, const EndSink &es,
                                       const PartOf<PR> &p, int end) {
  // analog runs carry weight 1 throughout: their weight sums are the counts
  // (filled in on the host), so only weighted runs add weights here
  const bool weighted = weights_summed(P);
  if (end == END_ABSORBED) { atomicAdd(&es.n_end[0], 1u); if (weighted) atomicAdd(&es.w_end[1], (double)p.w); }
  else if (end == END_LEAKED) { atomicAdd(&es.n_end[1], 1u); if (weighted) atomicAdd(&es.w_end[2], (double)p.w); }
  else if (end == END_CENSUSED) { atomicAdd(&es.n_end[2], 1u); if (weighted) atomicAdd(&es.w_end[3], (double)p.w); }
  else if (end == END_ROULETTE) { atomicAdd(&es.n_end[3], 1u); }
  if (A.records != nullptr && p.serial == 0u) {
    const uint64_t r = p.hid - A.offset;
    if (r < A.n_records) {
      Record rec;
      rec.hid = p.hid; rec.end = end; rec.g = p.g; rec.ctr = p.ctr;
      rec.n_seg = p.nseg; rec.n_col = p.ncol; rec.n_cross = p.ncross;
      if constexpr (PR::kLocal) {
        // global coordinates from the exact anchors
        rec.x = P.bounded[0] ? __ldg(P.faces[0] + p.i) + (double)p.x : 0.0;
        rec.y = (DIM == 3 && P.bounded[1]) ? __ldg(P.faces[1] + p.j) + (double)p.y : 0.0;
        rec.z = (DIM == 3 && P.bounded[2]) ? __ldg(P.faces[2] + p.k) + (double)p.z : 0.0;
        rec.t = P.T > 0 ? (p.tbin < P.T ? P.edges[p.tbin + 1] - (double)p.t : P.edges[P.T]) : 0.0;
      } else {
        rec.x = p.x; rec.y = p.y; rec.z = p.z; rec.t = p.t;
      }
      rec.w = (double)p.w;
      A.records[r] = rec;
    }
  }
}

// ---------------------------------------------------------------------------
// Per-event windows: the importance network evaluated at the particle.
// Inputs: position scaled to [-1, 1] over each bounded axis of the mesh; a
// network of 4 + G inputs also takes time as 2 (j + (t - t_j) / (t_j+1 - t_j))
// / T - 1 in time bin j (0 in steady state) and the group one-hot -- the
// continuous versions of the cell and bin centres the network is trained on
// (a network of 3 inputs takes the position alone).  FP64 mode evaluates in
// FP64 in the order of the oracle's loops; the FP32 modes in FP32.  Not
// inlined: the hidden layer lives in this call's own frame, off the
// tracker's registers.
template <class PR, int DIM>
__device__ __noinline__ typename PR::R net_window(const DevProblem &P, const PartOf<PR> &p) {
  using R = typename PR::R;
  double pos[3], t;
  if constexpr (PR::kLocal) {
    pos[0] = P.bounded[0] ? __ldg(P.faces[0] + p.i) + (double)p.x : 0.0;
    pos[1] = (DIM == 3 && P.bounded[1]) ? __ldg(P.faces[1] + p.j) + (double)p.y : 0.0;
    pos[2] = (DIM == 3 && P.bounded[2]) ? __ldg(P.faces[2] + p.k) + (double)p.z : 0.0;
    t = P.T > 0 ? P.edges[p.tbin + 1] - (double)p.t : 0.0;
  } else {
    pos[0] = p.x; pos[1] = p.y; pos[2] = p.z; t = p.t;
  }
  R f[4 + 16];
  for (int a = 0; a < 3; ++a)
    f[a] = P.bounded[a] ? (R)(2.0 * (pos[a] - P.origin[a]) / ((double)P.n[a] * P.width[a]) - 1.0)
                        : (R)0;
  if (P.ww_net_in == 3) {
    // position only
  } else if (P.T > 0) {
    const int j = p.tbin < P.T ? p.tbin : P.T - 1;
    const double u = (t - P.edges[j]) / (P.edges[j + 1] - P.edges[j]);
    f[3] = (R)(2.0 * ((double)j + u) / (double)P.T - 1.0);
  } else {
    f[3] = (R)0;
  }
  const int in = P.ww_net_in, H = P.ww_net_h;
  for (int k = 4; k < in; ++k) f[k] = (k - 4 == p.g) ? (R)1 : (R)0;
  const R *W1;
  if constexpr (PR::kF64) W1 = P.ww_net64; else W1 = P.ww_net32;
  const R *b1 = W1 + H * in, *W2 = b1 + H, *b2 = W2 + H * H, *W3 = b2 + H, *b3 = W3 + H;
  R h1[64];
  for (int j = 0; j < H; ++j) {
    R a = b1[j];
    for (int k = 0; k < in; ++k) a += W1[j * in + k] * f[k];
    if constexpr (PR::kF64) h1[j] = a / (1.0 + exp(-a)); else h1[j] = __fdividef(a, 1.0f + __expf(-a));
  }
  R y = b3[0];
  for (int j = 0; j < H; ++j) {
    R a = b2[j];
    for (int k = 0; k < H; ++k) a += W2[j * H + k] * h1[k];
    R h2;
    if constexpr (PR::kF64) h2 = a / (1.0 + exp(-a)); else h2 = __fdividef(a, 1.0f + __expf(-a));
    y += W3[j] * h2;
  }
  double lp = (double)y * P.ww_net_scale + P.ww_net_shift;
  if (lp < P.ww_net_floor) lp = P.ww_net_floor;
  const double e = lp - P.ww_net_top;
  return (R)(P.ww_net_wl0 * exp(e < 0.0 ? e : 0.0));
}

// ---------------------------------------------------------------------------
// Weight windows at collisions and cell crossings.  The split or roulette of
// a window check with lower bound wl (wl <= 0: no window here); returns false
// if the particle is rouletted away.  Children go to the warp's overflow
// stack (s_novf[0]: its size, s_novf[32]: its current limit) or the spill
// bank; s_novf[16] is the warp's reservation of the run's children budget.
template <class PR, int DIM>
__device__ bool ww_apply(const DevProblem &P, const RunArgs &A, const EndSink &es,
                         PartOf<PR> &p, typename PR::R wl, int *s_novf, PartOf<PR> *ovf) {
  using R = typename PR::R;
  if (!(wl > (R)0)) return true;
  R wu;
  if constexpr (PR::kF64) wu = P.ww_upper * wl; else wu = P.ww_upper32 * wl;
  if (p.w > wu) {
    const R nd = ceil(p.w / wu);
    const int n = nd > (R)P.ww_nmax ? P.ww_nmax : (int)nd;
    if (n > 1) {
      // children go to the warp's stack, else to the device-wide spill bank;
      // a child that finds no room is not made and the parent keeps its
      // weight (splitting is optional, so the estimate stays unbiased)
      const R wc = p.w / (R)n;
      int made = 0;
      // the run's budget of children: past it no child is made (as when the
      // banks are full), which bounds the work of windows that would split
      // without end.  The warp draws on a reservation in shared memory
      // (s_novf[16]) refilled from the run's counter 256 children at a time.
      int room = n - 1;
      if (A.children_made != nullptr) {
        int *left = s_novf + 16;
        if (atomicSub(left, n - 1) < n - 1) {
          atomicAdd(left, n - 1);
          const unsigned long long before = atomicAdd(A.children_made, 256ull);
          if (before + 256ull <= A.children_budget) atomicAdd(left, 256 - (n - 1));
          else room = 0;
        }
      }
      for (int c = 1; c <= room; ++c) {
        const U4 h = philox4x32_10_rk(0xFFFFFFFFu, p.serial, p.ctr, (uint32_t)c, A.rk);
        PartOf<PR> ch = p;
        ch.w = wc;
        ch.serial = h.a;
        ch.ctr = 0;
        ch.nseg = ch.ncol = ch.ncross = 0;
        ch.tau = -1.0f;                 // FP32 modes: drawn from the child's own stream
        const int slot = atomicAdd(s_novf, 1);
        if (slot < s_novf[32]) {          // the warp's current stack limit
          ovf[slot] = ch;
          made += 1;
        } else {
          atomicSub(s_novf, 1);
          if (A.spill_out != nullptr) {
            const unsigned long long gs = atomicAdd(A.spill_out_count, 1ull);
            if (gs < A.spill_cap) {
              reinterpret_cast<PartOf<PR> *>(A.spill_out)[gs] = ch;
              made += 1;
            }
          }
        }
      }
      p.w = (made == n - 1) ? wc : p.w - (R)made * wc;
      // children's serials hash the parent's (serial, counter): when flights
      // draw nothing (optical depth carried) a split consumes one counter
      // value, so two splits of a particle never hand out the same streams
      if constexpr (!PR::kF64) {
        if (!P.fresh_tau) p.ctr += 1;
      }
      atomicAdd(&es.n_end[5], 1u);
      atomicAdd(&es.n_end[6], (uint32_t)made);
      if (made < n - 1) atomicAdd(&es.n_end[8], (uint32_t)(n - 1 - made));
    }
    return true;
  }
  if (p.w < wl) {
    R ws;
    if constexpr (PR::kF64) ws = P.ww_survival * wl; else ws = P.ww_survival32 * wl;
    const U4 r = draw(p, p.ctr, A.rk);
    R xi;
    if constexpr (PR::kF64) xi = u01_f64(r.a, r.b); else xi = u01_f32(r.a);
    if (xi < p.w / ws) {
      p.w = ws;
      atomicAdd(&es.n_end[4], 1u);
      return true;
    }
    return false;
  }
  return true;
}

// A window check: the lower bound from the table, or from the network
// evaluated at the particle (one particle at a time; the FP32 network kernels
// evaluate a warp's checks together instead, see net_window_warp), then the
// split or roulette.
template <class PR, int DIM, bool NET>
__device__ bool weight_window(const DevProblem &P, const Tables<typename PR::R> &tb,
                              const RunArgs &A, const EndSink &es, PartOf<PR> &p,
                              int *s_novf, PartOf<PR> *ovf) {
  using R = typename PR::R;
  if (tb.ww == nullptr && !(NET && P.ww_net64 != nullptr)) return true;
  R wl;
  if (NET && P.ww_net64 != nullptr) {
    // FP64 kernels; the FP32 ones check in warps (flight and collide defer)
    if constexpr (NET && PR::kF64) wl = net_window<PR, DIM>(P, p);
    else wl = (R)0;
  } else {
    const int cell = cell_index<DIM>(P, p.i, p.j, p.k);
    const int bin = bin_index(P, cell, p.g, p.tbin);
    if (!MCDC_CHK(A.error, CHK_WW_BIN, bin >= 0 && bin < P.n_bins, bin)) return true;
    if constexpr (PR::kF64) wl = tb.ww[bin]; else wl = tb.ww32[bin];
  }
  return ww_apply<PR, DIM>(P, A, es, p, wl, s_novf, ovf);
}

// ---------------------------------------------------------------------------
// isotropic direction from one block: mu = 2 xi - 1 is the x cosine, phi =
// 2 pi xi' the azimuth.  A 1-D slab only ever uses the x cosine, so there
// the azimuth is drawn (the block is the same) but not evaluated.
template <class PR, int DIM>
__device__ __forceinline__ void isotropic(const U4 &r2, PartOf<PR> &p) {
  if constexpr (PR::kF64) {
    const double mu = 2.0 * u01_f64(r2.a, r2.b) - 1.0;
    p.ux = mu;
    if (DIM == 3) {
      const double two_pi = 6.283185307179586;
      const double phi = two_pi * u01_f64(r2.c, r2.d);
      const double s = sqrt(1.0 - mu * mu);
      p.uy = s * cos(phi); p.uz = s * sin(phi);
    } else {
      p.uy = 0.0; p.uz = 0.0;
    }
  } else {
    const float mu = 2.0f * u01_f32(r2.a) - 1.0f;
    p.ux = mu;
    if (DIM == 3) {
      const float s = sqrtf(fmaxf(0.0f, 1.0f - mu * mu));
      float sn, cs;
      sincospif(2.0f * u01_f32(r2.c), &sn, &cs);
      p.uy = s * cs; p.uz = s * sn;
    } else {
      p.uy = 0.0f; p.uz = 0.0f;
    }
  }
}

// ---------------------------------------------------------------------------
// source particle (counters 0..3: x,y | z,group | mu,phi | t)
template <class PR, int DIM>
__device__ void source_particle(const DevProblem &P, const Tables<typename PR::R> &tb,
                                const RoundKeys &rk, uint64_t hid, PartOf<PR> &p) {
  using R = typename PR::R;
  p.serial = 0; p.ctr = 0; p.hid = hid;
  p.nseg = p.ncol = p.ncross = 0;
  p.slot = 0;
  const U4 r0 = draw(p, p.ctr, rk);
  const U4 r1 = draw(p, p.ctr, rk);
  const U4 r2 = draw(p, p.ctr, rk);
  const U4 r3 = draw(p, p.ctr, rk);
  if constexpr (PR::kF64) p.g = sample_cdf<double>(tb.src_cdf, P.G, u01_f64(r1.c, r1.d));
  else p.g = sample_cdf<float>(tb.src_cdf, P.G, u01_f32(r1.c));
  if (P.src_kind == 1) {
    p.ux = (R)P.src_dir[0]; p.uy = (R)P.src_dir[1]; p.uz = (R)P.src_dir[2];
  } else {
    isotropic<PR, DIM>(r2, p);
  }
  p.w = (R)1;
  if constexpr (PR::kF64) {
    // FP64: the oracle's arithmetic (53-bit uniforms, loc2index)
    const double x = P.src_lo[0] + u01_f64(r0.a, r0.b) * (P.src_hi[0] - P.src_lo[0]);
    const double y = P.src_lo[1] + u01_f64(r0.c, r0.d) * (P.src_hi[1] - P.src_lo[1]);
    const double z = P.src_lo[2] + u01_f64(r1.a, r1.b) * (P.src_hi[2] - P.src_lo[2]);
    const double t = P.t0 + u01_f64(r3.a, r3.b) * (P.t1 - P.t0);
    p.tau = -1.0f;
    p.i = loc2index(P, 0, x);
    p.j = (DIM == 3) ? loc2index(P, 1, y) : 0;
    p.k = (DIM == 3) ? loc2index(P, 2, z) : 0;
    p.tbin = 0;
    if (P.T > 0)
      while (p.tbin < P.T && tb.edges[p.tbin + 1] <= t) p.tbin += 1;
    p.x = x; p.y = y; p.z = z; p.t = t;
  } else {
    // FP32 modes: 24-bit uniforms (the top bits of the FP64 run's), each
    // coordinate in cell units as one FP32 multiply-add, the cell its floor
    // and the offset from the cell's low face the rest -- no FP64 division.
    // The optical depth to the first collision comes from the time block's
    // third word (unused by the FP32 draws).
    p.tau = -logf(u01_f32(r3.c));
    const float xi[3] = {u01_f32(r0.a), u01_f32(r0.c), u01_f32(r1.a)};
    float off[3] = {0.0f, 0.0f, 0.0f};
    int idx[3] = {0, 0, 0};
#pragma unroll
    for (int a = 0; a < DIM; ++a) {
      if (!P.bounded[a]) continue;
      const float f = fmaf(xi[a], P.src_cell_b[a], P.src_cell_a[a]);
      const int i = min(max((int)floorf(f), 0), P.n[a] - 1);
      idx[a] = i;
      off[a] = fminf(fmaxf((f - (float)i) * P.width32[a], 0.0f), P.width32[a]);
    }
    p.i = idx[0]; p.j = idx[1]; p.k = idx[2];
    // birth time: t0 for a pulse (no FP64 work), else uniform in [t0, t1]
    const double t = P.t1 > P.t0 ? P.t0 + (double)u01_f32(r3.a) * (P.t1 - P.t0) : P.t0;
    p.tbin = 0;
    if (P.T > 0)
      while (p.tbin < P.T && tb.edges[p.tbin + 1] <= t) p.tbin += 1;
    if constexpr (PR::kLocal) {
      // offsets from the cell's low faces; time left to the next census edge
      p.x = off[0]; p.y = off[1]; p.z = off[2];
      p.t = (P.T > 0 && p.tbin < P.T) ? (float)(tb.edges[p.tbin + 1] - t) : 0.0f;
    } else {
      p.x = P.bounded[0] ? __ldg(P.faces[0] + p.i) + (double)off[0] : 0.0;
      p.y = (DIM == 3 && P.bounded[1]) ? __ldg(P.faces[1] + p.j) + (double)off[1] : 0.0;
      p.z = (DIM == 3 && P.bounded[2]) ? __ldg(P.faces[2] + p.k) + (double)off[2] : 0.0;
      p.t = t;
    }
  }
}

// ---------------------------------------------------------------------------
// one flight.  Returns 0 continue, 1 collision queued, 2 ended (end code in
// *end), 3 reached an interior census edge under population control (banked)
// 3 reached an interior census edge under population control (banked),
// 4 crossed into a new cell with its window check left to the warp (FP32
// network kernels: net_check_warp after the flight pass)
enum Outcome { OUT_CONT = 0, OUT_COLL = 1, OUT_DEAD = 2, OUT_BANKED = 3, OUT_WW = 4 };

template <class PR, int DIM, bool NET, bool PC, bool VR>
__device__ __forceinline__ int flight(const DevProblem &P, const Tables<typename PR::R> &tb,
                                      const RunArgs &A, const EndSink &es,
                                      PartOf<PR> &p, int &bin,
                                      typename PR::R &score, int &end, LocalCount &lc,
                                      int *s_novf, PartOf<PR> *ovf) {
  using R = typename PR::R;
  const int cell = cell_index<DIM>(P, p.i, p.j, p.k);
  if (!MCDC_CHK(A.error, CHK_CELL, cell >= 0 && cell < P.n_cells, cell) ||
      !MCDC_CHK(A.error, CHK_GROUP, p.g >= 0 && p.g < P.G, p.g) ||
      !MCDC_CHK(A.error, CHK_MATERIAL, __ldg(P.material + cell) < P.M, __ldg(P.material + cell))) {
    bin = -1; score = (R)0;
    end = END_LEAKED;
    return OUT_DEAD;
  }
  const int m = __ldg(P.material + cell);
  const int mg = m * P.G + p.g;
  const R sig_t = tb.sigma_t[mg];

  // distance to collision.  FP64: sampled afresh every flight (the oracle's
  // reading, for event-exact parity).  FP32 modes: by default the optical
  // depth tau to the next collision is carried across surface and census
  // events (the exponential law is memoryless, so the collision sites have
  // the same distribution) and redrawn only at collisions, births and for new
  // split children -- a flight needs no random number; with fresh_tau every
  // flight draws it as FP64 does (the same random numbers as an FP64 run).
  // Division: the approximate (2-ulp) quotient, far below the FP32 noise.
  R d_coll;
  if constexpr (PR::kF64) {
    const U4 r = draw(p, p.ctr, A.rk);
    const double xi = u01_f64(r.a, r.b);
    d_coll = sig_t > 0.0 ? -log(xi) / sig_t : rinf<double>();
  } else {
    if (P.fresh_tau || !(p.tau >= 0.0f)) {
      const U4 r = draw(p, p.ctr, A.rk);
      p.tau = -logf(u01_f32(r.a));
    }
    d_coll = sig_t > 0.0f ? __fdividef(p.tau, sig_t) : rinf<float>();
  }

  // distance to the mesh surface and to the time census
  R d_surf = rinf<R>();
  int ax = -1;
  R d_time = rinf<R>();
  if constexpr (PR::kLocal) {
    // cell-local offsets: the face ahead is at width (moving up) or 0
    {
      const float u = p.ux;
      if (P.bounded[0] && u != 0.0f) {
        float d = __fdividef(u > 0.0f ? P.width32[0] - p.x : -p.x, u);
        if (d < 0.0f) d = 0.0f;
        if (d < d_surf) { d_surf = d; ax = 0; }
      }
    }
    if (DIM == 3) {
      const float u = p.uy;
      if (P.bounded[1] && u != 0.0f) {
        float d = __fdividef(u > 0.0f ? P.width32[1] - p.y : -p.y, u);
        if (d < 0.0f) d = 0.0f;
        if (d < d_surf) { d_surf = d; ax = 1; }
      }
      const float v = p.uz;
      if (P.bounded[2] && v != 0.0f) {
        float d = __fdividef(v > 0.0f ? P.width32[2] - p.z : -p.z, v);
        if (d < 0.0f) d = 0.0f;
        if (d < d_surf) { d_surf = d; ax = 2; }
      }
    }
    if (P.T > 0) {
      d_time = tb.speed32[p.g] * p.t;
      if (d_time < 0.0f) d_time = 0.0f;
    }
  } else {
    {
      const R u = p.ux;
      if (P.bounded[0] && u != (R)0) {
        const double f = face_of(P, 0, p.i, u > (R)0);
        R d;
        if constexpr (PR::kF64) d = (f - p.x) / u; else d = __fdividef((float)(f - p.x), u);
        if (d < (R)0) d = (R)0;
        if (d < d_surf) { d_surf = d; ax = 0; }
      }
    }
    if (DIM == 3) {
      const R u = p.uy;
      if (P.bounded[1] && u != (R)0) {
        const double f = face_of(P, 1, p.j, u > (R)0);
        R d;
        if constexpr (PR::kF64) d = (f - p.y) / u; else d = __fdividef((float)(f - p.y), u);
        if (d < (R)0) d = (R)0;
        if (d < d_surf) { d_surf = d; ax = 1; }
      }
      const R v = p.uz;
      if (P.bounded[2] && v != (R)0) {
        const double f = face_of(P, 2, p.k, v > (R)0);
        R d;
        if constexpr (PR::kF64) d = (f - p.z) / v; else d = __fdividef((float)(f - p.z), v);
        if (d < (R)0) d = (R)0;
        if (d < d_surf) { d_surf = d; ax = 2; }
      }
    }

    // distance to the time census
    if (P.T > 0) {
      if constexpr (PR::kF64) d_time = tb.speed[p.g] * (tb.edges[p.tbin + 1] - p.t);
      else d_time = tb.speed32[p.g] * (float)(tb.edges[p.tbin + 1] - p.t);
      if (d_time < (R)0) d_time = (R)0;
    }

  }

  int ev = 0;  // 0 collision, 1 surface, 2 census
  R d = d_coll;
  if (d_surf <= d) { d = d_surf; ev = 1; }
  if (d_time <= d) { d = d_time; ev = 2; }

  lc.seg += 1;
  p.nseg += 1;
  if (d == rinf<R>()) {          // a flight with nothing ahead: gone to infinity
    bin = -1; score = (R)0;
    end = END_LEAKED;
    return OUT_DEAD;
  }
  if constexpr (!PR::kF64) {      // optical depth used up by a flight that did not collide
    if (ev != 0) p.tau = fmaxf(p.tau - sig_t * d, 0.0f);
  }
  if (P.estimator != 1) {         // track-length estimator (alone or combined)
    bin = bin_index(P, cell, p.g, p.tbin);
    score = p.w * d;
    if (!MCDC_CHK(A.error, CHK_TBIN, P.T == 0 || (p.tbin >= 0 && p.tbin < P.T), p.tbin)) bin = -1;
  }

  // move_particle (Figure "jitfunctions"): x += u d, t += d / v
  if constexpr (PR::kLocal) {
    p.x += p.ux * d;
    if (DIM == 3) { p.y += p.uy * d; p.z += p.uz * d; }
    if (P.T > 0) p.t -= d * tb.inv_speed[p.g];
  } else if constexpr (PR::kF64) {
    p.x += p.ux * d;
    if (DIM == 3) { p.y += p.uy * d; p.z += p.uz * d; }
    p.t += d / tb.speed[p.g];
  } else {
    p.x += (double)(p.ux * d);
    if (DIM == 3) { p.y += (double)(p.uy * d); p.z += (double)(p.uz * d); }
    if (P.T > 0) p.t += (double)(d * tb.inv_speed[p.g]);
  }

  if (ev == 2) {
    lc.census += 1;
    p.tbin += 1;
    if constexpr (PR::kLocal) p.t = p.tbin < P.T ? __ldg(P.binw32 + p.tbin) : 0.0f;
    else p.t = tb.edges[p.tbin];
    if (p.tbin == P.T) { end = END_CENSUSED; return OUT_DEAD; }
    if (PC && A.census_out != nullptr) return OUT_BANKED;   // waits for the comb
    return OUT_CONT;
  }
  if (ev == 1) {
    R u; int idx;
    if (ax == 0) { u = p.ux; idx = p.i; }
    else if (ax == 1) { u = p.uy; idx = p.j; }
    else { u = p.uz; idx = p.k; }
    const bool up = u > (R)0;
    const int nxt = idx + (up ? 1 : -1);
    const bool out = nxt < 0 || nxt >= P.n[ax];
    if constexpr (PR::kLocal) {
      // onto the face: the far side of the new cell, or the same face when
      // a reflecting boundary keeps the particle in its cell
      const float on = (up != out) ? 0.0f : P.width32[ax];
      if (ax == 0) p.x = on; else if (ax == 1) p.y = on; else p.z = on;
    } else {
      const double f = face_of(P, ax, idx, up);
      if (ax == 0) p.x = f; else if (ax == 1) p.y = f; else p.z = f;
    }
    if (out) {
      if (P.bc[2 * ax + (up ? 1 : 0)] == 1) {
        if (ax == 0) p.ux = -u; else if (ax == 1) p.uy = -u; else p.uz = -u;
        return OUT_CONT;
      }
      end = END_LEAKED;
      return OUT_DEAD;
    }
    if (ax == 0) p.i = nxt; else if (ax == 1) p.j = nxt; else p.k = nxt;
    p.ncross += 1;
    lc.cross += 1;
    if constexpr (NET && !PR::kF64) {
      if (P.ww_net32 != nullptr) return OUT_WW;
    }
    if constexpr (VR || NET) {
      if (!weight_window<PR, DIM, NET>(P, tb, A, es, p, s_novf, ovf)) { end = END_ROULETTE; return OUT_DEAD; }
    }
    return OUT_CONT;
  }
  return OUT_COLL;
}

// collision: absorb or scatter, new group from the transfer CDF, isotropic
// direction.  Returns true if the particle lives on.  Collision estimator:
// (cbin, cscore) is the arriving particle's score w / sigma_t.  Implicit
// capture: the weight is multiplied by sigma_s / sigma_t (the removed part is
// returned in wabs), a weight that reaches 0 ends as absorbed, and a weight
// below the cutoff is rouletted after the scatter (one more block).
template <class PR, int DIM, bool NET, bool PC, bool VR>
__device__ __forceinline__ bool collide(const DevProblem &P, const Tables<typename PR::R> &tb,
                                        const RunArgs &A, const EndSink &es,
                                        PartOf<PR> &p, int &end, LocalCount &lc,
                                        int *s_novf, PartOf<PR> *ovf,
                                        int &cbin, typename PR::R &cscore, double &wabs,
                                        bool &ww_pend) {
  using R = typename PR::R;
  const int cell = cell_index<DIM>(P, p.i, p.j, p.k);
  if (!MCDC_CHK(A.error, CHK_CELL, cell >= 0 && cell < P.n_cells, cell) ||
      !MCDC_CHK(A.error, CHK_GROUP, p.g >= 0 && p.g < P.G, p.g) ||
      !MCDC_CHK(A.error, CHK_MATERIAL, __ldg(P.material + cell) < P.M, __ldg(P.material + cell))) {
    end = END_ABSORBED;
    return false;
  }
  const int m = __ldg(P.material + cell);
  const int mg = m * P.G + p.g;
  p.ncol += 1;
  lc.col += 1;
  if (P.estimator != 0) {         // collision estimator (alone or combined)
    cbin = bin_index(P, cell, p.g, p.tbin);
    cscore = p.w / tb.sigma_t[mg];
    if (!MCDC_CHK(A.error, CHK_TBIN, P.T == 0 || (p.tbin >= 0 && p.tbin < P.T), p.tbin)) cbin = -1;
  }
  const U4 r1 = draw(p, p.ctr, A.rk);
  // FP32 modes with the optical depth carried use one 24-bit number per
  // choice: absorption r1.a, group r1.c, cosine and optical depth from the
  // direction block's a and b, azimuth from its c.  When the direction needs
  // no azimuth (1-D) or the group needs no number (one group), the first
  // block's b and d serve as the cosine and the optical depth (and its c as
  // the azimuth), and the collision draws one block instead of two.
  bool one_block = false;
  if constexpr (!PR::kF64) one_block = !P.fresh_tau && (DIM == 1 || P.G == 1);
  const U4 r2 = one_block ? U4{r1.b, r1.d, r1.c, r1.d} : draw(p, p.ctr, A.rk);
  const R ratio = tb.scat[mg];
  R xi1, xi2;
  if constexpr (PR::kF64) { xi1 = u01_f64(r1.a, r1.b); xi2 = u01_f64(r1.c, r1.d); }
  else { xi1 = u01_f32(r1.a); xi2 = u01_f32(r1.c); }
  // implicit capture exists in the weighted instantiations only
  constexpr bool kImplicit = VR || NET || PC;
  if (kImplicit && P.implicit) {
    if constexpr (PR::kF64) wabs = p.w * (1.0 - ratio);
    else wabs = (double)p.w * (1.0 - (double)ratio);
    p.w *= ratio;
    if (!(p.w > (R)0)) { end = END_ABSORBED; return false; }
  } else if (!(xi1 < ratio)) {
    end = END_ABSORBED;
    return false;
  }
  p.g = sample_cdf<R>(tb.cdf + mg * P.G, P.G, xi2);
  isotropic<PR, DIM>(r2, p);
  // FP32 modes: optical depth to the next collision from the direction
  // block's second word (unused by the FP32 draws)
  if constexpr (!PR::kF64) p.tau = -logf(u01_f32(r2.b));
  if (kImplicit && P.implicit) {
    R wcut, wsurv;
    if constexpr (PR::kF64) { wcut = P.wcut; wsurv = P.wsurv; }
    else { wcut = P.wcut32; wsurv = P.wsurv32; }
    if (p.w < wcut) {
      const U4 r = draw(p, p.ctr, A.rk);
      R xi;
      if constexpr (PR::kF64) xi = u01_f64(r.a, r.b); else xi = u01_f32(r.a);
      if (!(xi < p.w / wsurv)) { end = END_ROULETTE; return false; }
      p.w = wsurv;
      atomicAdd(&es.n_end[4], 1u);
    }
  }
  if constexpr (NET && !PR::kF64) {
    // FP32 network kernels: the check is left to the warp (net_check_warp)
    if (P.ww_net32 != nullptr) { ww_pend = true; return true; }
  }
  if constexpr (VR || NET) {
    if (!weight_window<PR, DIM, NET>(P, tb, A, es, p, s_novf, ovf)) { end = END_ROULETTE; return false; }
  }
  return true;
}

// ---------------------------------------------------------------------------
// tally scatter of one warp: optional warp aggregation of equal bins
// (global tallies: the FP32 slices gtally32 when set, else the FP64 gtally)
template <class TT, class R>
__device__ __forceinline__ void tally_scatter(TT *stally, double *gtally, float *gtally32,
                                              bool shared_mode, bool aggregate, bool valid,
                                              int bin, R score, long long goff, int32_t *err,
                                              long long extent) {
  bool act = valid && bin >= 0;
  if (act && !MCDC_CHK(err, CHK_TALLY, goff + bin < extent, goff + bin)) act = false;
  R v = score;
  if (aggregate) {
    // lanes scoring into the same bin add their scores first; the lowest
    // such lane issues the one atomic.  All 32 lanes run the same shuffles.
    const long long key = act ? goff + bin : -1ll;
    const unsigned peers = __match_any_sync(0xffffffffu, key);
    const bool dup = act && __popc(peers) > 1;
    if (__any_sync(0xffffffffu, dup)) {
      R sum = (R)0;
      for (int src = 0; src < 32; ++src) {
        const R o = __shfl_sync(0xffffffffu, v, src);
        if ((peers >> src) & 1u) sum += o;
      }
      if (act) {
        v = sum;
        act = ((threadIdx.x & 31) == __ffs(peers) - 1);
      }
    }
  }
  if (act) {
    if (shared_mode) atomicAdd(&stally[bin], (TT)v);
    else if (gtally32 != nullptr) atomicAdd(&gtally32[goff + bin], (float)v);
    else atomicAdd(&gtally[goff + bin], (double)v);
  }
}

// offset of the particle's tally slice (population control: one per batch)
__device__ __forceinline__ long long tally_offset(const DevProblem &P, const RunArgs &A,
                                                  uint64_t hid) {
  if (!A.tally_per_batch) return 0;
  return (long long)batch_of_run(A, hid - A.offset) * P.n_tally;
}

// population-control step tally: entry of (estimator half e, batch, cell x
// group) for a tally bin of the launch's time bin
__device__ __forceinline__ int step_bin(const DevProblem &P, const RunArgs &A, uint64_t hid,
                                        int bin, int e) {
  const int per = (int)(P.n_cells * P.G);
  return (e * A.n_batches + batch_of_run(A, hid - A.offset)) * per + bin / P.T1;
}

// ---------------------------------------------------------------------------
// index of the n-th (0-based) set bit of a 32-bit word (binary search on popc)
__device__ __forceinline__ int nth32(uint32_t m, int n) {
  int pos = 0;
#pragma unroll
  for (int s = 16; s > 0; s >>= 1) {
    const int c = __popc(m & ((1u << s) - 1u));
    if (n >= c) { n -= c; m >>= s; pos += s; }
  }
  return pos;
}

__device__ __forceinline__ uint32_t lanemask_lt() {
  return (1u << (threadIdx.x & 31)) - 1u;
}

// ---------------------------------------------------------------------------
// Warp-batched per-event windows (FP32 modes).  The window checks a warp
// meets in one flight pass or one collision pass are gathered into the rows
// of an M = 16 or 32 tile (the pending lanes in lane order: each writes its
// inputs as binary16 into row `rank` of the warp's tile in shared memory)
// and the network runs on the tensor cores as three products, mma.sync
// m16n8k16 with binary16 operands and FP32 accumulation (A fragments of the
// inputs by ldmatrix).  Layers 1 and 2 use halved weights and biases, so
// their accumulators are h = z / 2, and SiLU(z) = h + h tanh(h) (sigma(z) =
// (1 + tanh(z / 2)) / 2) runs on binary16 pairs, one tanh.approx.f16x2 for two
// values; the pairs are already the A fragments of the next product (an
// m16n8 C tile pair has the register layout of an m16k16 A tile).  The output
// layer is a product with one n-tile whose column 0 holds W3: its
// accumulator's column 0 is the output of each row.  Hidden units beyond the
// network's width have zero weights and biases (SiLU(0) = 0 keeps them out);
// inputs beyond n_in are zero.

__device__ __forceinline__ uint32_t pack_f16x2(float lo, float hi) {
  uint32_t d;
  asm("cvt.rn.f16x2.f32 %0, %1, %2;" : "=r"(d) : "f"(hi), "f"(lo));
  return d;
}

// SiLU(2 h0), SiLU(2 h1) as a binary16 pair: h + h tanh(h)
__device__ __forceinline__ uint32_t silu_half_f16x2(float h0, float h1) {
  const uint32_t h = pack_f16x2(h0, h1);
  uint32_t t, r;
  asm("tanh.approx.f16x2 %0, %1;" : "=r"(t) : "r"(h));
  asm("fma.rn.f16x2 %0, %1, %2, %1;" : "=r"(r) : "r"(h), "r"(t));
  return r;
}

__device__ __forceinline__ void mma_f16_16816(float (&c)[4], const uint32_t (&a)[4], uint2 b) {
  asm("mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 "
      "{%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, {%0, %1, %2, %3};"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b.x), "r"(b.y));
}

__device__ __forceinline__ void ldmatrix_x4(uint32_t (&r)[4], uint32_t addr) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0, %1, %2, %3}, [%4];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]) : "r"(addr));
}

// The network outputs y (before the window mapping) of rows 0..16 MT - 1 of
// the warp's tile, into ys[row]; all 32 lanes call it together.  NT n-tiles
// (8 hidden units each; even) hold the network's units, K2: a second K step
// of inputs (more than 16), MT M-tiles of 16 rows, run side by side (each B
// fragment is loaded once for both).  nf: the fragment block, tile_s: the
// warp's tile (shared-window address), ys: its outputs.
template <int NT, bool K2, int MT>
__device__ __forceinline__ void net_eval_t(const uint32_t *nf, uint32_t tile_s, float *ys,
                                           float b3) {
  constexpr int KS = NT / 2;            // K steps over the hidden units
  const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  const uint2 *w1 = reinterpret_cast<const uint2 *>(nf + kNetW1Frag);
  const uint2 *w2 = reinterpret_cast<const uint2 *>(nf + kNetW2Frag);
  const uint2 *w3 = reinterpret_cast<const uint2 *>(nf + kNetW3Frag);
  const float2 *b1 = reinterpret_cast<const float2 *>(nf + kNetB1);
  const float2 *b2 = reinterpret_cast<const float2 *>(nf + kNetB2);
  // A of layer 1: lanes 0-7 address matrix 0 (rows 0-7, inputs 0-7), 8-15
  // matrix 1 (rows 8-15), 16-23 matrix 2 (rows 0-7, inputs 8-15), 24-31
  // matrix 3 (rows 8-15, inputs 8-15)
  uint32_t a1[MT][K2 ? 2 : 1][4];
#pragma unroll
  for (int mt = 0; mt < MT; ++mt) {
    const int row = mt * 16 + (lane & 7) + ((lane >> 3) & 1) * 8;
    const uint32_t addr = tile_s + row * kNetRowBytes + (lane >> 4) * 16;
    ldmatrix_x4(a1[mt][0], addr);
    if constexpr (K2) ldmatrix_x4(a1[mt][1], addr + 32);
  }
  // layer 1 -> SiLU -> A of layer 2 (K step s = n-tiles 2 s, 2 s + 1)
  uint32_t a2[MT][KS][4];
#pragma unroll
  for (int j = 0; j < NT; ++j) {
    const float2 bb = b1[4 * j + t];
    const uint2 f0 = w1[(j * 2 + 0) * 32 + lane];
    uint2 f1 = make_uint2(0u, 0u);
    if constexpr (K2) f1 = w1[(j * 2 + 1) * 32 + lane];
#pragma unroll
    for (int mt = 0; mt < MT; ++mt) {
      float c[4] = {bb.x, bb.y, bb.x, bb.y};
      mma_f16_16816(c, a1[mt][0], f0);
      if constexpr (K2) mma_f16_16816(c, a1[mt][1], f1);
      a2[mt][j >> 1][2 * (j & 1) + 0] = silu_half_f16x2(c[0], c[1]);
      a2[mt][j >> 1][2 * (j & 1) + 1] = silu_half_f16x2(c[2], c[3]);
    }
  }
  // layer 2 -> SiLU -> A of the output layer
  uint32_t a3[MT][KS][4];
#pragma unroll
  for (int j = 0; j < NT; ++j) {
    const float2 bb = b2[4 * j + t];
    float c[MT][4];
#pragma unroll
    for (int mt = 0; mt < MT; ++mt) {
      c[mt][0] = bb.x; c[mt][1] = bb.y; c[mt][2] = bb.x; c[mt][3] = bb.y;
    }
#pragma unroll
    for (int s = 0; s < KS; ++s) {
      const uint2 f = w2[(j * 4 + s) * 32 + lane];
#pragma unroll
      for (int mt = 0; mt < MT; ++mt) mma_f16_16816(c[mt], a2[mt][s], f);
    }
#pragma unroll
    for (int mt = 0; mt < MT; ++mt) {
      a3[mt][j >> 1][2 * (j & 1) + 0] = silu_half_f16x2(c[mt][0], c[mt][1]);
      a3[mt][j >> 1][2 * (j & 1) + 1] = silu_half_f16x2(c[mt][2], c[mt][3]);
    }
  }
  // output layer: column 0 of the accumulator (lanes t = 0: rows g, g + 8)
  float c[MT][4];
#pragma unroll
  for (int mt = 0; mt < MT; ++mt) c[mt][0] = c[mt][1] = c[mt][2] = c[mt][3] = 0.0f;
#pragma unroll
  for (int s = 0; s < KS; ++s) {
    const uint2 f = w3[s * 32 + lane];
#pragma unroll
    for (int mt = 0; mt < MT; ++mt) mma_f16_16816(c[mt], a3[mt][s], f);
  }
  if (t == 0) {
#pragma unroll
    for (int mt = 0; mt < MT; ++mt) {
      ys[mt * 16 + g] = c[mt][0] + b3;
      ys[mt * 16 + 8 + g] = c[mt][2] + b3;
    }
  }
  __syncwarp();
}

// The network output y for every lane with chk set (0 elsewhere); all 32
// lanes call it together.  Each such lane writes its inputs (f0..f3 and the
// group one-hot from input 4 on, as binary16, zeros to input 31) into row
// `rank` of the warp's tile; the tile then runs through the instantiation for
// the network's width (16, 32 or 64 units, zero-padded), its inputs (K = 16
// or 32) and its rows (one or two M tiles) -- the same choice in every lane.
// One copy, called from both check sites, so the tracker's instruction
// working set stays small.
static __device__ __noinline__ float net_y_warp(const uint32_t *nf, unsigned char *tile,
                                                float f0, float f1, float f2, float f3, int grp,
                                                bool chk, int n_in, int H, float b3) {
  const uint32_t pm = __ballot_sync(0xffffffffu, chk);
  const int rank = __popc(pm & lanemask_lt());
  const int npend = __popc(pm);
  float *ys = reinterpret_cast<float *>(tile + 32 * kNetRowBytes);
  if (chk) {
    uint4 *row = reinterpret_cast<uint4 *>(tile + rank * kNetRowBytes);
    row[0] = make_uint4(pack_f16x2(f0, f1), pack_f16x2(f2, f3), 0u, 0u);
    row[1] = make_uint4(0u, 0u, 0u, 0u);
    row[2] = make_uint4(0u, 0u, 0u, 0u);
    row[3] = make_uint4(0u, 0u, 0u, 0u);
    if (n_in > 3)
      reinterpret_cast<unsigned short *>(tile + rank * kNetRowBytes)[4 + grp] = 0x3C00u;  // 1
  }
  __syncwarp();
  const uint32_t ts = (uint32_t)__cvta_generic_to_shared(tile);
  const int v = (H <= 16 ? 0 : H <= 32 ? 1 : 2) * 4 + (n_in > 16 ? 2 : 0) + (npend > 16 ? 1 : 0);
  switch (v) {
    case 0: net_eval_t<2, false, 1>(nf, ts, ys, b3); break;
    case 1: net_eval_t<2, false, 2>(nf, ts, ys, b3); break;
    case 2: net_eval_t<2, true, 1>(nf, ts, ys, b3); break;
    case 3: net_eval_t<2, true, 2>(nf, ts, ys, b3); break;
    case 4: net_eval_t<4, false, 1>(nf, ts, ys, b3); break;
    case 5: net_eval_t<4, false, 2>(nf, ts, ys, b3); break;
    case 6: net_eval_t<4, true, 1>(nf, ts, ys, b3); break;
    case 7: net_eval_t<4, true, 2>(nf, ts, ys, b3); break;
    case 8: net_eval_t<8, false, 1>(nf, ts, ys, b3); break;
    case 9: net_eval_t<8, false, 2>(nf, ts, ys, b3); break;
    case 10: net_eval_t<8, true, 1>(nf, ts, ys, b3); break;
    default: net_eval_t<8, true, 2>(nf, ts, ys, b3); break;
  }
  return chk ? ys[rank] : 0.0f;
}

// The window lower bound of every lane with chk set, evaluated together: the
// continuous network inputs of its particle in FP32 (position per bounded
// axis, time; the definitions of net_window), the network (net_y_warp) and
// the map of its output to w_L.  All 32 lanes call it; 0 where chk is unset.
// tile: the warp's kNetWarpBytes of shared memory.
template <class PR, int DIM>
__device__ __forceinline__ float net_lower_warp(const DevProblem &P, const uint32_t *nf,
                                                unsigned char *tile, const PartOf<PR> &p,
                                                bool chk) {
  float f[4] = {0.0f, 0.0f, 0.0f, 0.0f};
  if (chk) {
    const int idx[3] = {p.i, p.j, p.k};
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      if (!P.bounded[a] || (DIM == 1 && a > 0)) continue;
      // 2 (x - x_0) / (n dx) - 1 = i (2 / n) + o (2 / (n dx)) - 1 with the
      // offset o in cell i (cell-local), or from the FP64 coordinate
      if constexpr (PR::kLocal) {
        const float off = a == 0 ? p.x : a == 1 ? p.y : p.z;
        f[a] = fmaf((float)idx[a], P.net_cell[a], fmaf(off, P.net_off[a], -1.0f));
      } else {
        const double x = a == 0 ? (double)p.x : a == 1 ? (double)p.y : (double)p.z;
        f[a] = fmaf((float)(x - P.origin[a]), P.net_off[a], -1.0f);
      }
    }
    if (P.ww_net_in > 3 && P.T > 0) {
      // 2 (j + u) / T - 1, u the fraction of bin j passed
      const int j = p.tbin < P.T ? p.tbin : P.T - 1;
      float u;
      if constexpr (PR::kLocal) u = 1.0f - __fdividef((float)p.t, __ldg(P.binw32 + j));
      else u = (float)(((double)p.t - P.edges[j]) / (P.edges[j + 1] - P.edges[j]));
      f[3] = fmaf((float)j + u, 2.0f / (float)P.T, -1.0f);
    }
  }
  const float y = net_y_warp(nf, tile, f[0], f[1], f[2], f[3], chk ? p.g : 0, chk,
                             P.ww_net_in, P.ww_net_h, P.ww_net_b3);
  if (!chk) return 0.0f;
  const float lp = fmaxf(fmaf(y, P.ww_net_scale32, P.ww_net_shift32), P.ww_net_floor32);
  return P.ww_net_wl0_32 * __expf(fminf(lp - P.ww_net_top32, 0.0f));
}

// The window checks of every lane with chk set, together.  Returns false for
// a particle rouletted away.
template <class PR, int DIM>
__device__ __forceinline__ bool net_check_warp(const DevProblem &P, const RunArgs &A,
                                               const EndSink &es, const uint32_t *nf,
                                               unsigned char *tile, PartOf<PR> &p, bool chk,
                                               int *s_novf, PartOf<PR> *ovf) {
  const float wl = net_lower_warp<PR, DIM>(P, nf, tile, p, chk);
  if (!chk) return true;
  return ww_apply<PR, DIM>(P, A, es, p, (typename PR::R)wl, s_novf, ovf);
}

// ---------------------------------------------------------------------------
// The lower bounds the window check applies at given states (position x[3 s],
// time t[s], group g[s]): each state becomes a particle in the mode's own
// representation (cell of the position, clamped into the mesh; offsets from
// the cell's low faces and the time left to the next census edge in the
// cell-local mode) and goes through the kernels' own evaluation -- FP64 one
// at a time (net_window), FP32 a warp of 32 at a time (net_lower_warp, the
// fragment block and the warps' tiles in dynamic shared memory).  A group
// outside 0..G-1 gives NaN.
template <class PR, int DIM>
__global__ void __launch_bounds__(256) k_net_lower(const DevProblem P, const double *__restrict__ x,
                                                   const double *__restrict__ t,
                                                   const int32_t *__restrict__ g, long long n,
                                                   double *__restrict__ out) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int lane = threadIdx.x & 31;
  if constexpr (!PR::kF64) {
    for (int q = threadIdx.x; q < kNetFragWords / 4; q += blockDim.x)
      reinterpret_cast<uint4 *>(smem)[q] = __ldg(reinterpret_cast<const uint4 *>(P.ww_netfrag) + q);
    __syncthreads();
  }
  const long long warps = (long long)gridDim.x * (blockDim.x >> 5);
  for (long long base = ((long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5)) * 32;
       base < n; base += warps * 32) {
    const long long s = base + lane;
    bool ok = s < n;
    PartOf<PR> p{};
    if (ok) {
      const double pos[3] = {x[3 * s], x[3 * s + 1], x[3 * s + 2]};
      int idx[3] = {0, 0, 0};
      for (int a = 0; a < 3; ++a)
        if (P.bounded[a] && (DIM == 3 || a == 0))
          idx[a] = min(max((int)floor((pos[a] - P.origin[a]) / P.width[a]), 0), P.n[a] - 1);
      p.i = idx[0]; p.j = idx[1]; p.k = idx[2];
      const double ts = t[s];
      int j = 0;
      if (P.T > 0) {
        while (j + 1 < P.T && P.edges[j + 1] <= ts) ++j;
      }
      p.tbin = j;
      p.g = g[s];
      ok = p.g >= 0 && p.g < P.G;
      if constexpr (PR::kLocal) {
        const double off[3] = {P.bounded[0] ? pos[0] - P.faces[0][idx[0]] : 0.0,
                               (DIM == 3 && P.bounded[1]) ? pos[1] - P.faces[1][idx[1]] : 0.0,
                               (DIM == 3 && P.bounded[2]) ? pos[2] - P.faces[2][idx[2]] : 0.0};
        p.x = (float)off[0]; p.y = (float)off[1]; p.z = (float)off[2];
        p.t = P.T > 0 ? (float)(P.edges[j + 1] - ts) : 0.0f;
      } else {
        p.x = pos[0]; p.y = pos[1]; p.z = pos[2];
        p.t = ts;
      }
      if (!ok) out[s] = CUDART_NAN;
    }
    if constexpr (PR::kF64) {
      if (ok) out[s] = net_window<PR, DIM>(P, p);
    } else {
      const float wl = net_lower_warp<PR, DIM>(P, reinterpret_cast<const uint32_t *>(smem),
                                               smem + kNetFragBytes + (threadIdx.x >> 5) * kNetWarpBytes,
                                               p, ok);
      if (ok) out[s] = (double)wl;
    }
  }
}

// ---------------------------------------------------------------------------
// Persistent tracker.  Each lane flies one particle held in registers; the
// flights of a warp are one dense pass over its 32 lanes.  A flight that
// ends in a collision parks its particle in the warp's pool; once 32 are
// parked (or nothing else can progress) they are collided in one dense pass
// and marked ready; empty lanes take ready particles; when none are left,
// a dense pass of up to 32 births (split children first, then new source
// histories) refills the pool.  Occupancy bound: births happen only when no
// particle is ready and some lane is empty, so the warp never holds more
// than 31 + 31 + 32 particles and at least 33 slots are free before every
// flight pass -- room for every lane to park a collision.
//
// Shared mode: the CTA works on one batch at a time with its private
// shared-memory tally; warps claim the batch's histories through a shared
// cursor and meet at a CTA barrier only when the batch is drained, where the
// private tally is folded into the batch sums.  Global mode: warps claim
// histories of the launch's batch from a device-wide cursor and score into
// the device-wide batch tally.
// batched problems: CTAs claim (problem, history range) work items
struct WorkItem {
  int32_t p;
  int32_t pad;
  unsigned long long h0, h1;   // histories [h0, h1) of problem p
};
struct MultiArgs {
  const DevProblem *probs;
  const RunArgs *args;
  const WorkItem *items;
  int32_t n_items;
  unsigned long long *counter;
};

// PC: the population-control instantiation (global tally, one problem): census
// banking, the step tally, staged births and reserved input claims exist only
// there, so the other kernels carry none of their code.
// VR: particle weights vary (a window table is set, or implicit capture is
// on) -- the instantiation that carries the window checks (split, roulette,
// children) and implicit capture, which analog kernels leave out.
template <class PR, bool SHARED, int DIM, bool MULTI, bool NET = false, bool PC = false,
          bool VR = false>
__global__ void __launch_bounds__(NET ? kNetBlockMax : 512) k_track(const DevProblem Pin, const RunArgs Ain, const Layout L,
                                               const MultiArgs MA) {
  using R = typename PR::R;
  using TT = typename PR::TT;
  extern __shared__ __align__(16) unsigned char smem[];
  const int tid = threadIdx.x, nth = blockDim.x;
  const int lane = tid & 31, warp = tid >> 5, nwarps = nth >> 5;
  const int S = L.S;
  __shared__ DevProblem sP;      // batched problems: the current problem
  __shared__ RunArgs sA;
  __shared__ int s_cur_p;
  const DevProblem &P = MULTI ? sP : Pin;
  const RunArgs &A = MULTI ? sA : Ain;
  // population-control step tally: from the launch's own arguments (batched
  // launches fill sA only when a CTA claims an item, and never use it)
  const bool step_tally = PC && Ain.step_tally != 0;
  const int step_bins = step_tally ? Ain.step_bins : 0;
  const bool prefetch = PC && Ain.prefetch != 0 && Ain.spill_in != nullptr;
  // input positions matter to population control alone (global tally, single problem)
  const bool use_slot = PC && Ain.census_out != nullptr;
  // split children (warp stacks, spill banks) exist only where weights vary;
  // spilled or combed particles come in only there and under population control
  constexpr bool kChildren = VR || NET;
  constexpr bool kSpillIn = VR || NET || PC;

  // ---- carve shared memory
  unsigned char *ptr = smem;
  Tables<R> tb;
  {
    const int M = L.M, G = L.G;
    tb.sigma_t = (R *)ptr; ptr += align16((long long)sizeof(R) * M * G);
    tb.scat = (R *)ptr; ptr += align16((long long)sizeof(R) * M * G);
    tb.cdf = (R *)ptr; ptr += align16((long long)sizeof(R) * M * G * G);
    tb.src_cdf = (R *)ptr; ptr += align16((long long)sizeof(R) * G);
    tb.speed = (double *)ptr; ptr += align16(8ll * G);
    tb.inv_speed = (R *)ptr; ptr += align16((long long)sizeof(R) * G);
    tb.speed32 = (float *)ptr; ptr += align16(4ll * G);
    tb.edges = (double *)ptr; ptr += align16(8ll * (L.T + 1));
  }
  TT *stally = nullptr;
  if (SHARED || step_tally) { stally = (TT *)ptr; ptr += L.tally_bytes; }
  const Bank<PR> bk = bank_view<PR>(ptr, S, DIM);
  ptr += (long long)S * slot_bytes(PR::kF64, DIM, PR::kLocal);
  // FP32 network kernels: the fragment block after the bank (where the staged
  // births would go: population control never runs with windows)
  const uint32_t *nf = reinterpret_cast<const uint32_t *>(ptr);
  unsigned char *ntile = ptr + kNetFragBytes + (tid >> 5) * kNetWarpBytes;
  if constexpr (NET && !PR::kF64) {
    if (Pin.ww_netfrag != nullptr)
      for (int q = tid; q < kNetFragWords / 4; q += nth)
        reinterpret_cast<uint4 *>(ptr)[q] = __ldg(reinterpret_cast<const uint4 *>(Pin.ww_netfrag) + q);
  }
  // staged births (prefetch): 32 slots per warp in the pool layout
  const Bank<PR> stage =
      bank_view<PR>(ptr + (prefetch ? (long long)(tid >> 5) * 32 * slot_bytes(PR::kF64, DIM, PR::kLocal) : 0),
                    32, DIM);
  __shared__ uint64_t s_pf_bar[16];            // one mbarrier per warp
  __shared__ unsigned long long s_pf_first[16];
  __shared__ int s_pf_got[16], s_pf_phase[16], s_pf_lost[16];
  // population control: each warp's reservation [next, end) of input positions;
  // the particles in this launch's input bank (fixed while it runs: written by
  // the comb or the previous pass), read once instead of at every claim
  __shared__ unsigned long long s_res_next[16], s_res_end[16], s_in_total;

  __shared__ unsigned long long s_h_next, s_h_end;
  __shared__ int s_done, s_batch;
  __shared__ int s_novf[48];     // [w]: warp w's stack of children; [16 + w]: children it may
                                 // still make; [32 + w]: its stack limit for new children
  __shared__ double s_w[4];
  __shared__ uint32_t s_n[9];
  __shared__ double s_red[32];   // per-warp region sums (two estimators)

  // ---- tables of the current problem into shared memory
  auto load_tables = [&]() {
    const int M = P.M, G = P.G;
    tb.ww = P.ww_lower;
    tb.ww32 = P.ww_lower32;
    for (int q = tid; q < M * G; q += nth) {
      if constexpr (PR::kF64) { tb.sigma_t[q] = P.sigma_t[q]; tb.scat[q] = P.scat[q]; }
      else { tb.sigma_t[q] = P.sigma_t32[q]; tb.scat[q] = P.scat32[q]; }
    }
    for (int q = tid; q < M * G * G; q += nth) {
      if constexpr (PR::kF64) tb.cdf[q] = P.cdf[q]; else tb.cdf[q] = P.cdf32[q];
    }
    for (int q = tid; q < G; q += nth) {
      if constexpr (PR::kF64) { tb.src_cdf[q] = P.src_cdf[q]; tb.inv_speed[q] = 1.0 / P.speed[q]; }
      else { tb.src_cdf[q] = P.src_cdf32[q]; tb.inv_speed[q] = P.inv_speed32[q]; }
      tb.speed[q] = P.speed[q];
      tb.speed32[q] = P.speed32[q];
    }
    for (int q = tid; q <= P.T; q += nth) tb.edges[q] = P.edges[q];
  };
  if (!MULTI) load_tables();
  if (SHARED)
    for (long long q = tid; q < P.n_tally; q += nth) stally[q] = (TT)0;
  for (int q = tid; q < step_bins; q += nth) stally[q] = (TT)0;
  if (tid < 32) s_novf[tid] = 0;
  if (tid < 16) s_novf[32 + tid] = Ain.overflow_cap;
  if (tid < 4) s_w[tid] = 0.0;
  if (tid < 9) s_n[tid] = 0u;
  if (tid == 0) {
    s_done = 0; s_batch = -1; s_h_next = s_h_end = 0; s_cur_p = -1;
    s_in_total = (!MULTI && Ain.spill_in != nullptr) ? min(*Ain.spill_in_count, Ain.spill_cap) : 0ull;
  }
  if (prefetch && (tid & 31) == 0) {
    tc::mbar_init(&s_pf_bar[tid >> 5], 1);
    s_pf_got[tid >> 5] = 0;
    s_res_next[tid >> 5] = s_res_end[tid >> 5] = 0;
    s_pf_phase[tid >> 5] = 0;
    s_pf_lost[tid >> 5] = -1;
  }
  if (prefetch) tc::fence_async_smem();
  __syncthreads();

  EndSink es{s_w, s_n};
  LocalCount lc{0, 0, 0, 0};
  const int wid = blockIdx.x * nwarps + warp;                 // warp id in the grid
  // the warp's stack of split children (batched launches: one stack per warp
  // for every problem it serves; none when no problem has windows)
  PartOf<PR> *ovf =
      MULTI ? (Ain.overflow == nullptr
                   ? nullptr
                   : reinterpret_cast<PartOf<PR> *>(Ain.overflow) + (size_t)wid * Ain.overflow_cap)
            : reinterpret_cast<PartOf<PR> *>(A.overflow) + (size_t)wid * A.overflow_cap;
  int *novf = &s_novf[warp];
  const int pool0 = warp * kPool;                              // first slot of this warp
  bool agg = MULTI ? false : A.warp_aggregate != 0;

  uint64_t g_h0 = 0, g_h1 = 0;
  if (!SHARED && !MULTI) {
    g_h0 = A.tally_per_batch ? 0 : batch_start(A.n_hist, A.n_batches, A.batch);
    g_h1 = A.tally_per_batch ? A.n_hist : batch_start(A.n_hist, A.n_batches, A.batch + 1);
  }

  for (;;) {
    if (MULTI) {
      // ---- claim the next work item; switch problem when it changes
      if (tid == 0) {
        const unsigned long long it = atomicAdd(MA.counter, 1ull);
        if ((long long)it < MA.n_items) {
          const WorkItem w = MA.items[it];
          s_batch = w.p;
          s_h_next = w.h0;
          s_h_end = w.h1;
        } else {
          s_done = 1;
        }
      }
      __syncthreads();
      if (s_done) break;
      if (s_batch != s_cur_p) {
        if (tid == 0) { sP = MA.probs[s_batch]; sA = MA.args[s_batch]; s_cur_p = s_batch; }
        __syncthreads();
        load_tables();
        agg = A.warp_aggregate != 0;
        __syncthreads();
      }
    } else if (SHARED) {
      // ---- claim the next batch for the whole CTA
      if (tid == 0) {
        const unsigned long long b = atomicAdd(A.work, 1ull);
        if ((long long)b < A.n_batches) {
          s_batch = (int)b;
          s_h_next = batch_start(A.n_hist, A.n_batches, (int)b);
          s_h_end = batch_start(A.n_hist, A.n_batches, (int)b + 1);
        } else {
          s_done = 1;
        }
      }
      __syncthreads();
      if (s_done) break;
    }

    // ---- warp loop over this batch (shared) or the launch (global).  The
    // warp's kPool slots hold two stacks: particles ready to fly grow up from
    // slot 0 (rtop of them), particles waiting for their collision grow down
    // from the last slot (ctop of them).  At most 94 particles are ever
    // parked (see above), so the stacks never meet.
    PartOf<PR> p;
    bool has = false;
    int rtop = 0, ctop = 0;          // identical in every lane
    bool exhausted = false;
    const uint32_t lt = lanemask_lt();
    auto slot_of = [&](int s) {
      (void)MCDC_CHK(A.error, CHK_POOL, s >= 0 && s < kPool, s);
      return pool0 + min(max(s, 0), kPool - 1);
    };
#ifdef MCDC_CHECKS
    // entries of the tally a scatter indexes: the step tally, the CTA's
    // shared tally, or the global tally (one slice per batch when per batch)
    auto tally_extent = [&](bool step) -> long long {
      if (step) return step_bins;
      if (SHARED) return P.n_tally;
      return (A.tally_per_batch ? (long long)A.n_batches : 1ll) * P.n_tally;
    };
#endif
    // population control (lane 0): the first of the next 32 input positions,
    // from the warp's reservation, which one atomic refills kReserve at a
    // time (a claim per 32 would hold the warp for an atomic's round trip
    // every ~3 flights); 32-aligned, so a claim never straddles two
    // reservations, and a short claim still means the input is used up
    auto claim32 = [&]() -> unsigned long long {
      unsigned long long nx = s_res_next[warp];
      if (nx >= s_res_end[warp]) {
        nx = atomicAdd(A.spill_in_cursor, (unsigned long long)kReserve);
        s_res_end[warp] = nx + kReserve;
      }
      s_res_next[warp] = nx + 32ull;
      return nx;
    };
    for (;;) {
      __syncwarp();   // every lane sees the same overflow count below
      // (1) collisions: a dense pass when 32 are parked, or whatever is
      // parked once nothing is ready and no more births can come
      {
        const bool drain = exhausted && (*novf == 0) && !(prefetch && s_pf_got[warp] > 0);
        if (ctop >= 32 || (ctop > 0 && rtop == 0 && drain)) {
          const int n = min(ctop, 32);
          const bool mine = lane < n;
          PartOf<PR> q;
          if (mine) bk.load(slot_of(kPool - ctop + lane), q, DIM, use_slot);
          __syncwarp();   // every parked particle is read before survivors are written
          ctop -= n;
          bool alive = false;
          int cbin = -1;
          R cscore = (R)0;
          double wabs = 0.0;
          bool ww_pend = false;
          if (mine) {
            int end = END_NONE;
            alive = collide<PR, DIM, NET, PC, VR>(P, tb, A, es, q, end, lc, novf, ovf, cbin,
                                                  cscore, wabs, ww_pend);
            if (!alive) finish<PR, DIM>(P, A, es, q, end);
          }
          if (P.estimator != 0) {
            // combined estimator: the collision tally follows the track-length one
            const long long coff = P.estimator == 2 ? P.n_bins : 0;
            if (step_tally)
              tally_scatter<TT, R>(stally, A.tally, A.tally32, true, agg, mine,
                                   (mine && cbin >= 0) ? step_bin(P, A, q.hid, cbin, P.estimator == 2)
                                                       : -1, cscore, 0, A.error,
                                   MCDC_CHECKED_ONLY(tally_extent(true)));
            else
              tally_scatter<TT, R>(stally, A.tally, A.tally32, SHARED, agg, mine,
                                   (SHARED && mine) ? cbin + (int)coff : cbin, cscore,
                                   mine ? tally_offset(P, A, q.hid) + (SHARED ? 0 : coff) : 0,
                                   A.error, MCDC_CHECKED_ONLY(tally_extent(false)));
          }
          if ((VR || NET || PC) && P.implicit) {
            // weight removed by implicit capture: one shared add per warp
            for (int o = 16; o > 0; o >>= 1) wabs += __shfl_xor_sync(0xffffffffu, wabs, o);
            if (lane == 0) atomicAdd(&s_w[1], wabs);
          }
          if constexpr (NET && !PR::kF64) {
            // the pass's post-collision window checks, together
            const bool chk = alive && ww_pend;
            if (__any_sync(0xffffffffu, chk)) {
              const bool ok = net_check_warp<PR, DIM>(P, A, es, nf, ntile, q, chk, novf, ovf);
              if (!ok) { finish<PR, DIM>(P, A, es, q, END_ROULETTE); alive = false; }
            }
          }
          const uint32_t am = __ballot_sync(0xffffffffu, alive);
          if (alive) bk.store(slot_of(rtop + __popc(am & lt)), q, DIM, use_slot);
          rtop += __popc(am);
          __syncwarp();
        }
      }
      // (2) empty lanes take ready particles from the top of the stack
      {
        const uint32_t empty = __ballot_sync(0xffffffffu, !has);
        if (empty && rtop) {
          const int r = __popc(empty & lt);
          const bool take = !has && r < rtop;
          if (take) { bk.load(slot_of(rtop - 1 - r), p, DIM, use_slot); has = true; }
          rtop -= min(rtop, __popc(empty));
          __syncwarp();
        }
      }
      // (3) births when lanes are still empty and nothing is ready
      const bool staged_ready = prefetch && s_pf_got[warp] > 0;
      if (__any_sync(0xffffffffu, !has) && rtop == 0 &&
          !(exhausted && *novf == 0 && !staged_ready)) {
        const int n_o = kChildren ? min(32, min(*novf, A.overflow_cap)) : 0;
        int n_s = 0;
        unsigned long long h_first = 0;
        bool staged = false;
        if (n_o == 0 && staged_ready) {
          // the chunk staged during the last round: wait for its copies
          const bool done =
              __all_sync(0xffffffffu, tc::mbar_wait(&s_pf_bar[warp], (uint32_t)s_pf_phase[warp], 1 << 26));
          if (!done) {
            if (lane == 0) {
              atomicOr(A.error, ERRBIT_TIMEOUT);
              s_pf_lost[warp] = s_pf_phase[warp];   // waited for once more before exit
            }
            exhausted = true;                   // its particles are lost: the run reports it
          } else {
            staged = true;
            h_first = s_pf_first[warp];
            n_s = s_pf_got[warp];
          }
          __syncwarp();
          if (lane == 0) { s_pf_phase[warp] ^= 1; s_pf_got[warp] = 0; }
          __syncwarp();
        } else if (n_o < 32 && !exhausted) {
          const int want = 32 - n_o;
          unsigned long long first = 0;
          int got = 0;
          if (lane == 0) {
            if (kSpillIn && A.spill_in != nullptr && !MULTI) {
              const unsigned long long total = s_in_total;
              first = (prefetch && want == 32) ? claim32()
                                               : atomicAdd(A.spill_in_cursor, (unsigned long long)want);
              got = first < total ? (int)min((unsigned long long)want, total - first) : 0;
            } else if (SHARED || MULTI) {
              first = atomicAdd(&s_h_next, (unsigned long long)want);
              got = first < s_h_end ? (int)min((unsigned long long)want, s_h_end - first) : 0;
            } else {
              const unsigned long long c = atomicAdd(A.work, (unsigned long long)want);
              first = g_h0 + c;
              got = first < g_h1 ? (int)min((unsigned long long)want, g_h1 - first) : 0;
            }
          }
          first = __shfl_sync(0xffffffffu, first, 0);
          got = __shfl_sync(0xffffffffu, got, 0);
          h_first = first;
          n_s = got;
          if (got < want) {
            exhausted = true;
            // the warp's own particles are used up: with the device-wide banks,
            // children beyond a small stack go there and are shared by every
            // warp in the next pass, instead of one warp working through a
            // large family while the others have finished
            if (!SHARED && !MULTI && lane == 0 && A.spill_out != nullptr && A.overflow_tail >= 0)
              novf[32] = min(A.overflow_cap, A.overflow_tail);
          }
        }
        const int nb = n_o + n_s;
        const int top = min(*novf, A.overflow_cap);
        bool alive = false;
        PartOf<PR> q;
        if (lane < nb) {
          if (lane < n_o) {
            if (MCDC_CHK(A.error, CHK_STACK,
                         top - 1 - lane >= 0 &&
                             top - 1 - lane < (MULTI ? Ain.overflow_cap : A.overflow_cap),
                         top - 1 - lane)) {
              q = ovf[top - 1 - lane];
              alive = true;
            }
          } else if (kSpillIn && A.spill_in != nullptr && !MULTI) {
            const long long at = (long long)h_first + (lane - n_o);
            const bool in_ok =
                MCDC_CHK(A.error, CHK_SPILL_IN, at >= 0 && (unsigned long long)at < s_in_total, at);
            if (!in_ok) {
              // not read: the particle is lost and the run reports the check
            } else if (staged)               // staged by the bulk copies
              stage.load(lane, q, DIM);
            else if (PC && A.census_out != nullptr)     // population control: the combed bank (pool layout)
              bank_view<PR>(const_cast<void *>(A.spill_in), (long long)A.spill_cap, DIM)
                  .load((int)at, q, DIM);
            else
              q = reinterpret_cast<const PartOf<PR> *>(A.spill_in)[at];
            if (use_slot) q.slot = (uint32_t)at;             // position in the step's input
            alive = in_ok;
          } else {
            source_particle<PR, DIM>(P, tb, A.rk, A.offset + h_first + (lane - n_o), q);
            if (use_slot) q.slot = (uint32_t)(h_first + (lane - n_o));   // history's position in the run
            if (weights_summed(P)) atomicAdd(&s_w[0], 1.0);
            atomicAdd(&s_n[7], 1u);
            alive = !(P.T > 0 && q.tbin >= P.T);
            if (!alive) finish<PR, DIM>(P, A, es, q, END_CENSUSED);
          }
        }
        // the newborns go straight to the empty lanes; any left over are parked
        const uint32_t am = __ballot_sync(0xffffffffu, alive);
        const uint32_t empty = __ballot_sync(0xffffffffu, !has);
        const int na = __popc(am), ne = __popc(empty);
        const int k = __popc(am & lt);                 // rank of my newborn
        const int r = __popc(empty & lt);              // rank of my empty lane
        if (alive && k >= ne) bk.store(slot_of(k - ne), q, DIM, use_slot);
        __syncwarp();
        if (kChildren && lane == 0) *novf = min(*novf, A.overflow_cap) - n_o;
        // lane with the r-th empty slot receives the r-th newborn (a shuffle per field)
        const int src = (r < na) ? (int)nth32(am, r) : 0;
        PartOf<PR> got;
        got.x = __shfl_sync(0xffffffffu, q.x, src);
        got.y = __shfl_sync(0xffffffffu, q.y, src);
        got.z = __shfl_sync(0xffffffffu, q.z, src);
        got.t = __shfl_sync(0xffffffffu, q.t, src);
        got.ux = __shfl_sync(0xffffffffu, q.ux, src);
        got.uy = __shfl_sync(0xffffffffu, q.uy, src);
        got.uz = __shfl_sync(0xffffffffu, q.uz, src);
        got.w = __shfl_sync(0xffffffffu, q.w, src);
        got.g = __shfl_sync(0xffffffffu, q.g, src);
        got.i = __shfl_sync(0xffffffffu, q.i, src);
        got.j = __shfl_sync(0xffffffffu, q.j, src);
        got.k = __shfl_sync(0xffffffffu, q.k, src);
        got.tbin = __shfl_sync(0xffffffffu, q.tbin, src);
        got.ctr = __shfl_sync(0xffffffffu, q.ctr, src);
        got.serial = __shfl_sync(0xffffffffu, q.serial, src);
        got.hid = __shfl_sync(0xffffffffu, q.hid, src);
        got.nseg = __shfl_sync(0xffffffffu, q.nseg, src);
        got.ncol = __shfl_sync(0xffffffffu, q.ncol, src);
        got.ncross = __shfl_sync(0xffffffffu, q.ncross, src);
        got.slot = use_slot ? __shfl_sync(0xffffffffu, q.slot, src) : 0u;
        if constexpr (!PR::kF64) got.tau = __shfl_sync(0xffffffffu, q.tau, src);
        else got.tau = -1.0f;
        if (!has && r < na) { p = got; has = true; }
        rtop = max(0, na - ne);
        __syncwarp();
        // prefetch: claim the next 32 input positions and stage them with one
        // bulk copy per field array while the newborns fly (every lane has
        // read its staged slot by now; the fence orders those reads before
        // the copies' writes)
        if (prefetch && !exhausted && s_pf_got[warp] == 0) {
          int ng = 0;
          if (lane == 0) {
            const unsigned long long total = s_in_total;
            const unsigned long long nf = claim32();
            ng = nf < total ? (int)min(32ull, total - nf) : 0;
            if (ng > 0) {
              const Bank<PR> src =
                  bank_view<PR>(const_cast<void *>(A.spill_in), (long long)A.spill_cap, DIM);
              const uint32_t bytes = (uint32_t)ng * 16u;
              constexpr int arrays = 5 + ((DIM == 3 && !PR::kLocal) ? 1 : 0) + (PR::kF64 ? 1 : 0);
              uint64_t *bar = &s_pf_bar[warp];
              tc::fence_async_smem();
              tc::mbar_expect_tx(bar, bytes * arrays);
              tc::bulk_g2s(stage.xt, static_cast<const uint4 *>(src.xt) + nf, bytes, bar);
              if (DIM == 3 && !PR::kLocal) tc::bulk_g2s(stage.yz, src.yz + nf, bytes, bar);
              tc::bulk_g2s(stage.d0, static_cast<const uint4 *>(src.d0) + nf, bytes, bar);
              if constexpr (PR::kF64) tc::bulk_g2s(stage.d1, src.d1 + nf, bytes, bar);
              tc::bulk_g2s(stage.ids, src.ids + nf, bytes, bar);
              tc::bulk_g2s(stage.cell, src.cell + nf, bytes, bar);
              tc::bulk_g2s(stage.cnt, src.cnt + nf, bytes, bar);
              s_pf_first[warp] = nf;
              s_pf_got[warp] = ng;
            }
          }
          ng = __shfl_sync(0xffffffffu, ng, 0);
          if (ng < 32) exhausted = true;
          __syncwarp();
        }
      }
      // (4) nothing in flight: progress through collisions/births, or stop
      if (!__any_sync(0xffffffffu, has)) {
        if (ctop == 0 && rtop == 0 && exhausted && *novf == 0 &&
            !(prefetch && s_pf_got[warp] > 0))
          break;
        continue;
      }
      // (5) one flight for every lane that holds a particle
      {
        int outcome = OUT_CONT, end = END_NONE;
        int bin = -1;
        R score = (R)0;
        const bool flew = has;
        if (has) {
          outcome = flight<PR, DIM, NET, PC, VR>(P, tb, A, es, p, bin, score, end, lc, novf, ovf);
          if (outcome == OUT_DEAD) { finish<PR, DIM>(P, A, es, p, end); has = false; }
        }
        if (step_tally)
          tally_scatter<TT, R>(stally, A.tally, A.tally32, true, agg, flew,
                               (flew && bin >= 0) ? step_bin(P, A, p.hid, bin, 0) : -1, score, 0,
                               A.error, MCDC_CHECKED_ONLY(tally_extent(true)));
        else
          tally_scatter<TT, R>(stally, A.tally, A.tally32, SHARED, agg, flew, bin, score,
                               flew ? tally_offset(P, A, p.hid) : 0, A.error,
                               MCDC_CHECKED_ONLY(tally_extent(false)));
        if constexpr (NET && !PR::kF64) {
          // the pass's crossing window checks, together
          const bool chk = has && outcome == OUT_WW;
          if (__any_sync(0xffffffffu, chk)) {
            const bool ok = net_check_warp<PR, DIM>(P, A, es, nf, ntile, p, chk, novf, ovf);
            if (!ok) { finish<PR, DIM>(P, A, es, p, END_ROULETTE); has = false; }
          }
        }
        if (PC && A.census_out != nullptr) {
          // population control: a banked particle goes to its input position
          // (no splitting here, so every input yields at most one), which
          // keeps the bank in the order the step ran its particles
          const bool bank = has && outcome == OUT_BANKED;
          const uint32_t bm = __ballot_sync(0xffffffffu, bank);
          if (bm) {
            if (lane == 0) atomicAdd(A.census_count, (unsigned long long)__popc(bm));
            if (bank) {
              if (p.slot < A.census_cap) {
                bank_view<PR>(A.census_out, (long long)A.census_cap, DIM).store((int)p.slot, p, DIM);
                A.census_w[p.slot] = (double)p.w;
              } else {
                atomicOr(A.error, ERRBIT_OVERFLOW);
              }
              has = false;
            }
          }
        }
        const bool park = has && outcome == OUT_COLL;
        const uint32_t pm = __ballot_sync(0xffffffffu, park);
        if (pm) {
          if (park) { bk.store(slot_of(kPool - ctop - 1 - __popc(pm & lt)), p, DIM, use_slot); has = false; }
          ctop += __popc(pm);
          __syncwarp();
        }
      }
    }

    if (MULTI) { __syncthreads(); continue; }   // the item is drained in every warp
    if (!SHARED) break;
    // ---- the batch is drained in every warp: fold the private tally
    // (combined estimator: both halves, their product and both region sums)
    __syncthreads();
    double rsum = 0.0, rsum_c = 0.0;
    const long long per_cell = (long long)P.G * P.T1;
    const bool comb = P.estimator == 2;
    for (long long q = tid; q < P.n_bins; q += nth) {
      const double v = (double)stally[q];
      const double vc = comb ? (double)stally[P.n_bins + q] : 0.0;
      if (v != 0.0 || vc != 0.0) {
        atomicAdd(&A.sum1[q], v);
        atomicAdd(&A.sum2[q], v * v);
        if (comb) {
          atomicAdd(&A.sum1[P.n_bins + q], vc);
          atomicAdd(&A.sum2[P.n_bins + q], vc * vc);
          atomicAdd(&A.sum12[q], v * vc);
          stally[P.n_bins + q] = (TT)0;
        }
        const int cell = (int)(q / per_cell);
        const int ci = cell % P.n[0];
        const int cj = (cell / P.n[0]) % P.n[1];
        const int ck = cell / (P.n[0] * P.n[1]);
        if (ci >= P.region_lo[0] && ci < P.region_hi[0] && cj >= P.region_lo[1] &&
            cj < P.region_hi[1] && ck >= P.region_lo[2] && ck < P.region_hi[2]) {
          rsum += v;
          rsum_c += vc;
        }
        stally[q] = (TT)0;
      }
    }
    for (int o = 16; o > 0; o >>= 1) {
      rsum += __shfl_xor_sync(0xffffffffu, rsum, o);
      rsum_c += __shfl_xor_sync(0xffffffffu, rsum_c, o);
    }
    if (lane == 0) { s_red[warp] = rsum; s_red[nwarps + warp] = rsum_c; }
    __syncthreads();
    if (tid == 0) {
      double tot = 0.0, tot_c = 0.0;
      for (int w = 0; w < nwarps; ++w) { tot += s_red[w]; tot_c += s_red[nwarps + w]; }
      atomicAdd(&A.region[0], tot);
      atomicAdd(&A.region[1], tot * tot);
      if (comb) {
        atomicAdd(&A.region[2], tot_c);
        atomicAdd(&A.region[3], tot_c * tot_c);
        atomicAdd(&A.region[4], tot * tot_c);
      }
    }
    __syncthreads();
  }

  // a staged chunk whose wait ran out: give its copies one more bounded wait
  // so none is in flight when the CTA exits
  if (prefetch && lane == 0 && s_pf_lost[warp] >= 0)
    tc::mbar_wait(&s_pf_bar[warp], (uint32_t)s_pf_lost[warp], 1 << 26);

  // ---- population-control step tally: add the CTA's entries into the
  // per-batch slices of the global tally (time bin step_tbin)
  if (step_tally) {
    __syncthreads();
    const int per = (int)(P.n_cells * P.G);
    for (int q = tid; q < step_bins; q += nth) {
      const double v = (double)stally[q];
      if (v == 0.0) continue;
      const int cg = q % per, eb = q / per;
      const int b = eb % A.n_batches, e = eb / A.n_batches;
      const long long at = (long long)b * P.n_tally + e * P.n_bins + (long long)cg * P.T1 +
                           A.step_tbin;
      if (A.tally32 != nullptr) atomicAdd(&A.tally32[at], (float)v);
      else atomicAdd(&A.tally[at], v);
    }
  }

  // ---- flush event counters: warp sums, one atomic per field per warp.
  // (Batched problems share one stats block and error word; a CTA that never
  // claimed an item must not read its per-problem arguments.)
  Stats *const stats = MULTI ? MA.args[0].stats : A.stats;
  int32_t *const errw = MULTI ? MA.args[0].error : A.error;
  const int ovf_cap = MULTI ? Ain.overflow_cap : A.overflow_cap;
  uint32_t c4[4] = {lc.seg, lc.col, lc.cross, lc.census};
#pragma unroll
  for (int f = 0; f < 4; ++f)
    for (int o = 16; o > 0; o >>= 1) c4[f] += __shfl_xor_sync(0xffffffffu, c4[f], o);
  if (lane == 0) {
    atomicAdd(&stats->segments, (unsigned long long)c4[0]);
    atomicAdd(&stats->collisions, (unsigned long long)c4[1]);
    atomicAdd(&stats->crossings, (unsigned long long)c4[2]);
    atomicAdd(&stats->census, (unsigned long long)c4[3]);
    if (*novf > ovf_cap) atomicOr(errw, ERRBIT_OVERFLOW);
  }
  __syncthreads();
  if (tid == 0) {
    atomicAdd(&stats->absorbed, (unsigned long long)s_n[0]);
    atomicAdd(&stats->leaked, (unsigned long long)s_n[1]);
    atomicAdd(&stats->censused, (unsigned long long)s_n[2]);
    atomicAdd(&stats->roulette_killed, (unsigned long long)s_n[3]);
    atomicAdd(&stats->roulette_survived, (unsigned long long)s_n[4]);
    atomicAdd(&stats->splits, (unsigned long long)s_n[5]);
    atomicAdd(&stats->children, (unsigned long long)s_n[6]);
    atomicAdd(&stats->histories, (unsigned long long)s_n[7]);
    atomicAdd(&stats->splits_dropped, (unsigned long long)s_n[8]);
    atomicAdd(&stats->w_source, s_w[0]);
    atomicAdd(&stats->w_absorbed, s_w[1]);
    atomicAdd(&stats->w_leaked, s_w[2]);
    atomicAdd(&stats->w_censused, s_w[3]);
  }
}

}  // namespace mcdc
