// tracker.cuh -- persistent, event-based particle tracker.
//
// Each CTA owns a bank of S particle slots (SoA, shared memory) and loops:
//   refill   free slots <- split children (CTA-private overflow stack), then
//            new source particles of its current work item;
//   flight   every live particle takes one flight: distance to collision,
//            mesh surface and time census, move, track-length tally; surface
//            and census events are resolved in place; particles that reach a
//            collision are queued;
//   collide  the queued particles (now a dense list) absorb or scatter.
// Queues are built with a warp ballot + popc prefix and one shared atomic
// per warp, so every phase runs over a compacted list ("sort by event").
// Cross-section tables sit in shared memory.  The tally is either a
// CTA-private copy in shared memory holding one batch at a time (shared
// mode) or a device-wide batch tally (global mode), both fed through
// warp-aggregated atomics.
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

namespace mcdc {

struct PrecF64 {
  using R = double;    // direction, distance, cross sections
  using TT = double;   // shared-memory tally
  static constexpr bool kF64 = true;
};
struct PrecF32 {
  using R = float;
  using TT = float;
  static constexpr bool kF64 = false;
};

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
  double *edges;             // [T+1]
  const double *ww;          // global
  const float *ww32;
};

// SoA particle bank in shared memory
template <class R>
struct Bank {
  double *x, *y, *z, *t;
  uint64_t *hid;
  R *ux, *uy, *uz, *w;
  uint32_t *ctr, *serial, *nseg, *ncol, *ncross;
  uint16_t *i, *j, *k, *tbin;
  uint8_t *g;

  __device__ __forceinline__ void load(int s, Part<R> &p, int dim) const {
    p.x = x[s]; p.t = t[s];
    if (dim == 3) { p.y = y[s]; p.z = z[s]; } else { p.y = 0.0; p.z = 0.0; }
    p.hid = hid[s];
    p.ux = ux[s]; p.uy = uy[s]; p.uz = uz[s]; p.w = w[s];
    p.ctr = ctr[s]; p.serial = serial[s];
    p.nseg = nseg[s]; p.ncol = ncol[s]; p.ncross = ncross[s];
    p.i = i[s]; p.j = j[s]; p.k = k[s]; p.tbin = tbin[s]; p.g = g[s];
  }
  __device__ __forceinline__ void store(int s, const Part<R> &p, int dim) const {
    x[s] = p.x; t[s] = p.t;
    if (dim == 3) { y[s] = p.y; z[s] = p.z; }
    hid[s] = p.hid;
    ux[s] = p.ux; uy[s] = p.uy; uz[s] = p.uz; w[s] = p.w;
    ctr[s] = p.ctr; serial[s] = p.serial;
    nseg[s] = p.nseg; ncol[s] = p.ncol; ncross[s] = p.ncross;
    i[s] = (uint16_t)p.i; j[s] = (uint16_t)p.j; k[s] = (uint16_t)p.k;
    tbin[s] = (uint16_t)p.tbin; g[s] = (uint8_t)p.g;
  }
};

// bytes of one bank slot (kept in sync with Bank::carve)
__host__ __device__ inline int slot_bytes(bool f64, int dim) {
  const int r = f64 ? 8 : 4;
  return 8 * 2 + (dim == 3 ? 16 : 0) + 8 + 4 * r + 4 * 5 + 2 * 4 + 1 + 2 * 4 /* lists */;
}

// shared-memory layout of one CTA
struct Layout {
  int S;                 // slots
  int tables_bytes;
  long long tally_bytes; // 0 in global mode
  int bank_bytes;
  int total;
};

__host__ __device__ inline int align16(long long v) { return (int)((v + 15) & ~15ll); }

inline int tables_bytes_of(bool f64, int M, int G, int T) {
  const int r = f64 ? 8 : 4;
  long long b = 0;
  b += align16((long long)r * M * G) * 2;          // sigma_t, scat
  b += align16((long long)r * M * G * G);          // cdf
  b += align16((long long)r * G);                  // src cdf
  b += align16(8ll * G);                           // speed
  b += align16((long long)r * G);                  // inv speed
  b += align16(8ll * (T + 1));                     // edges
  return (int)b;
}

// per-thread event counters, flushed once per CTA
struct LocalCount {
  uint32_t seg, col, cross, census;
};

// ---------------------------------------------------------------------------
// geometry helpers (FP64 in both precisions)
__device__ __forceinline__ double face_of(const DevProblem &P, int a, int idx, bool up) {
  const int k = up ? idx + 1 : idx;
  return P.origin[a] + (double)k * P.width[a];
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
__device__ __forceinline__ int64_t cell_index(const DevProblem &P, int i, int j, int k) {
  if (DIM == 1) return i;
  return ((int64_t)k * P.n[1] + j) * P.n[0] + i;
}

__device__ __forceinline__ int64_t bin_index(const DevProblem &P, int64_t cell, int g, int tbin) {
  return (cell * P.G + g) * P.T1 + (P.T > 0 ? tbin : 0);
}

// ---------------------------------------------------------------------------
// records and termination bookkeeping
struct EndSink {
  double *w_end;        // shared [4]: source, absorbed, leaked, censused
  uint32_t *n_end;      // shared [8]: absorbed, leaked, censused, roulette kill, survive, splits, children, histories
};

template <class R, int DIM>
__device__ __forceinline__ void finish(const RunArgs &A, const EndSink &es, const Part<R> &p, int end) {
  if (end == END_ABSORBED) { atomicAdd(&es.n_end[0], 1u); atomicAdd(&es.w_end[1], (double)p.w); }
  else if (end == END_LEAKED) { atomicAdd(&es.n_end[1], 1u); atomicAdd(&es.w_end[2], (double)p.w); }
  else if (end == END_CENSUSED) { atomicAdd(&es.n_end[2], 1u); atomicAdd(&es.w_end[3], (double)p.w); }
  else if (end == END_ROULETTE) { atomicAdd(&es.n_end[3], 1u); }
  if (A.records != nullptr && p.serial == 0u) {
    const uint64_t r = p.hid - A.offset;
    if (r < A.n_records) {
      Record rec;
      rec.hid = p.hid; rec.end = end; rec.g = p.g; rec.ctr = p.ctr;
      rec.n_seg = p.nseg; rec.n_col = p.ncol; rec.n_cross = p.ncross;
      rec.x = p.x; rec.y = p.y; rec.z = p.z; rec.t = p.t; rec.w = (double)p.w;
      A.records[r] = rec;
    }
  }
}

// ---------------------------------------------------------------------------
// weight window at collisions and cell crossings.  Returns false if the
// particle is rouletted away.  Children go to the CTA's overflow stack.
template <class PR, int DIM>
__device__ bool weight_window(const DevProblem &P, const Tables<typename PR::R> &tb,
                              const RunArgs &A, const EndSink &es, Part<typename PR::R> &p,
                              int *s_novf, Part<typename PR::R> *ovf) {
  using R = typename PR::R;
  if (tb.ww == nullptr) return true;
  const int64_t cell = cell_index<DIM>(P, p.i, p.j, p.k);
  const int64_t bin = bin_index(P, cell, p.g, p.tbin);
  R wl;
  if constexpr (PR::kF64) wl = tb.ww[bin]; else wl = tb.ww32[bin];
  if (!(wl > (R)0)) return true;
  const R wu = (R)P.ww_upper * wl;
  if (p.w > wu) {
    const R nd = ceil(p.w / wu);
    const int n = nd > (R)P.ww_nmax ? P.ww_nmax : (int)nd;
    if (n > 1) {
      const R wc = p.w / (R)n;
      for (int c = 1; c < n; ++c) {
        const U4 h = philox4x32_10(0xFFFFFFFFu, p.serial, p.ctr, (uint32_t)c,
                                   (uint32_t)A.seed, (uint32_t)(A.seed >> 32));
        Part<R> ch = p;
        ch.w = wc;
        ch.serial = h.a;
        ch.ctr = 0;
        ch.nseg = ch.ncol = ch.ncross = 0;
        const int slot = atomicAdd(s_novf, 1);
        if (slot < A.overflow_cap) ovf[slot] = ch;
        else atomicOr(A.error, ERRBIT_OVERFLOW);
      }
      p.w = wc;
      atomicAdd(&es.n_end[5], 1u);
      atomicAdd(&es.n_end[6], (uint32_t)(n - 1));
    }
    return true;
  }
  if (p.w < wl) {
    const R ws = (R)P.ww_survival * wl;
    const U4 r = draw(p, p.ctr, A.seed);
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

// ---------------------------------------------------------------------------
// source particle (counters 0..3: x,y | z,group | mu,phi | t)
template <class PR, int DIM>
__device__ void source_particle(const DevProblem &P, const Tables<typename PR::R> &tb,
                                uint64_t seed, uint64_t hid, Part<typename PR::R> &p) {
  using R = typename PR::R;
  p.serial = 0; p.ctr = 0; p.hid = hid;
  p.nseg = p.ncol = p.ncross = 0;
  const U4 r0 = draw(p, p.ctr, seed);
  const U4 r1 = draw(p, p.ctr, seed);
  const U4 r2 = draw(p, p.ctr, seed);
  const U4 r3 = draw(p, p.ctr, seed);
  p.x = P.src_lo[0] + u01_f64(r0.a, r0.b) * (P.src_hi[0] - P.src_lo[0]);
  p.y = P.src_lo[1] + u01_f64(r0.c, r0.d) * (P.src_hi[1] - P.src_lo[1]);
  p.z = P.src_lo[2] + u01_f64(r1.a, r1.b) * (P.src_hi[2] - P.src_lo[2]);
  if constexpr (PR::kF64) p.g = sample_cdf<double>(tb.src_cdf, P.G, u01_f64(r1.c, r1.d));
  else p.g = sample_cdf<float>(tb.src_cdf, P.G, u01_f32(r1.c));
  if (P.src_kind == 1) {
    p.ux = (R)P.src_dir[0]; p.uy = (R)P.src_dir[1]; p.uz = (R)P.src_dir[2];
  } else if constexpr (PR::kF64) {
    const double two_pi = 6.283185307179586;
    const double mu = 2.0 * u01_f64(r2.a, r2.b) - 1.0;
    const double phi = two_pi * u01_f64(r2.c, r2.d);
    const double s = sqrt(1.0 - mu * mu);
    p.ux = mu; p.uy = s * cos(phi); p.uz = s * sin(phi);
  } else {
    const float mu = 2.0f * u01_f32(r2.a) - 1.0f;
    const float s = sqrtf(fmaxf(0.0f, 1.0f - mu * mu));
    float sn, cs;
    sincospif(2.0f * u01_f32(r2.c), &sn, &cs);
    p.ux = mu; p.uy = s * cs; p.uz = s * sn;
  }
  p.t = P.t0 + u01_f64(r3.a, r3.b) * (P.t1 - P.t0);
  p.w = (R)1;
  p.i = loc2index(P, 0, p.x);
  p.j = (DIM == 3) ? loc2index(P, 1, p.y) : 0;
  p.k = (DIM == 3) ? loc2index(P, 2, p.z) : 0;
  p.tbin = 0;
  if (P.T > 0)
    while (p.tbin < P.T && tb.edges[p.tbin + 1] <= p.t) p.tbin += 1;
}

// ---------------------------------------------------------------------------
// one flight.  Returns 0 continue, 1 collision queued, 2 ended (end code in *end)
enum Outcome { OUT_CONT = 0, OUT_COLL = 1, OUT_DEAD = 2 };

template <class PR, int DIM>
__device__ __forceinline__ int flight(const DevProblem &P, const Tables<typename PR::R> &tb,
                                      const RunArgs &A, const EndSink &es,
                                      Part<typename PR::R> &p, int64_t &bin,
                                      typename PR::R &score, int &end, LocalCount &lc,
                                      int *s_novf, Part<typename PR::R> *ovf) {
  using R = typename PR::R;
  const int64_t cell = cell_index<DIM>(P, p.i, p.j, p.k);
  const int m = __ldg(P.material + cell);
  const int mg = m * P.G + p.g;
  const R sig_t = tb.sigma_t[mg];

  // distance to collision
  const U4 r = draw(p, p.ctr, A.seed);
  R d_coll;
  if constexpr (PR::kF64) {
    const double xi = u01_f64(r.a, r.b);
    d_coll = sig_t > 0.0 ? -log(xi) / sig_t : rinf<double>();
  } else {
    const float xi = u01_f32(r.a);
    d_coll = sig_t > 0.0f ? -logf(xi) / sig_t : rinf<float>();
  }

  // distance to the mesh surface
  R d_surf = rinf<R>();
  int ax = -1;
  {
    const R u = p.ux;
    if (P.bounded[0] && u != (R)0) {
      const double f = face_of(P, 0, p.i, u > (R)0);
      R d;
      if constexpr (PR::kF64) d = (f - p.x) / u; else d = (float)(f - p.x) / u;
      if (d < (R)0) d = (R)0;
      if (d < d_surf) { d_surf = d; ax = 0; }
    }
  }
  if (DIM == 3) {
    const R u = p.uy;
    if (P.bounded[1] && u != (R)0) {
      const double f = face_of(P, 1, p.j, u > (R)0);
      R d;
      if constexpr (PR::kF64) d = (f - p.y) / u; else d = (float)(f - p.y) / u;
      if (d < (R)0) d = (R)0;
      if (d < d_surf) { d_surf = d; ax = 1; }
    }
    const R v = p.uz;
    if (P.bounded[2] && v != (R)0) {
      const double f = face_of(P, 2, p.k, v > (R)0);
      R d;
      if constexpr (PR::kF64) d = (f - p.z) / v; else d = (float)(f - p.z) / v;
      if (d < (R)0) d = (R)0;
      if (d < d_surf) { d_surf = d; ax = 2; }
    }
  }

  // distance to the time census
  R d_time = rinf<R>();
  if (P.T > 0) {
    if constexpr (PR::kF64) d_time = tb.speed[p.g] * (tb.edges[p.tbin + 1] - p.t);
    else d_time = (float)tb.speed[p.g] * (float)(tb.edges[p.tbin + 1] - p.t);
    if (d_time < (R)0) d_time = (R)0;
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
  bin = bin_index(P, cell, p.g, p.tbin);
  score = p.w * d;

  // move_particle (Figure "jitfunctions"): x += u d, t += d / v
  if constexpr (PR::kF64) {
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
    p.t = tb.edges[p.tbin + 1];
    p.tbin += 1;
    if (p.tbin == P.T) { end = END_CENSUSED; return OUT_DEAD; }
    return OUT_CONT;
  }
  if (ev == 1) {
    R u; int idx;
    if (ax == 0) { u = p.ux; idx = p.i; }
    else if (ax == 1) { u = p.uy; idx = p.j; }
    else { u = p.uz; idx = p.k; }
    const bool up = u > (R)0;
    const double f = face_of(P, ax, idx, up);
    if (ax == 0) p.x = f; else if (ax == 1) p.y = f; else p.z = f;
    const int nxt = idx + (up ? 1 : -1);
    if (nxt < 0 || nxt >= P.n[ax]) {
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
    if (!weight_window<PR, DIM>(P, tb, A, es, p, s_novf, ovf)) { end = END_ROULETTE; return OUT_DEAD; }
    return OUT_CONT;
  }
  return OUT_COLL;
}

// collision: absorb or scatter, new group from the transfer CDF, isotropic
// direction.  Returns true if the particle lives on.
template <class PR, int DIM>
__device__ __forceinline__ bool collide(const DevProblem &P, const Tables<typename PR::R> &tb,
                                        const RunArgs &A, const EndSink &es,
                                        Part<typename PR::R> &p, int &end, LocalCount &lc,
                                        int *s_novf, Part<typename PR::R> *ovf) {
  using R = typename PR::R;
  const int64_t cell = cell_index<DIM>(P, p.i, p.j, p.k);
  const int m = __ldg(P.material + cell);
  const int mg = m * P.G + p.g;
  p.ncol += 1;
  lc.col += 1;
  const U4 r1 = draw(p, p.ctr, A.seed);
  const U4 r2 = draw(p, p.ctr, A.seed);
  if constexpr (PR::kF64) {
    const double xi1 = u01_f64(r1.a, r1.b), xi2 = u01_f64(r1.c, r1.d);
    if (!(xi1 < tb.scat[mg])) { end = END_ABSORBED; return false; }
    p.g = sample_cdf<double>(tb.cdf + (int64_t)mg * P.G, P.G, xi2);
    const double two_pi = 6.283185307179586;
    const double mu = 2.0 * u01_f64(r2.a, r2.b) - 1.0;
    const double phi = two_pi * u01_f64(r2.c, r2.d);
    const double s = sqrt(1.0 - mu * mu);
    p.ux = mu; p.uy = s * cos(phi); p.uz = s * sin(phi);
  } else {
    const float xi1 = u01_f32(r1.a), xi2 = u01_f32(r1.c);
    if (!(xi1 < tb.scat[mg])) { end = END_ABSORBED; return false; }
    p.g = sample_cdf<float>(tb.cdf + mg * P.G, P.G, xi2);
    const float mu = 2.0f * u01_f32(r2.a) - 1.0f;
    const float s = sqrtf(fmaxf(0.0f, 1.0f - mu * mu));
    float sn, cs;
    sincospif(2.0f * u01_f32(r2.c), &sn, &cs);
    p.ux = mu; p.uy = s * cs; p.uz = s * sn;
  }
  if (!weight_window<PR, DIM>(P, tb, A, es, p, s_novf, ovf)) { end = END_ROULETTE; return false; }
  return true;
}

// ---------------------------------------------------------------------------
// tally scatter of one warp: optional warp aggregation of equal bins
template <class TT, class R>
__device__ __forceinline__ void tally_scatter(TT *stally, double *gtally, bool shared_mode,
                                              bool aggregate, bool valid, int64_t bin, R score) {
  bool act = valid && bin >= 0;
  R v = score;
  if (aggregate) {
    // lanes scoring into the same bin add their scores first; the lowest
    // such lane issues the one atomic.  All 32 lanes run the same shuffles.
    const long long key = act ? (long long)bin : -1ll;
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
    else atomicAdd(&gtally[bin], (double)v);
  }
}

// ---------------------------------------------------------------------------
template <class PR, bool SHARED, int DIM>
__global__ void __launch_bounds__(512) k_track(const DevProblem P, const RunArgs A, const Layout L) {
  using R = typename PR::R;
  using TT = typename PR::TT;
  extern __shared__ __align__(16) unsigned char smem[];
  const int tid = threadIdx.x, nth = blockDim.x;
  const int lane = tid & 31, warp = tid >> 5;
  const int S = L.S;

  // ---- carve shared memory
  unsigned char *ptr = smem;
  Tables<R> tb;
  const int M = P.M, G = P.G;
  tb.sigma_t = (R *)ptr; ptr += align16((long long)sizeof(R) * M * G);
  tb.scat = (R *)ptr; ptr += align16((long long)sizeof(R) * M * G);
  tb.cdf = (R *)ptr; ptr += align16((long long)sizeof(R) * M * G * G);
  tb.src_cdf = (R *)ptr; ptr += align16((long long)sizeof(R) * G);
  tb.speed = (double *)ptr; ptr += align16(8ll * G);
  tb.inv_speed = (R *)ptr; ptr += align16((long long)sizeof(R) * G);
  tb.edges = (double *)ptr; ptr += align16(8ll * (P.T + 1));
  tb.ww = P.ww_lower;
  tb.ww32 = P.ww_lower32;
  TT *stally = nullptr;
  if (SHARED) { stally = (TT *)ptr; ptr += L.tally_bytes; }
  Bank<R> bk;
  bk.x = (double *)ptr; ptr += 8 * S;
  bk.t = (double *)ptr; ptr += 8 * S;
  if (DIM == 3) { bk.y = (double *)ptr; ptr += 8 * S; bk.z = (double *)ptr; ptr += 8 * S; }
  else { bk.y = bk.z = nullptr; }
  bk.hid = (uint64_t *)ptr; ptr += 8 * S;
  bk.ux = (R *)ptr; ptr += sizeof(R) * S;
  bk.uy = (R *)ptr; ptr += sizeof(R) * S;
  bk.uz = (R *)ptr; ptr += sizeof(R) * S;
  bk.w = (R *)ptr; ptr += sizeof(R) * S;
  bk.ctr = (uint32_t *)ptr; ptr += 4 * S;
  bk.serial = (uint32_t *)ptr; ptr += 4 * S;
  bk.nseg = (uint32_t *)ptr; ptr += 4 * S;
  bk.ncol = (uint32_t *)ptr; ptr += 4 * S;
  bk.ncross = (uint32_t *)ptr; ptr += 4 * S;
  bk.i = (uint16_t *)ptr; ptr += 2 * S;
  bk.j = (uint16_t *)ptr; ptr += 2 * S;
  bk.k = (uint16_t *)ptr; ptr += 2 * S;
  bk.tbin = (uint16_t *)ptr; ptr += 2 * S;
  uint16_t *act = (uint16_t *)ptr; ptr += 2 * S;
  uint16_t *nxt = (uint16_t *)ptr; ptr += 2 * S;
  uint16_t *colq = (uint16_t *)ptr; ptr += 2 * S;
  uint16_t *freel = (uint16_t *)ptr; ptr += 2 * S;
  bk.g = (uint8_t *)ptr; ptr += S;

  __shared__ int s_nact, s_nnext, s_ncol, s_nfree, s_novf, s_take_ovf, s_take_src, s_done, s_nalloc,
      s_exhausted;
  __shared__ unsigned long long s_h_next, s_h_end;
  __shared__ int s_batch;
  __shared__ double s_w[4];
  __shared__ uint32_t s_n[8];
  __shared__ double s_red[32];

  // ---- load tables
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
  }
  for (int q = tid; q <= P.T; q += nth) tb.edges[q] = P.edges ? P.edges[q] : 0.0;
  if (SHARED)
    for (long long q = tid; q < P.n_bins; q += nth) stally[q] = (TT)0;
  for (int q = tid; q < S; q += nth) freel[q] = (uint16_t)(S - 1 - q);
  if (tid == 0) {
    s_nact = 0; s_nfree = S; s_novf = 0; s_done = 0; s_nalloc = 0; s_exhausted = 0;
    s_h_next = s_h_end = 0; s_batch = -1;
  }
  if (tid < 4) s_w[tid] = 0.0;
  if (tid < 8) s_n[tid] = 0u;
  __syncthreads();

  EndSink es{s_w, s_n};
  LocalCount lc{0, 0, 0, 0};
  Part<R> *ovf = reinterpret_cast<Part<R> *>(A.overflow) + (size_t)blockIdx.x * A.overflow_cap;
  const bool agg = A.warp_aggregate != 0;

  for (;;) {
    // ---- control: claim work.  Shared mode holds one batch in the private
    // tally, so a new batch is claimed only once the bank has drained;
    // global mode claims the next chunk as soon as the current one is used.
    if (tid == 0) {
      s_take_ovf = 0; s_take_src = 0;
      if (s_h_next >= s_h_end && !s_exhausted) {
        if (SHARED) {
          if (s_nact == 0 && s_novf == 0) {
            const unsigned long long b = atomicAdd(A.work, 1ull);
            if ((long long)b < A.n_batches) {
              s_batch = (int)b;
              s_h_next = batch_start(A.n_hist, A.n_batches, (int)b);
              s_h_end = batch_start(A.n_hist, A.n_batches, (int)b + 1);
            } else {
              s_exhausted = 1;
            }
          }
        } else {
          const uint64_t h0 = batch_start(A.n_hist, A.n_batches, A.batch);
          const uint64_t h1 = batch_start(A.n_hist, A.n_batches, A.batch + 1);
          const unsigned long long c = atomicAdd(A.work, (unsigned long long)A.chunk);
          if (h0 + c < h1) {
            s_h_next = h0 + c;
            s_h_end = min((unsigned long long)h1, (unsigned long long)(h0 + c + A.chunk));
          } else {
            s_exhausted = 1;
          }
        }
      }
      if (s_exhausted && s_h_next >= s_h_end && s_nact == 0 && s_novf == 0) s_done = 1;
      if (!s_done) {
        int room = s_nfree;
        const int from_ovf = min(room, min(s_novf, A.overflow_cap));
        room -= from_ovf;
        const unsigned long long left = s_h_end - s_h_next;
        s_take_ovf = from_ovf;
        s_take_src = (int)min((unsigned long long)room, left);
      }
    }
    __syncthreads();
    if (s_done) break;

    // ---- refill: overflow children first, then new source particles.  Live
    // births take the top entries of the free list in warp-append order;
    // a birth after the last census edge is censused at once and takes none.
    {
      const int n_o = s_take_ovf, n_s = s_take_src, n_new = n_o + n_s;
      const int top = s_nfree;
      const int nact0 = s_nact;
      const int base_ovf = min(s_novf, A.overflow_cap) - n_o;
      for (int base = warp * 32; base < n_new; base += nth) {
        const int q = base + lane;
        const bool valid = q < n_new;
        bool alive = false;
        Part<R> p;
        if (valid) {
          if (q < n_o) {
            p = ovf[base_ovf + q];
            alive = true;
          } else {
            const uint64_t hid = A.offset + s_h_next + (uint64_t)(q - n_o);
            source_particle<PR, DIM>(P, tb, A.seed, hid, p);
            atomicAdd(&s_w[0], 1.0);
            atomicAdd(&s_n[7], 1u);
            alive = !(P.T > 0 && p.tbin >= P.T);
            if (!alive) finish<R, DIM>(A, es, p, END_CENSUSED);
          }
        }
        const int k = warp_append(alive, &s_nalloc);
        if (alive) {
          const int slot = freel[top - 1 - k];
          bk.store(slot, p, DIM);
          act[nact0 + k] = (uint16_t)slot;
        }
      }
      __syncthreads();
      if (tid == 0) {
        s_nfree = top - s_nalloc;
        s_nact = nact0 + s_nalloc;
        s_nalloc = 0;
        s_novf = min(s_novf, A.overflow_cap) - n_o;
        s_h_next += (unsigned long long)n_s;
        s_nnext = 0;
        s_ncol = 0;
      }
      __syncthreads();
    }

    // ---- flight phase over the live list
    const int nact = s_nact;
    for (int base = warp * 32; base < nact; base += nth) {
      const int q = base + lane;
      const bool valid = q < nact;
      const int slot = valid ? act[q] : 0;
      int outcome = OUT_CONT, end = END_NONE;
      int64_t bin = -1;
      R score = (R)0;
      Part<R> p;
      if (valid) {
        bk.load(slot, p, DIM);
        outcome = flight<PR, DIM>(P, tb, A, es, p, bin, score, end, lc, &s_novf, ovf);
        if (outcome == OUT_DEAD) finish<R, DIM>(A, es, p, end);
        else bk.store(slot, p, DIM);
      }
      tally_scatter<TT, R>(stally, A.tally, SHARED, agg, valid, bin, score);
      const bool to_next = valid && outcome == OUT_CONT;
      const bool to_col = valid && outcome == OUT_COLL;
      const bool to_free = valid && outcome == OUT_DEAD;
      const int pn = warp_append(to_next, &s_nnext);
      const int pc = warp_append(to_col, &s_ncol);
      const int pf = warp_append(to_free, &s_nfree);
      if (to_next) nxt[pn] = (uint16_t)slot;
      if (to_col) colq[pc] = (uint16_t)slot;
      if (to_free) freel[pf] = (uint16_t)slot;
    }
    __syncthreads();

    // ---- collision phase over the compacted collision queue
    const int ncol = s_ncol;
    for (int base = warp * 32; base < ncol; base += nth) {
      const int q = base + lane;
      const bool valid = q < ncol;
      const int slot = valid ? colq[q] : 0;
      bool alive = false;
      if (valid) {
        Part<R> p;
        bk.load(slot, p, DIM);
        int end = END_NONE;
        alive = collide<PR, DIM>(P, tb, A, es, p, end, lc, &s_novf, ovf);
        if (alive) bk.store(slot, p, DIM);
        else finish<R, DIM>(A, es, p, end);
      }
      const bool to_next = valid && alive;
      const bool to_free = valid && !alive;
      const int pn = warp_append(to_next, &s_nnext);
      const int pf = warp_append(to_free, &s_nfree);
      if (to_next) nxt[pn] = (uint16_t)slot;
      if (to_free) freel[pf] = (uint16_t)slot;
    }
    __syncthreads();

    // ---- swap lists; fold a finished batch out of the private tally
    const int nn = s_nnext;
    for (int q = tid; q < nn; q += nth) act[q] = nxt[q];
    if (SHARED) {
      const bool batch_done = (s_h_next >= s_h_end) && nn == 0 && s_novf == 0 && s_batch >= 0;
      if (batch_done) {
        double rsum = 0.0;
        for (long long q = tid; q < P.n_bins; q += nth) {
          const double v = (double)stally[q];
          if (v != 0.0) {
            atomicAdd(&A.sum1[q], v);
            atomicAdd(&A.sum2[q], v * v);
            const long long cell = q / ((long long)P.G * P.T1);
            const int ci = (int)(cell % P.n[0]);
            const int cj = (int)((cell / P.n[0]) % P.n[1]);
            const int ck = (int)(cell / ((long long)P.n[0] * P.n[1]));
            if (ci >= P.region_lo[0] && ci < P.region_hi[0] && cj >= P.region_lo[1] &&
                cj < P.region_hi[1] && ck >= P.region_lo[2] && ck < P.region_hi[2])
              rsum += v;
            stally[q] = (TT)0;
          }
        }
        // block reduction of the region sum of this batch
        for (int o = 16; o > 0; o >>= 1) rsum += __shfl_xor_sync(0xffffffffu, rsum, o);
        if (lane == 0) s_red[warp] = rsum;
        __syncthreads();
        if (tid == 0) {
          double tot = 0.0;
          for (int w = 0; w < nth / 32; ++w) tot += s_red[w];
          atomicAdd(&A.region[0], tot);
          atomicAdd(&A.region[1], tot * tot);
          s_batch = -1;
        }
      }
    }
    __syncthreads();
    if (tid == 0) s_nact = nn;
    __syncthreads();
  }

  // ---- flush event counters: warp sums, one atomic per field per warp
  uint32_t c4[4] = {lc.seg, lc.col, lc.cross, lc.census};
#pragma unroll
  for (int f = 0; f < 4; ++f)
    for (int o = 16; o > 0; o >>= 1) c4[f] += __shfl_xor_sync(0xffffffffu, c4[f], o);
  if (lane == 0) {
    atomicAdd(&A.stats->segments, (unsigned long long)c4[0]);
    atomicAdd(&A.stats->collisions, (unsigned long long)c4[1]);
    atomicAdd(&A.stats->crossings, (unsigned long long)c4[2]);
    atomicAdd(&A.stats->census, (unsigned long long)c4[3]);
  }
  if (tid == 0) {
    atomicAdd(&A.stats->absorbed, (unsigned long long)s_n[0]);
    atomicAdd(&A.stats->leaked, (unsigned long long)s_n[1]);
    atomicAdd(&A.stats->censused, (unsigned long long)s_n[2]);
    atomicAdd(&A.stats->roulette_killed, (unsigned long long)s_n[3]);
    atomicAdd(&A.stats->roulette_survived, (unsigned long long)s_n[4]);
    atomicAdd(&A.stats->splits, (unsigned long long)s_n[5]);
    atomicAdd(&A.stats->children, (unsigned long long)s_n[6]);
    atomicAdd(&A.stats->histories, (unsigned long long)s_n[7]);
    atomicAdd(&A.stats->w_source, s_w[0]);
    atomicAdd(&A.stats->w_absorbed, s_w[1]);
    atomicAdd(&A.stats->w_leaked, s_w[2]);
    atomicAdd(&A.stats->w_censused, s_w[3]);
    if (s_novf > A.overflow_cap) atomicOr(A.error, ERRBIT_OVERFLOW);
  }
}

}  // namespace mcdc
