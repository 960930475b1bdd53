// track_fp32.cu -- FP32-split instantiations of the tracker (FP32 direction,
// distance and cross sections; FP64 position, time and tally reduction) and
// the FP32 cell-local instantiations, and the dispatch over all precisions.
#include <algorithm>

#include "launch.h"
#include "tracker.cuh"

namespace mcdc {

cudaError_t launch_track_f64(const TrackKey &, int, int, int, cudaStream_t, const DevProblem &,
                             const RunArgs &, const Layout &, const MultiArgs *);
cudaError_t prepare_track_f64(const TrackKey &, int);
int track_regs_f64(const TrackKey &);
int track_occupancy_f64(const TrackKey &, int, int);
cudaError_t launch_net_lower_f64(const TrackKey &, cudaStream_t, const DevProblem &, const double *,
                                 const double *, const int32_t *, long long, double *, int);

namespace {
template <class PR, bool SH, int DIM, bool MU, bool NET = false, bool PC = false, bool VR = false>
void *fp32_kernel() { return (void *)k_track<PR, SH, DIM, MU, NET, PC, VR>; }

// the instantiation for a tally mode and dimension, with or without varying weights
template <class PR, bool SH, bool MU>
void *pick_vr(const TrackKey &k) {
  if (k.vr) return k.dim == 1 ? fp32_kernel<PR, SH, 1, MU, false, false, true>()
                              : fp32_kernel<PR, SH, 3, MU, false, false, true>();
  return k.dim == 1 ? fp32_kernel<PR, SH, 1, MU>() : fp32_kernel<PR, SH, 3, MU>();
}

template <class PR>
void *pick_prec(const TrackKey &k) {
  if (k.pc) return k.dim == 1 ? fp32_kernel<PR, false, 1, false, false, true>()
                              : fp32_kernel<PR, false, 3, false, false, true>();
  if (k.net) return k.dim == 1 ? fp32_kernel<PR, false, 1, false, true>()
                               : fp32_kernel<PR, false, 3, false, true>();
  if (k.multi) return pick_vr<PR, false, true>(k);
  if (k.shared) return pick_vr<PR, true, false>(k);
  return pick_vr<PR, false, false>(k);
}

void *pick(const TrackKey &k) { return k.local ? pick_prec<PrecF32L>(k) : pick_prec<PrecF32>(k); }
}  // namespace

cudaError_t launch_track(const TrackKey &key, int grid, int block, int smem, cudaStream_t stream,
                         const DevProblem &P, const RunArgs &A, const Layout &L,
                         const MultiArgs *MA) {
  if (key.f64) return launch_track_f64(key, grid, block, smem, stream, P, A, L, MA);
  const MultiArgs none{};
  void *args[] = {(void *)&P, (void *)&A, (void *)&L, (void *)(MA ? MA : &none)};
  return cudaLaunchKernel(pick(key), dim3(grid), dim3(block), args, (size_t)smem, stream);
}

cudaError_t prepare_track(const TrackKey &key, int smem) {
  if (key.f64) return prepare_track_f64(key, smem);
  return cudaFuncSetAttribute(pick(key), cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
}

int track_occupancy(const TrackKey &key, int block, int smem) {
  if (key.f64) return track_occupancy_f64(key, block, smem);
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, pick(key), block, (size_t)smem) != cudaSuccess)
    return -1;
  return n;
}

namespace {
template <class PR>
cudaError_t net_lower_prec(const TrackKey &key, cudaStream_t s, const DevProblem &P,
                           const double *x, const double *t, const int32_t *g, long long n,
                           double *out, int blocks) {
  void *k = key.dim == 1 ? (void *)k_net_lower<PR, 1> : (void *)k_net_lower<PR, 3>;
  const int smem = kNetFragBytes + 8 * kNetWarpBytes;          // 256 threads: 8 warps
  if (cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, smem))
    return e;
  void *args[] = {(void *)&P, (void *)&x, (void *)&t, (void *)&g, (void *)&n, (void *)&out};
  return cudaLaunchKernel(k, dim3(blocks), dim3(256), args, (size_t)smem, s);
}
}  // namespace

cudaError_t launch_net_lower(const TrackKey &key, cudaStream_t s, const DevProblem &P,
                             const double *x, const double *t, const int32_t *g, long long n,
                             double *out, int sms) {
  if (n <= 0) return cudaSuccess;
  if (key.f64) return launch_net_lower_f64(key, s, P, x, t, g, n, out, sms);
  const int blocks = (int)std::min<long long>((n + 255) / 256, 8ll * sms);
  return key.local ? net_lower_prec<PrecF32L>(key, s, P, x, t, g, n, out, blocks)
                   : net_lower_prec<PrecF32>(key, s, P, x, t, g, n, out, blocks);
}

int track_regs(const TrackKey &key) {
  if (key.f64) return track_regs_f64(key);
  cudaFuncAttributes a;
  if (cudaFuncGetAttributes(&a, pick(key)) != cudaSuccess) return -1;
  return a.numRegs;
}

}  // namespace mcdc
