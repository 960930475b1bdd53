// track_fp64.cu -- FP64 instantiations of the tracker.  This translation unit
// is compiled with -fmad=false so that every product and sum is rounded on
// its own, in the order the source states them.
#include <algorithm>

#include "launch.h"
#include "tracker.cuh"

namespace mcdc {
namespace {
template <bool SH, int DIM, bool MU, bool NET = false, bool PC = false, bool VR = false>
void *fp64_kernel() { return (void *)k_track<PrecF64, SH, DIM, MU, NET, PC, VR>; }

template <bool SH, bool MU>
void *pick_vr(const TrackKey &k) {
  if (k.vr) return k.dim == 1 ? fp64_kernel<SH, 1, MU, false, false, true>()
                              : fp64_kernel<SH, 3, MU, false, false, true>();
  return k.dim == 1 ? fp64_kernel<SH, 1, MU>() : fp64_kernel<SH, 3, MU>();
}

void *pick(const TrackKey &k) {
  if (k.pc) return k.dim == 1 ? fp64_kernel<false, 1, false, false, true>()
                              : fp64_kernel<false, 3, false, false, true>();
  if (k.net) return k.dim == 1 ? fp64_kernel<false, 1, false, true>() : fp64_kernel<false, 3, false, true>();
  if (k.multi) return pick_vr<false, true>(k);
  if (k.shared) return pick_vr<true, false>(k);
  return pick_vr<false, false>(k);
}
}  // namespace

cudaError_t launch_track_f64(const TrackKey &key, int grid, int block, int smem,
                             cudaStream_t stream, const DevProblem &P, const RunArgs &A,
                             const Layout &L, const MultiArgs *MA) {
  const MultiArgs none{};
  void *args[] = {(void *)&P, (void *)&A, (void *)&L, (void *)(MA ? MA : &none)};
  return cudaLaunchKernel(pick(key), dim3(grid), dim3(block), args, (size_t)smem, stream);
}

cudaError_t prepare_track_f64(const TrackKey &key, int smem) {
  return cudaFuncSetAttribute(pick(key), cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
}

int track_occupancy_f64(const TrackKey &key, int block, int smem) {
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, pick(key), block, (size_t)smem) != cudaSuccess)
    return -1;
  return n;
}

cudaError_t launch_net_lower_f64(const TrackKey &key, cudaStream_t s, const DevProblem &P,
                                 const double *x, const double *t, const int32_t *g,
                                 long long n, double *out, int sms) {
  const int blocks = (int)std::min<long long>((n + 255) / 256, 8ll * sms);
  if (key.dim == 1) k_net_lower<PrecF64, 1><<<blocks, 256, 0, s>>>(P, x, t, g, n, out);
  else k_net_lower<PrecF64, 3><<<blocks, 256, 0, s>>>(P, x, t, g, n, out);
  return cudaGetLastError();
}

int track_regs_f64(const TrackKey &key) {
  cudaFuncAttributes a;
  if (cudaFuncGetAttributes(&a, pick(key)) != cudaSuccess) return -1;
  return a.numRegs;
}

}  // namespace mcdc
