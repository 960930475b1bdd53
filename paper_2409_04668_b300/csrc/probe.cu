// probe.cu -- throughput of the FP64 pipe on the current GPU, measured for the
// roofline of the FP32-split tracker (whose flights accumulate position and
// time in FP64: FP32->FP64 conversions, FP64 adds, FP64->FP32 conversions).
//
// Two kernels, each thread running 8 independent dependency chains so that
// latency is hidden and the pipe's issue rate is what the clock measures:
//   k_probe_add: x = x * c + d per step (one FP64 fused multiply-add);
//   k_probe_cvt: f = (float)((double)f + d) per step (two conversions and an
//                add).
// One CTA of 512 threads per SM.  Every thread writes one value so the work
// cannot be removed; nothing is read back but the timing.
#include <cuda_runtime.h>

#include "../../include/mcdc.h"
#include "launch.h"

namespace mcdc {

__global__ void __launch_bounds__(512) k_probe_add(double *out, int steps) {
  double a[8];
#pragma unroll
  for (int c = 0; c < 8; ++c) a[c] = 1.0 + 1e-9 * (double)(threadIdx.x + c);
  for (int i = 0; i < steps; ++i) {
#pragma unroll
    for (int c = 0; c < 8; ++c) a[c] = a[c] * 0.9999999 + 1e-7;
  }
  double s = 0.0;
#pragma unroll
  for (int c = 0; c < 8; ++c) s += a[c];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void __launch_bounds__(512) k_probe_cvt(double *out, int steps) {
  float f[8];
#pragma unroll
  for (int c = 0; c < 8; ++c) f[c] = 1.0f + 1e-6f * (float)(threadIdx.x + c);
  for (int i = 0; i < steps; ++i) {
#pragma unroll
    for (int c = 0; c < 8; ++c) f[c] = (float)((double)f[c] + 1e-9);
  }
  double s = 0.0;
#pragma unroll
  for (int c = 0; c < 8; ++c) s += (double)f[c];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace mcdc

using namespace mcdc;

extern "C" int mcdc_measure_fp64_pipe(double *add_per_s, double *cvt_per_s) {
  if (!add_per_s || !cvt_per_s) return set_error(MCDC_ERR_INVALID, "outputs are required");
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
    cudaGetLastError();
    return set_error(MCDC_ERR_NO_DEVICE, "no CUDA device");
  }
  const int threads = 512, steps = 4000;
  double *out = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  auto done = [&](int rc, const char *msg) {
    if (out) cudaFree(out);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (rc != MCDC_OK) {
      cudaGetLastError();
      return set_error(rc, msg);
    }
    return MCDC_OK;
  };
  if (cudaMalloc(&out, sizeof(double) * (size_t)sms * threads) != cudaSuccess)
    return done(MCDC_ERR_CUDA, "cudaMalloc failed");
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
    return done(MCDC_ERR_CUDA, "cudaEventCreate failed");
  // lane-operations per launch: threads x 8 chains x steps (x3 for the
  // conversion kernel: widen, add, narrow)
  const double lane_ops = (double)sms * threads * 8.0 * steps;
  float best[2] = {1e30f, 1e30f};
  for (int rep = 0; rep < 4; ++rep) {
    for (int kind = 0; kind < 2; ++kind) {
      cudaEventRecord(e0);
      if (kind == 0) k_probe_add<<<sms, threads>>>(out, steps);
      else k_probe_cvt<<<sms, threads>>>(out, steps);
      cudaEventRecord(e1);
      if (cudaEventSynchronize(e1) != cudaSuccess) return done(MCDC_ERR_CUDA, "probe kernel failed");
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      if (rep > 0 && ms < best[kind]) best[kind] = ms;   // the first round warms up
    }
  }
  if (cudaGetLastError() != cudaSuccess) return done(MCDC_ERR_CUDA, "probe kernel failed");
  *add_per_s = lane_ops / (best[0] * 1e-3);
  // the conversion kernel's step is two conversions plus one add: remove the
  // add at the measured add rate, what is left is the conversions' time
  const double t_cvt = best[1] * 1e-3 - lane_ops / *add_per_s;
  *cvt_per_s = t_cvt > 0.0 ? 2.0 * lane_ops / t_cvt : 0.0;
  return done(MCDC_OK, "");
}
