// rng.cu -- the transport's counter-based generator as a library call:
// Philox4x32-10 blocks for caller-given counters under a 64-bit seed, through
// the same round-key path (round_keys, philox4x32_10_rk) every draw of the
// tracker takes.  Lets a user reproduce any random number of a run (counter
// words: event counter, particle serial, history id low, high) and lets the
// generator be checked against independent implementations.
#include <algorithm>
#include <string>

#include <cuda_runtime.h>

#include "../../include/mcdc.h"
#include "common.cuh"
#include "launch.h"

namespace mcdc {

__global__ void k_philox_blocks(const uint4 *__restrict__ ctr, int64_t n, RoundKeys rk,
                                uint4 *__restrict__ out) {
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n;
       q += (int64_t)gridDim.x * blockDim.x) {
    const uint4 c = ctr[q];
    const U4 r = philox4x32_10_rk(c.x, c.y, c.z, c.w, rk);
    out[q] = make_uint4(r.a, r.b, r.c, r.d);
  }
}

namespace {
bool on_device(const void *p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}
}  // namespace

}  // namespace mcdc

using namespace mcdc;

extern "C" int mcdc_philox(uint64_t seed, const uint32_t *ctr, int64_t n, uint32_t *out) {
  if (n < 0 || (n > 0 && (!ctr || !out))) return set_error(MCDC_ERR_INVALID, "bad arguments");
  if (n == 0) return MCDC_OK;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
    cudaGetLastError();
    return set_error(MCDC_ERR_NO_DEVICE, "no CUDA device");
  }
  const size_t bytes = (size_t)n * 16;
  const bool din = on_device(ctr), dout = on_device(out);
  uint4 *dc = nullptr, *dr = nullptr;
  cudaError_t e = cudaSuccess;
  if (!din) e = cudaMalloc(&dc, bytes);
  if (e == cudaSuccess && !dout) e = cudaMalloc(&dr, bytes);
  if (e == cudaSuccess && !din) e = cudaMemcpy(dc, ctr, bytes, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) {
    const uint4 *c = din ? reinterpret_cast<const uint4 *>(ctr) : dc;
    uint4 *r = dout ? reinterpret_cast<uint4 *>(out) : dr;
    const int64_t blocks = std::min<int64_t>((n + 255) / 256, (int64_t)sms * 16);
    k_philox_blocks<<<(unsigned)blocks, 256>>>(c, n, round_keys(seed), r);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e == cudaSuccess && !dout) e = cudaMemcpy(out, dr, bytes, cudaMemcpyDeviceToHost);
  }
  if (dc) cudaFree(dc);
  if (dr) cudaFree(dr);
  if (e != cudaSuccess) {
    return set_error(e == cudaErrorMemoryAllocation ? MCDC_ERR_OOM : MCDC_ERR_CUDA,
                     std::string("philox: ") + cudaGetErrorString(e));
  }
  return MCDC_OK;
}
