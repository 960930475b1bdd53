// checks.cu -- the checked build's entry points: whether this library was
// compiled with the bounds checks (-DMCDC_CHECKS), the message of a failed
// check, and a self-test of the check machinery that accesses nothing out of
// bounds in either build.
#include <cstdio>
#include <string>

#include <cuda_runtime.h>

#include "../../include/mcdc.h"
#include "common.cuh"
#include "launch.h"

namespace mcdc {

// one warp indexes a 16-entry shared array at its lane: lanes 16..31 fail
// their check (checked build); the explicit bound keeps the normal build,
// whose check is `true`, inside the array too
__global__ void k_check_selftest(int32_t *err, int32_t *made) {
  __shared__ int32_t buf[16];
  const int lane = threadIdx.x & 31;
  if (lane < 16) buf[lane] = 0;
  __syncwarp();
  if (MCDC_CHK(err, CHK_SELFTEST, lane < 16, lane) && lane < 16) atomicAdd(&buf[lane], 1);
  __syncwarp();
  if (lane < 16) atomicAdd(made, buf[lane]);
}

std::string check_message(const int32_t *words) {
  static const char *names[CHK_SITES] = {
      "none", "cell index", "group", "material", "time bin", "tally entry",
      "window-table bin", "warp pool slot", "warp stack of split children",
      "input bank position", "comb output slot", "comb input position", "self-test"};
  const int site = words[1];
  const long long idx =
      (long long)(((unsigned long long)(uint32_t)words[3] << 32) | (uint32_t)words[2]);
  char b[160];
  snprintf(b, sizeof b, "bounds check failed: %s (site %d), index %lld; the access was skipped",
           (site >= 0 && site < CHK_SITES) ? names[site] : "unknown", site, idx);
  return b;
}

}  // namespace mcdc

using namespace mcdc;

extern "C" int mcdc_build_checked(void) { return kChecked ? 1 : 0; }

extern "C" int mcdc_check_selftest(int32_t *words) {
  if (!words) return set_error(MCDC_ERR_INVALID, "words is required");
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return set_error(MCDC_ERR_NO_DEVICE, "no CUDA device");
  }
  int32_t *d = nullptr;
  if (cudaMalloc(&d, 5 * sizeof(int32_t)) != cudaSuccess) {
    cudaGetLastError();
    return set_error(MCDC_ERR_OOM, "cudaMalloc failed");
  }
  cudaError_t e = cudaMemset(d, 0, 5 * sizeof(int32_t));
  if (e == cudaSuccess) {
    k_check_selftest<<<1, 32>>>(d, d + 4);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpy(words, d, 5 * sizeof(int32_t), cudaMemcpyDeviceToHost);
  cudaFree(d);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return set_error(MCDC_ERR_CUDA, cudaGetErrorString(e));
  }
  return MCDC_OK;
}
