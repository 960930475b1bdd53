// Philox4x32-10 blocks from cuRAND's device routine, an implementation
// independent of the library's, for the generator cross-check test (the
// test compiles this file itself).
#include <cstdint>
#include <cuda_runtime.h>
#include <curand_kernel.h>

__global__ void k_ref(const uint4 *ctr, const uint2 *key, int64_t n, uint4 *out) {
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n;
       q += (int64_t)gridDim.x * blockDim.x)
    out[q] = curand_Philox4x32_10(ctr[q], key[q]);
}

// ctr: n x 4 words, key: n x 2 words, out: n x 4 words (host); 0 on success
extern "C" int curand_philox_ref(const uint32_t *ctr, const uint32_t *key, int64_t n,
                                 uint32_t *out) {
  uint4 *dc = nullptr, *dout = nullptr;
  uint2 *dk = nullptr;
  if (cudaMalloc(&dc, n * 16) || cudaMalloc(&dk, n * 8) || cudaMalloc(&dout, n * 16)) return 1;
  int rc = 0;
  if (cudaMemcpy(dc, ctr, n * 16, cudaMemcpyHostToDevice) ||
      cudaMemcpy(dk, key, n * 8, cudaMemcpyHostToDevice)) rc = 2;
  if (!rc) {
    k_ref<<<1024, 256>>>(dc, dk, n, dout);
    if (cudaDeviceSynchronize() || cudaMemcpy(out, dout, n * 16, cudaMemcpyDeviceToHost)) rc = 3;
  }
  cudaFree(dc);
  cudaFree(dk);
  cudaFree(dout);
  return rc;
}
