// misc.cu -- batch fold and finalisation kernels (streaming, HBM-bound).
#include <cmath>
#include "launch.h"

namespace mcdc {

// Global-tally mode, after each batch: sum1 += x, sum2 += x*x, x = 0 for
// every bin, plus the batch's region sum.  Reads 8 B per bin and
// read-modify-writes 32 B per bin that scored.
__global__ void __launch_bounds__(512) k_fold(const DevProblem P, double *__restrict__ tally,
                                              double *__restrict__ sum1,
                                              double *__restrict__ sum2,
                                              double *__restrict__ region_batch) {
  __shared__ double red[16];
  double rs = 0.0;
  const long long per_cell = (long long)P.G * P.T1;
  const long long n = P.n_bins;
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n;
       q += (long long)gridDim.x * blockDim.x) {
    const double v = tally[q];
    if (v != 0.0) {
      sum1[q] += v;
      sum2[q] += v * v;
      tally[q] = 0.0;
      const long long cell = q / per_cell;
      const int ci = (int)(cell % P.n[0]);
      const int cj = (int)((cell / P.n[0]) % P.n[1]);
      const int ck = (int)(cell / ((long long)P.n[0] * P.n[1]));
      if (ci >= P.region_lo[0] && ci < P.region_hi[0] && cj >= P.region_lo[1] &&
          cj < P.region_hi[1] && ck >= P.region_lo[2] && ck < P.region_hi[2])
        rs += v;
    }
  }
  for (int o = 16; o > 0; o >>= 1) rs += __shfl_xor_sync(0xffffffffu, rs, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = rs;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
    if (t != 0.0) atomicAdd(region_batch, t);
  }
}

__global__ void k_region_fold(double *region_batch, double *region) {
  const double b = *region_batch;
  region[0] += b;
  region[1] += b * b;
  *region_batch = 0.0;
}

// m_b = B s_b / (N V); mean = S1 / (N V); var of the mean from the spread of
// the batch means: (B^2 / (N V)^2) (S2 - S1^2 / B) / (B (B - 1)).
__global__ void __launch_bounds__(512) k_finalize(long long n, const double *__restrict__ sum1,
                                                  const double *__restrict__ sum2, double nv,
                                                  double B, double *__restrict__ mean,
                                                  double *__restrict__ relerr) {
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n;
       q += (long long)gridDim.x * blockDim.x) {
    const double s1 = sum1[q], s2 = sum2[q];
    const double m = s1 / nv;
    double ss = s2 - s1 * s1 / B;
    if (ss < 0.0) ss = 0.0;
    const double var = (B * B / (nv * nv)) * ss / (B * (B - 1.0));
    if (mean) mean[q] = m;
    if (relerr) relerr[q] = m != 0.0 ? sqrt(var) / fabs(m) : 0.0;
  }
}

cudaError_t launch_fold(cudaStream_t s, const DevProblem &P, double *tally, double *sum1,
                        double *sum2, double *region_batch, double *region, int sms) {
  const long long blocks = std::min<long long>((P.n_bins + 511) / 512, (long long)sms * 8);
  k_fold<<<(int)std::max<long long>(blocks, 1), 512, 0, s>>>(P, tally, sum1, sum2, region_batch);
  k_region_fold<<<1, 1, 0, s>>>(region_batch, region);
  return cudaGetLastError();
}

cudaError_t launch_finalize(cudaStream_t s, int64_t n_bins, const double *sum1,
                            const double *sum2, uint64_t n_hist, int n_batches, double volume,
                            double *mean, double *relerr, int sms) {
  const long long blocks = std::min<long long>((n_bins + 511) / 512, (long long)sms * 8);
  k_finalize<<<(int)std::max<long long>(blocks, 1), 512, 0, s>>>(
      n_bins, sum1, sum2, (double)n_hist * volume, (double)n_batches, mean, relerr);
  return cudaGetLastError();
}

}  // namespace mcdc
