// misc.cu -- batch fold and finalisation kernels (streaming, HBM-bound).
#include <cmath>
#include "launch.h"

namespace mcdc {

// Global-tally mode, after each batch: sum1 += x, sum2 += x*x, x = 0 for
// every bin, plus the batch's region sum.  Reads 8 B per bin and
// read-modify-writes 32 B per bin that scored.  Combined estimator: the
// collision tally (second half) likewise, plus sum12 += x_track x_collision
// and the collision region sum.
// ST: the batch tally's type (FP64, or FP32 for the FP32 modes' slices); the
// sums are FP64 either way.
template <class ST>
__global__ void __launch_bounds__(512) k_fold(const DevProblem P, ST *__restrict__ tally,
                                              double *__restrict__ sum1,
                                              double *__restrict__ sum2,
                                              double *__restrict__ sum12,
                                              double *__restrict__ region_batch) {
  __shared__ double red[32];
  double rs = 0.0, rc = 0.0;
  const long long n = P.n_bins;
  const bool comb = P.estimator == 2;
  const RegionTest region(P);
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n;
       q += (long long)gridDim.x * blockDim.x) {
    const double v = (double)tally[q];
    const double vc = comb ? (double)tally[n + q] : 0.0;
    if (v != 0.0 || vc != 0.0) {
      sum1[q] += v;
      sum2[q] += v * v;
      tally[q] = (ST)0;
      if (comb) {
        sum1[n + q] += vc;
        sum2[n + q] += vc * vc;
        sum12[q] += v * vc;
        tally[n + q] = (ST)0;
      }
      if (region(P, q)) {
        rs += v;
        rc += vc;
      }
    }
  }
  for (int o = 16; o > 0; o >>= 1) {
    rs += __shfl_xor_sync(0xffffffffu, rs, o);
    rc += __shfl_xor_sync(0xffffffffu, rc, o);
  }
  const int nw = (int)(blockDim.x >> 5);
  if ((threadIdx.x & 31) == 0) { red[threadIdx.x >> 5] = rs; red[nw + (threadIdx.x >> 5)] = rc; }
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0, tc = 0.0;
    for (int w = 0; w < nw; ++w) { t += red[w]; tc += red[nw + w]; }
    if (t != 0.0) atomicAdd(&region_batch[0], t);
    if (tc != 0.0) atomicAdd(&region_batch[1], tc);
  }
}

// One-launch runs: every slice folded in one pass over the bins.  Reads each
// slice once and writes zeros back, and read-modify-writes sum1 and sum2 once
// per bin instead of once per batch.
template <class ST>
__global__ void __launch_bounds__(256) k_fold_slices(const DevProblem P, ST *__restrict__ tally,
                                                     long long nt, int B,
                                                     double *__restrict__ sum1,
                                                     double *__restrict__ sum2,
                                                     double *__restrict__ sum12,
                                                     double *__restrict__ rb) {
  extern __shared__ double srb[];          // [2 B] this block's region partials
  for (int i = threadIdx.x; i < 2 * B; i += blockDim.x) srb[i] = 0.0;
  __syncthreads();
  const long long n = P.n_bins;
  const bool comb = P.estimator == 2;
  const RegionTest region(P);
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n;
       q += (long long)gridDim.x * blockDim.x) {
    double s1 = 0.0, s2 = 0.0, c1 = 0.0, c2 = 0.0, x12 = 0.0;
    bool any = false;
    int in = -1;                           // region test, taken at the first score
    for (int b = 0; b < B; ++b) {
      ST *slice = tally + (long long)b * nt;
      const double v = (double)slice[q];
      const double vc = comb ? (double)slice[n + q] : 0.0;
      if (v != 0.0 || vc != 0.0) {
        s1 += v;
        s2 += v * v;
        slice[q] = (ST)0;
        if (comb) {
          c1 += vc;
          c2 += vc * vc;
          x12 += v * vc;
          slice[n + q] = (ST)0;
        }
        any = true;
        if (in < 0) in = region(P, q) ? 1 : 0;
        if (in) {
          atomicAdd(&srb[b], v);
          if (comb) atomicAdd(&srb[B + b], vc);
        }
      }
    }
    if (any) {
      sum1[q] += s1;
      sum2[q] += s2;
      if (comb) {
        sum1[n + q] += c1;
        sum2[n + q] += c2;
        sum12[q] += x12;
      }
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < 2 * B; i += blockDim.x)
    if (srb[i] != 0.0) atomicAdd(&rb[i], srb[i]);
}

// region[0..4] from the B per-batch region sums, batch by batch (the order of
// B k_region_fold calls); rb is zeroed for the next run
__global__ void k_region_slices(double *rb, int B, double *region, bool comb) {
  for (int b = 0; b < B; ++b) {
    const double x = rb[b];
    region[0] += x;
    region[1] += x * x;
    rb[b] = 0.0;
    if (comb) {
      const double c = rb[B + b];
      region[2] += c;
      region[3] += c * c;
      region[4] += x * c;
      rb[B + b] = 0.0;
    }
  }
}

// region[0..1] += (b, b^2) of the track-length (or only) region batch sum b;
// combined: region[2..3] for the collision sum c and region[4] += b c
__global__ void k_region_fold(double *region_batch, double *region, bool comb) {
  const double b = region_batch[0];
  region[0] += b;
  region[1] += b * b;
  region_batch[0] = 0.0;
  if (comb) {
    const double c = region_batch[1];
    region[2] += c;
    region[3] += c * c;
    region[4] += b * c;
    region_batch[1] = 0.0;
  }
}

// m_b = B s_b / (N V); mean = S1 / (N V); var of the mean from the spread of
// the batch means: (B^2 / (N V)^2) (S2 - S1^2 / B) / (B (B - 1)).
__host__ __device__ __forceinline__ void batch_moments(double s1, double s2, double nv, double B,
                                                       double &m, double &rel) {
  m = s1 / nv;
  double ss = s2 - s1 * s1 / B;
  if (ss < 0.0) ss = 0.0;
  const double var = (B * B / (nv * nv)) * ss / (B * (B - 1.0));
  rel = m != 0.0 ? sqrt(var) / fabs(m) : 0.0;
}

// The moments of batch_moments with the run's constants as reciprocals made
// once on the host (1 / (N V), 1 / B and the variance factor): per bin one
// FP64 division and one square root instead of four divisions and a square
// root -- FP64 division is a long sequence on the slow FP64 pipe, and the
// 3e7-bin channel tally took 2.7 ms to finalise.  Agrees with batch_moments
// to a few units in the last place.
__global__ void __launch_bounds__(512) k_finalize(long long n, const double *__restrict__ sum1,
                                                  const double *__restrict__ sum2, double inv_nv,
                                                  double inv_B, double cvar,
                                                  double *__restrict__ mean,
                                                  double *__restrict__ relerr) {
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n;
       q += (long long)gridDim.x * blockDim.x) {
    const double s1 = sum1[q], s2 = sum2[q];
    const double m = s1 * inv_nv;
    if (mean) mean[q] = m;
    if (relerr) {
      double ss = s2 - s1 * s1 * inv_B;
      if (ss < 0.0) ss = 0.0;
      relerr[q] = m != 0.0 ? sqrt(ss * cvar) / fabs(m) : 0.0;
    }
  }
}

// Combined estimator, per bin: batch values x_b (track length) and y_b
// (collision), each B s_b / (N V).  With the sample variances s_xx, s_yy and
// covariance s_xy of the batch values, the minimum-variance combination
// a x + (1 - a) y takes a = (s_yy - s_xy) / (s_xx + s_yy - 2 s_xy) (a = 1/2
// if that denominator is not positive: the two differ by a constant), clipped
// to [0, 1] (in a bin that one batch alone scores the two are perfectly
// correlated and the unclipped optimum is an estimate of zero); the variance
// of its mean is (a^2 s_xx + (1-a)^2 s_yy + 2 a (1-a) s_xy) / B.
// parts (optional): [5][n] track mean, track relerr, collision mean,
// collision relerr, a.
__host__ __device__ __forceinline__ void combine_moments(double s1x, double s2x, double s1y, double s2y,
                                                double s12, double nv, double B, double &m,
                                                double &rel, double &a) {
  const double c = B / nv;
  const double mx = c * s1x / B, my = c * s1y / B;
  const double sxx = (c * c * s2x - B * mx * mx) / (B - 1.0);
  const double syy = (c * c * s2y - B * my * my) / (B - 1.0);
  const double sxy = (c * c * s12 - B * mx * my) / (B - 1.0);
  const double den = sxx + syy - 2.0 * sxy;
  a = den > 0.0 ? (syy - sxy) / den : 0.5;
  a = a < 0.0 ? 0.0 : (a > 1.0 ? 1.0 : a);
  m = a * mx + (1.0 - a) * my;
  double var = (a * a * sxx + (1.0 - a) * (1.0 - a) * syy + 2.0 * a * (1.0 - a) * sxy) / B;
  if (var < 0.0) var = 0.0;
  rel = m != 0.0 ? sqrt(var) / fabs(m) : 0.0;
}

__global__ void __launch_bounds__(512) k_finalize_combined(
    long long n, const double *__restrict__ sum1, const double *__restrict__ sum2,
    const double *__restrict__ sum12, double nv, double B, double *__restrict__ mean,
    double *__restrict__ relerr, double *__restrict__ parts) {
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n;
       q += (long long)gridDim.x * blockDim.x) {
    const double s1x = sum1[q], s2x = sum2[q], s1y = sum1[n + q], s2y = sum2[n + q];
    double m, rel, a;
    combine_moments(s1x, s2x, s1y, s2y, sum12[q], nv, B, m, rel, a);
    if (mean) mean[q] = m;
    if (relerr) relerr[q] = rel;
    if (parts) {
      batch_moments(s1x, s2x, nv, B, parts[q], parts[n + q]);
      batch_moments(s1y, s2y, nv, B, parts[2 * n + q], parts[3 * n + q]);
      parts[4 * n + q] = a;
    }
  }
}

template <class ST>
cudaError_t fold_batch(cudaStream_t s, const DevProblem &P, ST *tally, double *sum1,
                       double *sum2, double *sum12, double *region_batch, double *region,
                       int sms) {
  const long long blocks = std::min<long long>((P.n_bins + 511) / 512, (long long)sms * 8);
  k_fold<ST><<<(int)std::max<long long>(blocks, 1), 512, 0, s>>>(P, tally, sum1, sum2, sum12,
                                                                 region_batch);
  k_region_fold<<<1, 1, 0, s>>>(region_batch, region, P.estimator == 2);
  return cudaGetLastError();
}
cudaError_t launch_fold(cudaStream_t s, const DevProblem &P, double *tally, double *sum1,
                        double *sum2, double *sum12, double *region_batch, double *region,
                        int sms) {
  return fold_batch(s, P, tally, sum1, sum2, sum12, region_batch, region, sms);
}
cudaError_t launch_fold(cudaStream_t s, const DevProblem &P, float *tally, double *sum1,
                        double *sum2, double *sum12, double *region_batch, double *region,
                        int sms) {
  return fold_batch(s, P, tally, sum1, sum2, sum12, region_batch, region, sms);
}

template <class ST>
cudaError_t fold_slices_all(cudaStream_t s, const DevProblem &P, ST *tally, long long nt, int B,
                            double *sum1, double *sum2, double *sum12, double *rb,
                            double *region, int sms) {
  const long long blocks = std::min<long long>((P.n_bins + 255) / 256, (long long)sms * 16);
  k_fold_slices<ST><<<(int)std::max<long long>(blocks, 1), 256, 2 * B * sizeof(double), s>>>(
      P, tally, nt, B, sum1, sum2, sum12, rb);
  k_region_slices<<<1, 1, 0, s>>>(rb, B, region, P.estimator == 2);
  return cudaGetLastError();
}
cudaError_t launch_fold_slices(cudaStream_t s, const DevProblem &P, double *tally, long long nt,
                               int B, double *sum1, double *sum2, double *sum12, double *rb,
                               double *region, int sms) {
  return fold_slices_all(s, P, tally, nt, B, sum1, sum2, sum12, rb, region, sms);
}
cudaError_t launch_fold_slices(cudaStream_t s, const DevProblem &P, float *tally, long long nt,
                               int B, double *sum1, double *sum2, double *sum12, double *rb,
                               double *region, int sms) {
  return fold_slices_all(s, P, tally, nt, B, sum1, sum2, sum12, rb, region, sms);
}

cudaError_t launch_finalize(cudaStream_t s, int64_t n_bins, const double *sum1,
                            const double *sum2, uint64_t n_hist, int n_batches, double volume,
                            double *mean, double *relerr, int sms) {
  const long long blocks = std::min<long long>((n_bins + 511) / 512, (long long)sms * 8);
  const double nv = (double)n_hist * volume, B = (double)n_batches;
  const double cvar = (B * B / (nv * nv)) / (B * (B - 1.0));
  k_finalize<<<(int)std::max<long long>(blocks, 1), 512, 0, s>>>(
      n_bins, sum1, sum2, 1.0 / nv, 1.0 / B, cvar, mean, relerr);
  return cudaGetLastError();
}

cudaError_t launch_finalize_combined(cudaStream_t s, int64_t n_bins, const double *sum1,
                                     const double *sum2, const double *sum12, uint64_t n_hist,
                                     int n_batches, double volume, double *mean, double *relerr,
                                     double *parts, int sms) {
  const long long blocks = std::min<long long>((n_bins + 511) / 512, (long long)sms * 8);
  k_finalize_combined<<<(int)std::max<long long>(blocks, 1), 512, 0, s>>>(
      n_bins, sum1, sum2, sum12, (double)n_hist * volume, (double)n_batches, mean, relerr, parts);
  return cudaGetLastError();
}

void scalar_moments(double s1, double s2, uint64_t n_hist, int n_batches, double volume,
                    double *mean, double *relerr) {
  double m, rel;
  batch_moments(s1, s2, (double)n_hist * volume, (double)n_batches, m, rel);
  *mean = m;
  *relerr = rel;
}

void combine_scalar(const double r[5], uint64_t n_hist, int n_batches, double volume,
                    double *mean, double *relerr, double *alpha) {
  double m, rel, a;
  combine_moments(r[0], r[1], r[2], r[3], r[4], (double)n_hist * volume, (double)n_batches, m,
                  rel, a);
  if (mean) *mean = m;
  if (relerr) *relerr = rel;
  if (alpha) *alpha = a;
}

}  // namespace mcdc
