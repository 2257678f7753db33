// k_stats.cu -- statistics of the VMC samples (Sec. VMC): the walker mean of
// the local energy per sweep, and the error bar of the VMC average from those
// correlated means by reblocking (blocks of doubling size until the estimate
// plateaus).  FP64 throughout, every sum in a fixed order, so that repeated
// calls give identical results.
#include "jagp_launch.h"

namespace jagp {

namespace {

constexpr int kStatThreads = 1024;

// fixed-order tree sum of one value per thread over the CTA (kStatThreads)
__device__ double block_sum(double v, double *sh) {
  sh[threadIdx.x] = v;
  __syncthreads();
  for (int o = kStatThreads / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
    __syncthreads();
  }
  const double r = sh[0];
  __syncthreads();
  return r;
}

// m[t] = (1/W) sum_w eL[t][w]: one CTA per sweep
__global__ void __launch_bounds__(kStatThreads) k_sweep_means(const double *__restrict__ eL, int W,
                                                               double *__restrict__ m) {
  __shared__ double sh[kStatThreads];
  const int t = blockIdx.x;
  double a = 0.0;
  for (int w = threadIdx.x; w < W; w += kStatThreads) a += eL[(size_t)t * W + w];
  const double s = block_sum(a, sh);
  if (threadIdx.x == 0) m[t] = s / W;
}

// Every level k < nlev of the series m[0..T): n_k = T >> k blocks of 2^k
// sweeps (the ragged tail dropped), their means b_j, sigma_k =
// sqrt(sum (b_j - bbar)^2 / (n_k (n_k - 1))) and err_k = sigma_k /
// sqrt(2 (n_k - 1)); then the plateau choice (the smallest k whose next level
// has >= 8 blocks and lies within err_k of sigma_k; else the last level with
// >= 8 blocks).  One CTA.
__global__ void __launch_bounds__(kStatThreads) k_reblock(const double *__restrict__ m, int T, int nlev,
                                                           double *__restrict__ levels, double *__restrict__ stats) {
  __shared__ double sh[kStatThreads];
  double a = 0.0;
  for (int t = threadIdx.x; t < T; t += kStatThreads) a += m[t];
  const double mean = block_sum(a, sh) / T;
  for (int k = 0; k < nlev; ++k) {
    const long B = 1L << k, nb = (long)T >> k;
    double s = 0.0;
    for (long j = threadIdx.x; j < nb; j += kStatThreads) {
      double b = 0.0;
      for (long t = 0; t < B; ++t) b += m[j * B + t];
      s += b / B;
    }
    const double bbar = block_sum(s, sh) / nb;
    double q = 0.0;
    for (long j = threadIdx.x; j < nb; j += kStatThreads) {
      double b = 0.0;
      for (long t = 0; t < B; ++t) b += m[j * B + t];
      const double d = b / B - bbar;
      q += d * d;
    }
    const double ss = block_sum(q, sh);
    if (threadIdx.x == 0) {
      const double sig = sqrt(ss / ((double)nb * (double)(nb - 1)));
      levels[4 * k + 0] = (double)B;
      levels[4 * k + 1] = (double)nb;
      levels[4 * k + 2] = sig;
      levels[4 * k + 3] = sig / sqrt(2.0 * (double)(nb - 1));
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    int chosen = -1, plateau = 0;
    for (int k = 0; k + 1 < nlev; ++k) {
      if (levels[4 * (k + 1) + 1] < 8.0) break;
      if (fabs(levels[4 * (k + 1) + 2] - levels[4 * k + 2]) <= levels[4 * k + 3]) {
        chosen = k;
        plateau = 1;
        break;
      }
    }
    if (chosen < 0)
      for (int k = 0; k < nlev; ++k)
        if (levels[4 * k + 1] >= 8.0) chosen = k;
    if (chosen < 0) chosen = 0;
    stats[0] = mean;
    stats[1] = nlev > 0 ? levels[4 * chosen + 2] : 0.0;
    stats[2] = (double)chosen;
    stats[3] = (double)plateau;
  }
}

}  // namespace

int reblock_levels(int T) {
  int n = 0;
  for (long B = 1; T / B >= 2; B *= 2) n++;
  return n;
}

cudaError_t launch_reblock(const double *eL, int T, int W, double *work, double *levels, double *stats,
                           cudaStream_t st) {
  k_sweep_means<<<T, kStatThreads, 0, st>>>(eL, W, work);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_reblock<<<1, kStatThreads, 0, st>>>(work, T, reblock_levels(T), levels, stats);
  return cudaGetLastError();
}

}  // namespace jagp
