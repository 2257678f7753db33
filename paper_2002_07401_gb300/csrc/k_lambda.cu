// k_lambda.cu -- the dominant contraction of the sweep: lambda products of
// whole orbital rows (Sec. AGP, Eq. agp_expansion), A_up rows phi^T lambda and
// Bt rows lambda phi, batched over walkers.
#include "jagp_group.cuh"
#include "jagp_launch.h"

namespace jagp {

// ---------------------------------------------------------------------------
// lambda products of whole orbital rows, batched over walkers:
//   Out[row][c] = sum_k P[row][k] Lam[k][c]
// with Lam = lambda (A_up rows phi^T lambda) or lambda^T (Bt rows lambda phi).
// In the sweep only the accepted moves' rows are listed, so the cost is
// (accepted moves) x L^2.  64 x 64 output tile, 256 threads each holding a
// 4 x 4 register block (rows ty + 16 i, columns tx + 16 j), k-chunks of 16.
// FP64 CUDA-core arithmetic.
// ---------------------------------------------------------------------------
struct LambdaRows {
  static __device__ __forceinline__ void run(const double *__restrict__ P, const double *__restrict__ Lam,
                                             double *__restrict__ Out, const int *__restrict__ list,
                                             const int *__restrict__ count, int nrows, int nsub, int stride, int L,
                                             const uint3 bid, const uint3 gdim) {
    assume_global(P, Lam, Out);
    const int rows = count ? *count : nrows;
    const int m0 = bid.y * 64;
    if (m0 >= rows) return;
    const int n0 = bid.x * 64;
    __shared__ double As[16][64];
    __shared__ double Bs[16][64];
    __shared__ long rowoff[64];
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    if (tid < 64) {
      const int m = m0 + tid;
      long phys = -1;
      if (m < rows) phys = list ? (long)list[m] : (long)(m / nsub) * stride + (m % nsub);
      rowoff[tid] = phys < 0 ? -1 : phys * (long)L;
    }
    __syncthreads();
    double acc[4][4];
  #pragma unroll
    for (int i = 0; i < 4; ++i)
  #pragma unroll
      for (int j = 0; j < 4; ++j) acc[i][j] = 0.0;
    const int lm = tid >> 2, lk = (tid & 3) * 4;   // P tile loader: row lm, k lk..lk+3
    const int bk = tid >> 4, bc = (tid & 15) * 4;  // Lam tile loader: k bk, columns bc..bc+3
    for (int k0 = 0; k0 < L; k0 += 16) {
      const long ro = rowoff[lm];
  #pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int k = k0 + lk + q;
        As[lk + q][lm] = (ro >= 0 && k < L) ? P[ro + k] : 0.0;
      }
  #pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int k = k0 + bk, c = n0 + bc + q;
        Bs[bk][bc + q] = (k < L && c < L) ? Lam[(size_t)k * L + c] : 0.0;
      }
      __syncthreads();
  #pragma unroll
      for (int kk = 0; kk < 16; ++kk) {
        double a[4], b[4];
  #pragma unroll
        for (int i = 0; i < 4; ++i) a[i] = As[kk][ty + 16 * i];
  #pragma unroll
        for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx + 16 * j];
  #pragma unroll
        for (int i = 0; i < 4; ++i)
  #pragma unroll
          for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
      }
      __syncthreads();
    }
  #pragma unroll
    for (int i = 0; i < 4; ++i) {
      const long ro = rowoff[ty + 16 * i];
      if (ro < 0) continue;
  #pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int c = n0 + tx + 16 * j;
        if (c < L) Out[ro + c] = acc[i][j];
      }
    }
}
};
__global__ void __launch_bounds__(256) k_lambda_rows(const double *__restrict__ P, const double *__restrict__ Lam,
                                                     double *__restrict__ Out, const int *__restrict__ list,
                                                     const int *__restrict__ count, int nrows, int nsub, int stride,
                                                     int L) {
  LambdaRows::run(P, Lam, Out, list, count, nrows, nsub, stride, L, blockIdx, gridDim);
}

cudaError_t launch_lambda_rows(const double *P, const double *Lam, double *Out, const int *list, const int *count,
                               int nrows, int nsub, int stride, int L, int max_rows, cudaStream_t st) {
  if (max_rows <= 0) return cudaSuccess;
  dim3 grid((L + 63) / 64, (max_rows + 63) / 64);
  return launch_or_record<LambdaRows, 256>(k_lambda_rows, grid, dim3(256), 0, st, P, Lam, Out, list, count, nrows,
                                           nsub > 0 ? nsub : 1, stride, L);
}

}  // namespace jagp
