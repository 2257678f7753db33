// k_linalg.cu -- the dense contractions and the FP64 inverse refresh of the
// geminal matrix (Sec. AGP, Eq. agp_expansion: G~ = Phi_up lambda Phi_dn^T | Phi_up C).
#include <math.h>

#include "jagp_group.cuh"
#include "jagp_launch.h"

namespace jagp {

// ---------------------------------------------------------------------------
// Per-walker small GEMM against row-major operands sharing the contraction
// index:  Out[w][a][b] = sum_k X[w][a][k] Y[w][b][k].
// Used for the proposed rows (Phi'_up . Bt), the proposed columns
// (Phi'_dn . A_up) and G~ at a refresh (Phi_up . Bt).  16 x 16 output tile per
// CTA, one output per thread, operands staged through shared memory in
// k-chunks of 64 (row pitch 65 doubles: conflict-free column reads).
// ---------------------------------------------------------------------------
template <typename T>
struct GemmRows {
  static __device__ __forceinline__ void run(const T *__restrict__ X, size_t xw, const T *__restrict__ Y, size_t yw,
                                             int ma, int nb, int K, T *__restrict__ Out, size_t ow, int ldo,
                                             const uint3 bid, const uint3 gdim) {
    assume_global(X, Y, Out);
    __shared__ T Xs[16][65];
    __shared__ T Ys[16][65];
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    const int w = bid.z, a0 = bid.y * 16, b0 = bid.x * 16;
    const T *Xw = X + (size_t)w * xw;
    const T *Yw = Y + (size_t)w * yw;
    T acc = T(0);
    for (int k0 = 0; k0 < K; k0 += 64) {
  #pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int idx = threadIdx.x + q * 256, row = idx >> 6, col = idx & 63;
        const int k = k0 + col;
        const int a = a0 + row, b = b0 + row;
        Xs[row][col] = (a < ma && k < K) ? Xw[(size_t)a * K + k] : T(0);
        Ys[row][col] = (b < nb && k < K) ? Yw[(size_t)b * K + k] : T(0);
      }
      __syncthreads();
  #pragma unroll 16
      for (int k = 0; k < 64; ++k) acc = fma(Xs[ty][k], Ys[tx][k], acc);
      __syncthreads();
    }
    if (a0 + ty < ma && b0 + tx < nb) Out[(size_t)w * ow + (size_t)(a0 + ty) * ldo + b0 + tx] = acc;
}
};
template <typename T>
__global__ void __launch_bounds__(256) k_gemm_rows(const T *__restrict__ X, size_t xw, const T *__restrict__ Y,
                                                   size_t yw, int ma, int nb, int K, T *__restrict__ Out, size_t ow,
                                                   int ldo) {
  GemmRows<T>::run(X, xw, Y, yw, ma, nb, K, Out, ow, ldo, blockIdx, gridDim);
}

// The refresh's G~ = Phi_up Bt^T in the FP32 path: the same tile scheme with a
// compensated dot product (error-free product by fma, error-free sum, the
// errors summed separately; Ogita, Rump and Oishi 2005) over two-float
// operands X + Xlo and Y + Ylo (the low parts' products with the high parts go
// into the error sum; lo * lo is below the result's precision), so that G~ is
// as accurate as the double-word tables rather than FP32.  The _rn intrinsics
// keep the compiler from fusing the steps.
struct GemmRowsDot2 {
  static __device__ __forceinline__ void run(const float *__restrict__ X, const float *__restrict__ Xlo, size_t xw,
                                             const float *__restrict__ Y, const float *__restrict__ Ylo, size_t yw,
                                             int ma, int nb, int K, double *__restrict__ Out, size_t ow, int ldo,
                                             const uint3 bid, const uint3 gdim) {
    assume_global(X, Y, Out);
    __shared__ float Xs[16][65];
    __shared__ float Xl[16][65];
    __shared__ float Ys[16][65];
    __shared__ float Yl[16][65];
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    const int w = bid.z, a0 = bid.y * 16, b0 = bid.x * 16;
    float s = 0.0f, c = 0.0f;
    for (int k0 = 0; k0 < K; k0 += 64) {
  #pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int idx = threadIdx.x + q * 256, row = idx >> 6, col = idx & 63;
        const int k = k0 + col;
        const int a = a0 + row, b = b0 + row;
        const bool xa = a < ma && k < K, yb = b < nb && k < K;
        const size_t xi = (size_t)w * xw + (size_t)a * K + k, yi = (size_t)w * yw + (size_t)b * K + k;
        Xs[row][col] = xa ? X[xi] : 0.0f;
        Xl[row][col] = (Xlo && xa) ? Xlo[xi] : 0.0f;
        Ys[row][col] = yb ? Y[yi] : 0.0f;
        Yl[row][col] = (Ylo && yb) ? Ylo[yi] : 0.0f;
      }
      __syncthreads();
  #pragma unroll 8
      for (int k = 0; k < 64; ++k) {
        const float x = Xs[ty][k], y = Ys[tx][k];
        const float p = __fmul_rn(x, y);
        const float pe = __fmaf_rn(x, y, -p);
        const float t = __fadd_rn(s, p);
        const float z = __fsub_rn(t, s);
        const float se = __fadd_rn(__fsub_rn(s, __fsub_rn(t, z)), __fsub_rn(p, z));
        s = t;
        const float cross = __fmaf_rn(Xl[ty][k], y, __fmul_rn(x, Yl[tx][k]));
        c = __fadd_rn(c, __fadd_rn(__fadd_rn(cross, pe), se));
      }
      __syncthreads();
    }
    // the pair (s, c) carries more than FP32 precision: keep it in FP64
    if (a0 + ty < ma && b0 + tx < nb)
      Out[(size_t)w * ow + (size_t)(a0 + ty) * ldo + b0 + tx] = static_cast<double>(s) + static_cast<double>(c);
}
};
__global__ void __launch_bounds__(256) k_gemm_rows_dot2(const float *__restrict__ X, const float *__restrict__ Xlo,
                                                        size_t xw, const float *__restrict__ Y,
                                                        const float *__restrict__ Ylo, size_t yw, int ma, int nb,
                                                        int K, double *__restrict__ Out, size_t ow, int ldo) {
  GemmRowsDot2::run(X, Xlo, xw, Y, Ylo, yw, ma, nb, K, Out, ow, ldo, blockIdx, gridDim);
}

// ---------------------------------------------------------------------------
// Register-blocked variant of the two kernels above for N_up >= 32: a TM x TM
// output tile per CTA of 256 threads, R x R outputs per thread (R = TM / 16),
// operands staged through shared memory in k-chunks of 32, transposed so that
// each thread reads R consecutive entries of a column.  With DOT2 every output
// keeps the compensated pair (s, c) of the kernel above; the order of the
// k-sum is the same as there.
// ---------------------------------------------------------------------------
template <typename T, int TM, bool DOT2, typename OutT>
struct GemmRowsBlk {
  static __device__ __forceinline__ void run(const T *__restrict__ X, const float *__restrict__ Xlo, size_t xw,
                                             const T *__restrict__ Y, const float *__restrict__ Ylo, size_t yw,
                                             int ma, int nb, int K, OutT *__restrict__ Out, size_t ow, int ldo,
                                             const uint3 bid, const uint3 gdim) {
    assume_global(X, Y, Out);
    constexpr int KC = 32, R = TM / 16, PAD = TM + 1;
    __shared__ T Xs[KC][PAD];
    __shared__ T Ys[KC][PAD];
    __shared__ float Xl[DOT2 ? KC : 1][DOT2 ? PAD : 1];
    __shared__ float Yl[DOT2 ? KC : 1][DOT2 ? PAD : 1];
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    const int w = bid.z, a0 = bid.y * TM, b0 = bid.x * TM;
    const T *Xw = X + (size_t)w * xw;
    const T *Yw = Y + (size_t)w * yw;
    T acc[R][R];
    float cmp[DOT2 ? R : 1][DOT2 ? R : 1];
  #pragma unroll
    for (int i = 0; i < R; ++i)
  #pragma unroll
      for (int j = 0; j < R; ++j) {
        acc[i][j] = T(0);
        if constexpr (DOT2) cmp[i][j] = 0.0f;
      }
    for (int k0 = 0; k0 < K; k0 += KC) {
      // TM rows x KC columns of each operand; consecutive threads take consecutive k
  #pragma unroll
      for (int q = 0; q < TM * KC / 256; ++q) {
        const int idx = tid + q * 256, row = idx / KC, kk = idx % KC;
        const int k = k0 + kk, a = a0 + row, b = b0 + row;
        const bool xa = a < ma && k < K, yb = b < nb && k < K;
        const size_t xi = (size_t)a * K + k, yi = (size_t)b * K + k;
        Xs[kk][row] = xa ? Xw[xi] : T(0);
        Ys[kk][row] = yb ? Yw[yi] : T(0);
        if constexpr (DOT2) {
          Xl[kk][row] = (Xlo && xa) ? Xlo[(size_t)w * xw + xi] : 0.0f;
          Yl[kk][row] = (Ylo && yb) ? Ylo[(size_t)w * yw + yi] : 0.0f;
        }
      }
      __syncthreads();
  #pragma unroll 4
      for (int kk = 0; kk < KC; ++kk) {
        T xa[R], yb[R];
  #pragma unroll
        for (int i = 0; i < R; ++i) xa[i] = Xs[kk][ty * R + i];
  #pragma unroll
        for (int j = 0; j < R; ++j) yb[j] = Ys[kk][tx * R + j];
        if constexpr (DOT2) {
          float xl[R], yl[R];
  #pragma unroll
          for (int i = 0; i < R; ++i) xl[i] = Xl[kk][ty * R + i];
  #pragma unroll
          for (int j = 0; j < R; ++j) yl[j] = Yl[kk][tx * R + j];
  #pragma unroll
          for (int i = 0; i < R; ++i)
  #pragma unroll
            for (int j = 0; j < R; ++j) {
              const float x = xa[i], y = yb[j], s = acc[i][j];
              const float p = __fmul_rn(x, y);
              const float pe = __fmaf_rn(x, y, -p);
              const float t = __fadd_rn(s, p);
              const float z = __fsub_rn(t, s);
              const float se = __fadd_rn(__fsub_rn(s, __fsub_rn(t, z)), __fsub_rn(p, z));
              acc[i][j] = t;
              const float cross = __fmaf_rn(xl[i], y, __fmul_rn(x, yl[j]));
              cmp[i][j] = __fadd_rn(cmp[i][j], __fadd_rn(__fadd_rn(cross, pe), se));
            }
        } else {
  #pragma unroll
          for (int i = 0; i < R; ++i)
  #pragma unroll
            for (int j = 0; j < R; ++j) acc[i][j] = fma(xa[i], yb[j], acc[i][j]);
        }
      }
      __syncthreads();
    }
  #pragma unroll
    for (int i = 0; i < R; ++i) {
      const int a = a0 + ty * R + i;
      if (a >= ma) continue;
  #pragma unroll
      for (int j = 0; j < R; ++j) {
        const int b = b0 + tx * R + j;
        if (b >= nb) continue;
        OutT v;
        if constexpr (DOT2)
          v = static_cast<double>(acc[i][j]) + static_cast<double>(cmp[i][j]);
        else
          v = acc[i][j];
        Out[(size_t)w * ow + (size_t)a * ldo + b] = v;
      }
    }
}
};
template <typename T, int TM, bool DOT2, typename OutT>
__global__ void __launch_bounds__(256) k_gemm_rows_blk(const T *__restrict__ X, const float *__restrict__ Xlo,
                                                       size_t xw, const T *__restrict__ Y,
                                                       const float *__restrict__ Ylo, size_t yw, int ma, int nb,
                                                       int K, OutT *__restrict__ Out, size_t ow, int ldo) {
  GemmRowsBlk<T, TM, DOT2, OutT>::run(X, Xlo, xw, Y, Ylo, yw, ma, nb, K, Out, ow, ldo, blockIdx, gridDim);
}

// tile of the blocked variant for an ma x nb output (0: the one-output-per-thread kernel)
inline int gemm_rows_tile(int ma, int nb) {
  const int m = ma < nb ? ma : nb;
  return m >= 64 ? 64 : (m >= 32 ? 32 : 0);
}

// The compensated product for small blocks (ma, nb <= 16): four walkers per
// CTA, 64 threads each with a 2 x 2 output block, so that every shared-memory
// operand read serves two outputs instead of one; k order as above.
struct GemmRowsDot2Small {
  static __device__ __forceinline__ void run(const float *__restrict__ X, const float *__restrict__ Xlo, size_t xw,
                                             const float *__restrict__ Y, const float *__restrict__ Ylo, size_t yw,
                                             int ma, int nb, int K, double *__restrict__ Out, size_t ow, int ldo,
                                             int W, const uint3 bid, const uint3 gdim) {
    assume_global(X, Y, Out);
    constexpr int KC = 32;
    __shared__ float Xs[4][KC][17], Xl[4][KC][17], Ys[4][KC][17], Yl[4][KC][17];
    const int sub = threadIdx.x >> 6, t = threadIdx.x & 63;
    const int w = bid.x * 4 + sub;
    const bool active = w < W;  // inactive groups still take part in the barriers
    const int tx = t & 7, ty = t >> 3;  // outputs (2 ty + i, 2 tx + j)
    float s[2][2] = {{0.0f, 0.0f}, {0.0f, 0.0f}}, c[2][2] = {{0.0f, 0.0f}, {0.0f, 0.0f}};
    for (int k0 = 0; k0 < K; k0 += KC) {
      for (int idx = t; idx < 16 * KC; idx += 64) {
        const int row = idx / KC, kk = idx % KC, k = k0 + kk;
        const bool xa = active && row < ma && k < K, yb = active && row < nb && k < K;
        const size_t xi = (size_t)w * xw + (size_t)row * K + k, yi = (size_t)w * yw + (size_t)row * K + k;
        Xs[sub][kk][row] = xa ? X[xi] : 0.0f;
        Xl[sub][kk][row] = (Xlo && xa) ? Xlo[xi] : 0.0f;
        Ys[sub][kk][row] = yb ? Y[yi] : 0.0f;
        Yl[sub][kk][row] = (Ylo && yb) ? Ylo[yi] : 0.0f;
      }
      __syncthreads();
  #pragma unroll 4
      for (int kk = 0; kk < KC; ++kk) {
        const float x0 = Xs[sub][kk][2 * ty], x1 = Xs[sub][kk][2 * ty + 1];
        const float l0 = Xl[sub][kk][2 * ty], l1 = Xl[sub][kk][2 * ty + 1];
        const float y0 = Ys[sub][kk][2 * tx], y1 = Ys[sub][kk][2 * tx + 1];
        const float m0 = Yl[sub][kk][2 * tx], m1 = Yl[sub][kk][2 * tx + 1];
        const float xv[2] = {x0, x1}, xl[2] = {l0, l1}, yv[2] = {y0, y1}, yl[2] = {m0, m1};
  #pragma unroll
        for (int i = 0; i < 2; ++i)
  #pragma unroll
          for (int j = 0; j < 2; ++j) {
            const float x = xv[i], y = yv[j], sv = s[i][j];
            const float p = __fmul_rn(x, y);
            const float pe = __fmaf_rn(x, y, -p);
            const float tt = __fadd_rn(sv, p);
            const float z = __fsub_rn(tt, sv);
            const float se = __fadd_rn(__fsub_rn(sv, __fsub_rn(tt, z)), __fsub_rn(p, z));
            s[i][j] = tt;
            const float cross = __fmaf_rn(xl[i], y, __fmul_rn(x, yl[j]));
            c[i][j] = __fadd_rn(c[i][j], __fadd_rn(__fadd_rn(cross, pe), se));
          }
      }
      __syncthreads();
    }
    if (!active) return;
  #pragma unroll
    for (int i = 0; i < 2; ++i)
  #pragma unroll
      for (int j = 0; j < 2; ++j) {
        const int a = 2 * ty + i, b = 2 * tx + j;
        if (a < ma && b < nb)
          Out[(size_t)w * ow + (size_t)a * ldo + b] = static_cast<double>(s[i][j]) + static_cast<double>(c[i][j]);
      }
}
};
__global__ void __launch_bounds__(256) k_gemm_rows_dot2_small(const float *__restrict__ X,
                                                              const float *__restrict__ Xlo, size_t xw,
                                                              const float *__restrict__ Y,
                                                              const float *__restrict__ Ylo, size_t yw, int ma,
                                                              int nb, int K, double *__restrict__ Out, size_t ow,
                                                              int ldo, int W) {
  GemmRowsDot2Small::run(X, Xlo, xw, Y, Ylo, yw, ma, nb, K, Out, ow, ldo, W, blockIdx, gridDim);
}

cudaError_t launch_gemm_rows_dot2(const float *X, const float *Xlo, size_t xw, const float *Y, const float *Ylo,
                                  size_t yw, int ma, int nb, int K, double *Out, size_t ow, int ldo, int W,
                                  cudaStream_t st, int tile) {
  if (W <= 0 || ma <= 0 || nb <= 0) return cudaSuccess;
  if (tile != -1 && tile != 0 && tile != 16 && tile != 32 && tile != 64) return cudaErrorInvalidValue;
  const int tm = tile >= 0 ? tile : (ma <= 16 && nb <= 16 ? 16 : gemm_rows_tile(ma, nb));
  if (tm == 16) {
    if (ma > 16 || nb > 16) return cudaErrorInvalidValue;
    return launch_or_record<GemmRowsDot2Small, 256>(k_gemm_rows_dot2_small, dim3((W + 3) / 4), dim3(256), 0, st, X,
                                                     Xlo, xw, Y, Ylo, yw, ma, nb, K, Out, ow, ldo, W);
  }
  if (tm) {
    dim3 grid((nb + tm - 1) / tm, (ma + tm - 1) / tm, W);
    if (tm == 64)
      return launch_or_record<GemmRowsBlk<float, 64, true, double>, 256>(k_gemm_rows_blk<float, 64, true, double>, grid, dim3(256), 0, st, X, Xlo, xw, Y, Ylo, yw, ma, nb, K, Out, ow,
          ldo);
    return launch_or_record<GemmRowsBlk<float, 32, true, double>, 256>(k_gemm_rows_blk<float, 32, true, double>, grid, dim3(256), 0, st, X, Xlo, xw, Y, Ylo, yw, ma, nb, K, Out, ow,
        ldo);
  }
  dim3 grid((nb + 15) / 16, (ma + 15) / 16, W);
  return launch_or_record<GemmRowsDot2, 256>(k_gemm_rows_dot2, grid, dim3(256), 0, st, X, Xlo, xw, Y, Ylo, yw, ma, nb,
                                             K, Out, ow, ldo);
}

template <typename T>
cudaError_t launch_gemm_rows(const T *X, size_t xw, const T *Y, size_t yw, int ma, int nb, int K, T *Out, size_t ow,
                             int ldo, int W, cudaStream_t st, int tile) {
  if (W <= 0 || ma <= 0 || nb <= 0) return cudaSuccess;
  if (tile != -1 && tile != 0 && tile != 32 && tile != 64) return cudaErrorInvalidValue;
  const int tm = tile >= 0 ? tile : gemm_rows_tile(ma, nb);
  if (tm) {
    dim3 grid((nb + tm - 1) / tm, (ma + tm - 1) / tm, W);
    const float *none = nullptr;
    if (tm == 64)
      return launch_or_record<GemmRowsBlk<T, 64, false, T>, 256>(k_gemm_rows_blk<T, 64, false, T>, grid, dim3(256), 0,
                                                                 st, X, none, xw, Y, none, yw, ma, nb, K, Out, ow, ldo);
    return launch_or_record<GemmRowsBlk<T, 32, false, T>, 256>(k_gemm_rows_blk<T, 32, false, T>, grid, dim3(256), 0,
                                                               st, X, none, xw, Y, none, yw, ma, nb, K, Out, ow, ldo);
  }
  dim3 grid((nb + 15) / 16, (ma + 15) / 16, W);
  return launch_or_record<GemmRows<T>, 256>(k_gemm_rows<T>, grid, dim3(256), 0, st, X, xw, Y, yw, ma, nb, K, Out, ow,
                                            ldo);
}
template cudaError_t launch_gemm_rows<double>(const double *, size_t, const double *, size_t, int, int, int, double *,
                                              size_t, int, int, cudaStream_t, int);
template cudaError_t launch_gemm_rows<float>(const float *, size_t, const float *, size_t, int, int, int, float *,
                                             size_t, int, int, cudaStream_t, int);

template <typename T>
__global__ void k_fill_unpaired(const double *__restrict__ unp, T *__restrict__ bt, int W, int nu, int nd,
                                int L) {
  const int k = nu - nd;
  const long total = (long)W * k * L;
  for (long idx = blockIdx.x * (long)blockDim.x + threadIdx.x; idx < total; idx += (long)gridDim.x * blockDim.x) {
    const int c = (int)(idx % L);
    const long t = idx / L;
    const int l = (int)(t % k);
    const int w = (int)(t / k);
    bt[((size_t)w * nu + nd + l) * L + c] = static_cast<T>(unp[(size_t)l * L + c]);
  }
}

template <typename T>
cudaError_t launch_fill_unpaired(const DevSystem &s, T *bt, int W, cudaStream_t st) {
  if (W <= 0 || s.n_up == s.n_dn) return cudaSuccess;
  const long total = (long)W * (s.n_up - s.n_dn) * s.L;
  long blocks = (total + 255) / 256;
  if (blocks > 152 * 8) blocks = 152 * 8;
  k_fill_unpaired<T><<<(int)blocks, 256, 0, st>>>(s.unpaired, bt, W, s.n_up, s.n_dn, s.L);
  return cudaGetLastError();
}
template cudaError_t launch_fill_unpaired<double>(const DevSystem &, double *, int, cudaStream_t);

__global__ void k_fill_unpaired_lo(const double *__restrict__ unp, float *__restrict__ lo, int W, int nu, int nd,
                                   int L) {
  const int k = nu - nd;
  const long total = (long)W * k * L;
  for (long idx = blockIdx.x * (long)blockDim.x + threadIdx.x; idx < total; idx += (long)gridDim.x * blockDim.x) {
    const int c = (int)(idx % L);
    const long t = idx / L;
    const int l = (int)(t % k);
    const int w = (int)(t / k);
    const double v = unp[(size_t)l * L + c];
    lo[((size_t)w * nu + nd + l) * L + c] = static_cast<float>(v - static_cast<double>(static_cast<float>(v)));
  }
}

cudaError_t launch_fill_unpaired_lo(const DevSystem &s, float *lo, int W, cudaStream_t st) {
  if (W <= 0 || s.n_up == s.n_dn) return cudaSuccess;
  const long total = (long)W * (s.n_up - s.n_dn) * s.L;
  long blocks = (total + 255) / 256;
  if (blocks > 152 * 8) blocks = 152 * 8;
  k_fill_unpaired_lo<<<(int)blocks, 256, 0, st>>>(s.unpaired, lo, W, s.n_up, s.n_dn, s.L);
  return cudaGetLastError();
}
template cudaError_t launch_fill_unpaired<float>(const DevSystem &, float *, int, cudaStream_t);

// 1/p in FP64 from an FP32 seed and two Newton steps y <- y (2 - p y) (error
// squares each step: 2^-23 -> 2^-46 -> below FP64 rounding); p must be a
// normal number within FP32 range, else the FP64 division is used.
__device__ __forceinline__ double recip_newton(double p) {
  const double a = fabs(p);
  if (!(a > 1e-37 && a < 1e37)) return 1.0 / p;
  double y = static_cast<double>(__frcp_rn(static_cast<float>(p)));
  y = y * fma(-p, y, 2.0);
  y = y * fma(-p, y, 2.0);
  return y;
}

// log|prod of pivots| without a logarithm per pivot: the product is kept as a
// mantissa in [1/2, 1) and a binary exponent (frexp after every factor), and
// one log at the end gives log|m| + E ln 2.
struct PivotProduct {
  double m = 1.0;
  int e = 0;
  __device__ __forceinline__ void mul(double pv) {
    int e1, e2;
    const double a = frexp(fabs(pv), &e1);
    m = frexp(m * a, &e2);
    e += e1 + e2;
  }
  __device__ __forceinline__ double log_abs() const { return log(m) + e * 0.6931471805599453; }
};

// ---------------------------------------------------------------------------
// FP64 refresh: Gauss-Jordan elimination with partial pivoting.  log|det G~| is
// log|prod of pivots|, the sign the product of pivot signs and the parity of
// the row order.  The fresh inverse replaces the Sherman-Morrison one; their
// largest difference times max|G~| is the walker's drift.
// ---------------------------------------------------------------------------
constexpr size_t kMmatSmemMax = 200 * 1024;  // k_mmat stages G~^{-1} whole up to this footprint
constexpr size_t kRefreshSmemMax = 200 * 1024;  // shared-memory rows of the in-place refresh up to this footprint

// N_up <= 32: register-resident in-place Gauss-Jordan.  A group of NM lanes
// (NM = 8, 16 or 32, the smallest >= N_up) holds one walker's matrix, lane c
// its column c in NM registers (rows and columns past N_up are the identity);
// a warp holds 32 / NM walkers.  No rows are swapped: step k pivots on the
// largest |entry| of column k among the rows not yet pivoted (the lowest row
// on ties), with the in-place update of the exchange form (pivot row scaled by
// 1/p, -f_i / p into column k, f_i = A[i][k]).  After the last step row p_k
// holds x_k, so inverse[k][p_k'] is entry (p_k, k') of the result, and the
// determinant's sign is that of the pivot product times (-1)^(inversions of
// the pivot order).  Pivot keys compare as the integer bits of |value|.
template <typename T, int NM>
struct RefreshInverseReg {
  static __device__ __forceinline__ void run(const double *__restrict__ gm, T *__restrict__ ginv,
                                             double *__restrict__ scal, int *__restrict__ status, int n, int W,
                                             int check_drift, double drift_tol, double *__restrict__ ginv64,
                                             const uint3 bid, const uint3 gdim) {
    assume_global(gm, ginv, scal, status);
    constexpr int kGroups = 32 / NM;
    constexpr unsigned kFull = 0xffffffffu;
    const int lane = threadIdx.x & 31, c = lane & (NM - 1), g0 = lane - c;
    const int w = (bid.x * 4 + (threadIdx.x >> 5)) * kGroups + lane / NM;
    const bool live = w < W;  // lanes of walkers past W run on the identity and write nothing
    const double *Gw = gm + (size_t)(live ? w : 0) * n * n;
    double a[NM];
    double gmax = 0.0;
  #pragma unroll
    for (int i = 0; i < NM; ++i) {
      double v = i == c ? 1.0 : 0.0;
      if (live && i < n && c < n) {
        v = Gw[i * n + c];
        gmax = fmax(gmax, fabs(v));
      }
      a[i] = v;
    }
    const unsigned rows_n = n >= 32 ? kFull : ((1u << n) - 1u);
    unsigned used = 0;  // rows pivoted so far (the same in every lane of a group)
    int inversions = 0, myp = 0, myq = 0;  // lane c: pivot row of step c; step at which row c was pivoted
    PivotProduct pp;
    bool neg = false, ok = true;
    for (int k = 0; k < n; ++k) {
      // lane i of the group picks up f_i = A[i][k] from lane k
      double fme = 0.0;
  #pragma unroll
      for (int i = 0; i < NM; ++i) {
        const double t = __shfl_sync(kFull, a[i], g0 + k);
        if (c == i) fme = t;
      }
      unsigned long long key = (c < n && !((used >> c) & 1u))
                                   ? static_cast<unsigned long long>(__double_as_longlong(fme)) & 0x7fffffffffffffffull
                                   : 0ull;
      int pi = c;
  #pragma unroll
      for (int o = NM / 2; o > 0; o >>= 1) {
        const unsigned long long ok2 = __shfl_xor_sync(kFull, key, o);
        const int oi = __shfl_xor_sync(kFull, pi, o);
        if (ok2 > key || (ok2 == key && oi < pi)) {
          key = ok2;
          pi = oi;
        }
      }
      const int p = pi;
      const double pv = __shfl_sync(kFull, fme, g0 + p);
      ok = ok && !((used >> p) & 1u) && pv != 0.0 && isfinite(pv);
      inversions += __popc(~used & rows_n & ((1u << p) - 1u));
      used |= 1u << p;
      if (c == k) myp = p;
      if (c == p) myq = k;
      pp.mul(pv);
      neg ^= pv < 0.0;
      const double ip = recip_newton(pv);
      double prow = 0.0;
  #pragma unroll
      for (int i = 0; i < NM; ++i)
        if (i == p) prow = a[i];
      prow = c == k ? ip : prow * ip;
      const bool colk = c == k;
  #pragma unroll
      for (int i = 0; i < NM; ++i) {
        const double fi = __shfl_sync(kFull, a[i], g0 + k);
        a[i] = i == p ? prow : fma(-fi, prow, colk ? 0.0 : a[i]);
      }
    }
    // inverse[k][p_c] = result[p_k][c]: row i of the result goes to row q_i
    T *gi = ginv + (size_t)(live ? w : 0) * n * n;
    double dmax = 0.0;
  #pragma unroll
    for (int i = 0; i < NM; ++i) {
      const int qi = __shfl_sync(kFull, myq, g0 + i);
      if (live && ok && i < n && c < n) {
        const size_t idx = (size_t)qi * n + myp;
        if (check_drift) dmax = fmax(dmax, fabs(a[i] - static_cast<double>(gi[idx])));
        gi[idx] = static_cast<T>(a[i]);
        if (ginv64) ginv64[(size_t)w * n * n + idx] = a[i];
      }
    }
  #pragma unroll
    for (int o = NM / 2; o > 0; o >>= 1) {
      dmax = fmax(dmax, __shfl_xor_sync(kFull, dmax, o));
      gmax = fmax(gmax, __shfl_xor_sync(kFull, gmax, o));
    }
    if (!live || c != 0) return;
    double *sw = scal + (size_t)w * S_STRIDE;
    if (!ok) {
      status[w] |= JAGP_WS_SINGULAR;
      sw[S_LOGDET] = -INFINITY;
      sw[S_SIGN] = 0.0;
      return;
    }
    sw[S_LOGDET] = pp.log_abs();
    sw[S_SIGN] = (neg != (inversions & 1)) ? -1.0 : 1.0;
    if (check_drift) {
      const double drift = dmax * gmax;
      sw[S_DRIFT] = drift;
      if (!(drift <= drift_tol)) status[w] |= JAGP_WS_DRIFT;
    }
}
};
template <typename T, int NM>
__global__ void __launch_bounds__(128) k_refresh_inverse_reg(const double *__restrict__ gm, T *__restrict__ ginv,
                                                             double *__restrict__ scal, int *__restrict__ status,
                                                             int n, int W, int check_drift, double drift_tol,
                                                             double *__restrict__ ginv64) {
  RefreshInverseReg<T, NM>::run(gm, ginv, scal, status, n, W, check_drift, drift_tol, ginv64, blockIdx, gridDim);
}

// 32 < N_up <= 64: the same register-resident scheme on two warps per walker.
// Warp h of a walker holds rows 32 h .. 32 h + 31, lane c the columns c and
// c + 32 (identity past N_up); the pivot of each step is found per warp by
// shuffles and between the two warps through shared memory, and the warp
// holding the pivot row publishes it, scaled, for both.  Each step passes two
// 64-thread named barriers; the exchange slots are double-buffered by step
// parity, so no third barrier is needed.  Two walkers per CTA of 128 threads.
template <typename T>
struct RefreshInverseReg64 {
  static __device__ __forceinline__ void run(const double *__restrict__ gm, T *__restrict__ ginv,
                                             double *__restrict__ scal, int *__restrict__ status, int n, int W,
                                             int check_drift, double drift_tol, double *__restrict__ ginv64,
                                             const uint3 bid, const uint3 gdim) {
    assume_global(gm, ginv, scal, status);
    constexpr unsigned kFull = 0xffffffffu;
    __shared__ double s_prow[2][2][64];                 // [walker slot][parity][column]
    __shared__ unsigned long long s_key[2][2][2];       // [slot][parity][half]
    __shared__ int s_idx[2][2][2];
    __shared__ double s_val[2][2][2];
    __shared__ int s_q[2][64];                          // step at which each row was pivoted
    __shared__ double s_red[2][2][2];                   // [slot][half][gmax, dmax]
    const int lane = threadIdx.x & 31, wi = threadIdx.x >> 5, slot = wi >> 1, h = wi & 1;
    const int w = bid.x * 2 + slot;
    if (w >= W) return;  // both warps of the walker leave; its barriers involve no one else
    const int bar_id = 1 + slot;
    const int c0 = lane, c1 = lane + 32, r0 = 32 * h;
    const double *Gw = gm + (size_t)w * n * n;
    double a0[32], a1[32];
    double gmax = 0.0;
  #pragma unroll
    for (int i = 0; i < 32; ++i) {
      const int r = r0 + i;
      double v0 = r == c0 ? 1.0 : 0.0, v1 = r == c1 ? 1.0 : 0.0;
      if (r < n) {
        if (c0 < n) v0 = Gw[(size_t)r * n + c0];
        if (c1 < n) v1 = Gw[(size_t)r * n + c1];
        gmax = fmax(gmax, fmax(c0 < n ? fabs(v0) : 0.0, c1 < n ? fabs(v1) : 0.0));
      }
      a0[i] = v0;
      a1[i] = v1;
    }
    unsigned long long used = 0;
    int inversions = 0, myp0 = 0, myp1 = 0;
    PivotProduct pp;
    bool neg = false, ok = true;
    const unsigned long long rows_n = n >= 64 ? ~0ull : ((1ull << n) - 1ull);
    for (int k = 0; k < n; ++k) {
      const int par = k & 1, kl = k & 31;
      const bool hi = k >= 32;
      // this warp's rows of column k: lane i keeps f of row r0 + i
      double fme = 0.0;
      if (hi) {
  #pragma unroll
        for (int i = 0; i < 32; ++i) {
          const double t = __shfl_sync(kFull, a1[i], kl);
          if (lane == i) fme = t;
        }
      } else {
  #pragma unroll
        for (int i = 0; i < 32; ++i) {
          const double t = __shfl_sync(kFull, a0[i], kl);
          if (lane == i) fme = t;
        }
      }
      const int myrow = r0 + lane;
      unsigned long long key = (myrow < n && !((used >> myrow) & 1ull))
                                   ? static_cast<unsigned long long>(__double_as_longlong(fme)) & 0x7fffffffffffffffull
                                   : 0ull;
      int pi = myrow;
  #pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long k2 = __shfl_xor_sync(kFull, key, o);
        const int i2 = __shfl_xor_sync(kFull, pi, o);
        if (k2 > key || (k2 == key && i2 < pi)) {
          key = k2;
          pi = i2;
        }
      }
      const double pval = __shfl_sync(kFull, fme, pi - r0);
      if (lane == 0) {
        s_key[slot][par][h] = key;
        s_idx[slot][par][h] = pi;
        s_val[slot][par][h] = pval;
      }
      asm volatile("bar.sync %0, 64;" ::"r"(bar_id) : "memory");
      // the better of the two halves (the lower rows on ties)
      const unsigned long long ka = s_key[slot][par][0], kb = s_key[slot][par][1];
      const int hp = kb > ka ? 1 : 0;
      const int p = s_idx[slot][par][hp];
      const double pv = s_val[slot][par][hp];
      ok = ok && !((used >> p) & 1ull) && pv != 0.0 && isfinite(pv);
      inversions += __popcll(~used & rows_n & ((1ull << p) - 1ull));
      used |= 1ull << p;
      if (k == c0) myp0 = p;
      if (k == c1) myp1 = p;
      if (h == 0 && lane == 0) s_q[slot][p] = k;
      pp.mul(pv);
      neg ^= pv < 0.0;
      const double ip = recip_newton(pv);
      if ((p >> 5) == h) {
        // this warp holds the pivot row: publish it scaled (column k: 1/p)
        const int pl = p & 31;
        double x0 = 0.0, x1 = 0.0;
  #pragma unroll
        for (int i = 0; i < 32; ++i)
          if (i == pl) {
            x0 = a0[i];
            x1 = a1[i];
          }
        s_prow[slot][par][c0] = c0 == k ? ip : x0 * ip;
        s_prow[slot][par][c1] = c1 == k ? ip : x1 * ip;
      }
      asm volatile("bar.sync %0, 64;" ::"r"(bar_id) : "memory");
      const double v0 = s_prow[slot][par][c0], v1 = s_prow[slot][par][c1];
      const bool k0 = c0 == k, k1 = c1 == k;
      if (hi) {
  #pragma unroll
        for (int i = 0; i < 32; ++i) {
          const int r = r0 + i;
          if (r >= n) break;  // warp-uniform
          const double fi = __shfl_sync(kFull, a1[i], kl);
          a0[i] = r == p ? v0 : fma(-fi, v0, a0[i]);
          a1[i] = r == p ? v1 : fma(-fi, v1, k1 ? 0.0 : a1[i]);
        }
      } else {
  #pragma unroll
        for (int i = 0; i < 32; ++i) {
          const int r = r0 + i;
          if (r >= n) break;  // warp-uniform
          const double fi = __shfl_sync(kFull, a0[i], kl);
          a0[i] = r == p ? v0 : fma(-fi, v0, k0 ? 0.0 : a0[i]);
          a1[i] = r == p ? v1 : fma(-fi, v1, a1[i]);
        }
      }
    }
    asm volatile("bar.sync %0, 64;" ::"r"(bar_id) : "memory");  // s_q complete
    // inverse[k][p_c] = result[p_k][c]: row r of the result goes to row q_r
    T *gi = ginv + (size_t)w * n * n;
    double dmax = 0.0;
    if (ok) {
  #pragma unroll
      for (int i = 0; i < 32; ++i) {
        const int r = r0 + i;
        if (r >= n) break;
        const size_t row = (size_t)s_q[slot][r] * n;
        if (c0 < n) {
          if (check_drift) dmax = fmax(dmax, fabs(a0[i] - static_cast<double>(gi[row + myp0])));
          gi[row + myp0] = static_cast<T>(a0[i]);
          if (ginv64) ginv64[(size_t)w * n * n + row + myp0] = a0[i];
        }
        if (c1 < n) {
          if (check_drift) dmax = fmax(dmax, fabs(a1[i] - static_cast<double>(gi[row + myp1])));
          gi[row + myp1] = static_cast<T>(a1[i]);
          if (ginv64) ginv64[(size_t)w * n * n + row + myp1] = a1[i];
        }
      }
    }
  #pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      dmax = fmax(dmax, __shfl_xor_sync(kFull, dmax, o));
      gmax = fmax(gmax, __shfl_xor_sync(kFull, gmax, o));
    }
    if (lane == 0) {
      s_red[slot][h][0] = gmax;
      s_red[slot][h][1] = dmax;
    }
    asm volatile("bar.sync %0, 64;" ::"r"(bar_id) : "memory");
    if (h != 0 || lane != 0) return;
    gmax = fmax(s_red[slot][0][0], s_red[slot][1][0]);
    dmax = fmax(s_red[slot][0][1], s_red[slot][1][1]);
    double *sw = scal + (size_t)w * S_STRIDE;
    if (!ok) {
      status[w] |= JAGP_WS_SINGULAR;
      sw[S_LOGDET] = -INFINITY;
      sw[S_SIGN] = 0.0;
      return;
    }
    sw[S_LOGDET] = pp.log_abs();
    sw[S_SIGN] = (neg != (inversions & 1)) ? -1.0 : 1.0;
    if (check_drift) {
      const double drift = dmax * gmax;
      sw[S_DRIFT] = drift;
      if (!(drift <= drift_tol)) status[w] |= JAGP_WS_DRIFT;
    }
}
};
template <typename T>
__global__ void __launch_bounds__(128) k_refresh_inverse_reg64(const double *__restrict__ gm, T *__restrict__ ginv,
                                                               double *__restrict__ scal, int *__restrict__ status,
                                                               int n, int W, int check_drift, double drift_tol,
                                                               double *__restrict__ ginv64) {
  RefreshInverseReg64<T>::run(gm, ginv, scal, status, n, W, check_drift, drift_tol, ginv64, blockIdx, gridDim);
}

// In-place Gauss-Jordan (N_up > 32): step k scales the pivot row, stores
// -f_i / p in column k and updates the rest, so the inverse takes the place of
// G~ (half the work of eliminating [G~ | I]); the row swaps of the partial
// pivoting become column swaps of the result, undone in reverse order at the
// end.  Rows i < rs are copied to shared memory (row pitch n + 1); the others
// are overwritten in global memory, where they stay L2-resident while the CTA
// works on them (the launch keeps one CTA per SM, so the resident rows of all
// CTAs together fit in L2).
template <typename T>
struct RefreshInverseInplace {
  static __device__ __forceinline__ void run(double *__restrict__ gm, T *__restrict__ ginv, double *__restrict__ scal,
                                             int *__restrict__ status, int n, int rs, int check_drift,
                                             double drift_tol, double *__restrict__ ginv64, const uint3 bid,
                                             const uint3 gdim) {
    assume_global(gm, ginv, scal, status);
    extern __shared__ double sm[];
    const int ld = n + 1;
    double *prow = sm + (size_t)rs * ld;          // n: the scaled pivot row
    double *f = prow + n;                         // n: column k before the step
    int *perm = reinterpret_cast<int *>(f + n);   // n: pivot row of each step
    __shared__ int s_piv;
    __shared__ double s_pv;
    __shared__ double red[32];
    const int tid = threadIdx.x, bs = blockDim.x, w = bid.x, lane = tid & 31, warp = tid >> 5, nw = bs >> 5;
    double *const G = gm + (size_t)w * n * n;
    auto R = [&](int i) -> double * { return i < rs ? sm + (size_t)i * ld : G + (size_t)i * n; };
    double gmax = 0.0;
    for (int idx = tid; idx < n * n; idx += bs) {
      const int i = idx / n, j = idx - i * n;
      const double v = G[idx];
      gmax = fmax(gmax, fabs(v));
      if (i < rs) sm[(size_t)i * ld + j] = v;
    }
    PivotProduct pp;
    double sgn = 1.0;
    bool ok = true;
    __syncthreads();
    for (int k = 0; k < n; ++k) {
      if (warp == 0) {
        double best = -1.0;
        int bi = k;
        for (int i = k + lane; i < n; i += 32) {
          const double v = fabs(R(i)[k]);
          if (v > best) {
            best = v;
            bi = i;
          }
        }
  #pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
          const double ob = __shfl_xor_sync(0xffffffffu, best, o);
          const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
          if (ob > best || (ob == best && oi < bi)) {
            best = ob;
            bi = oi;
          }
        }
        if (lane == 0) {
          s_piv = bi;
          s_pv = R(bi)[k];
        }
      }
      __syncthreads();
      const int p = s_piv;
      const double pv = s_pv;
      if (!(pv != 0.0) || !isfinite(pv)) {
        ok = false;
        break;
      }
      if (p != k) {
        double *Rk = R(k), *Rp = R(p);
        for (int j = tid; j < n; j += bs) {
          const double t = Rk[j];
          Rk[j] = Rp[j];
          Rp[j] = t;
        }
        sgn = -sgn;
      }
      pp.mul(pv);
      if (pv < 0.0) sgn = -sgn;
      if (tid == 0) perm[k] = p;
      __syncthreads();
      const double ip = recip_newton(pv);
      {
        const double *Rk = R(k);
        for (int j = tid; j < n; j += bs) prow[j] = j == k ? ip : Rk[j] * ip;
      }
      for (int i = tid; i < n; i += bs) f[i] = i == k ? 0.0 : R(i)[k];
      __syncthreads();
      for (int i = warp; i < n; i += nw) {
        double *Ai = R(i);
        if (i == k) {
          for (int j = lane; j < n; j += 32) Ai[j] = prow[j];
        } else {
          // eight columns per lane at a time, all loads before the stores, so
          // that they are in flight together (Ai may be global memory)
          const double fi = f[i];
          for (int jb = 0; jb < n; jb += 256) {
            double v[8];
  #pragma unroll
            for (int t = 0; t < 8; ++t) {
              const int j = jb + lane + 32 * t;
              v[t] = j < n ? Ai[j] : 0.0;
            }
  #pragma unroll
            for (int t = 0; t < 8; ++t) {
              const int j = jb + lane + 32 * t;
              if (j < n) Ai[j] = fma(-fi, prow[j], v[t]);
            }
          }
        }
      }
      __syncthreads();
      // column k of the other rows: -f_i / p (replacing what the update left there)
      for (int i = tid; i < n; i += bs)
        if (i != k) R(i)[k] = -f[i] * ip;
      __syncthreads();
    }
    T *gi = ginv + (size_t)w * n * n;
    if (!ok) {
      if (tid == 0) {
        status[w] |= JAGP_WS_SINGULAR;
        scal[(size_t)w * S_STRIDE + S_LOGDET] = -INFINITY;
        scal[(size_t)w * S_STRIDE + S_SIGN] = 0.0;
      }
      return;
    }
    for (int k = n - 1; k >= 0; --k) {
      const int p = perm[k];
      if (p != k)
        for (int i = tid; i < n; i += bs) {
          double *Ai = R(i);
          const double t = Ai[k];
          Ai[k] = Ai[p];
          Ai[p] = t;
        }
      __syncthreads();
    }
    double dmax = 0.0;
    for (int idx = tid; idx < n * n; idx += bs) {
      const double v = R(idx / n)[idx % n];
      if (check_drift) dmax = fmax(dmax, fabs(v - static_cast<double>(gi[idx])));
      gi[idx] = static_cast<T>(v);
      if (ginv64) ginv64[(size_t)w * n * n + idx] = v;
    }
    for (int o = 16; o > 0; o >>= 1) {
      dmax = fmax(dmax, __shfl_xor_sync(0xffffffffu, dmax, o));
      gmax = fmax(gmax, __shfl_xor_sync(0xffffffffu, gmax, o));
    }
    if (lane == 0) {
      red[warp] = dmax;
      red[16 + warp] = gmax;
    }
    __syncthreads();
    if (tid == 0) {
      double d = 0.0, g = 0.0;
      for (int q = 0; q < nw; ++q) {
        d = fmax(d, red[q]);
        g = fmax(g, red[16 + q]);
      }
      scal[(size_t)w * S_STRIDE + S_LOGDET] = pp.log_abs();
      scal[(size_t)w * S_STRIDE + S_SIGN] = sgn;
      if (check_drift) {
        const double drift = d * g;
        scal[(size_t)w * S_STRIDE + S_DRIFT] = drift;
        if (!(drift <= drift_tol)) status[w] |= JAGP_WS_DRIFT;
      }
    }
}
};
template <typename T>
__global__ void __launch_bounds__(512) k_refresh_inverse_inplace(double *__restrict__ gm, T *__restrict__ ginv,
                                                                 double *__restrict__ scal, int *__restrict__ status,
                                                                 int n, int rs, int check_drift, double drift_tol,
                                                                 double *__restrict__ ginv64) {
  RefreshInverseInplace<T>::run(gm, ginv, scal, status, n, rs, check_drift, drift_tol, ginv64, blockIdx, gridDim);
}


template <typename T>
cudaError_t launch_refresh_inverse(double *gm, T *ginv, double *scal, int *status, int n, int W,
                                   int check_drift, double drift_tol, cudaStream_t st, double *ginv64) {
  if (W <= 0) return cudaSuccess;
  const size_t aux = (size_t)n * (2 * sizeof(double) + sizeof(int));
  const size_t inplace_smem = (size_t)n * (n + 1) * sizeof(double) + aux;
  if (n > 32 && n <= 64) {
    return launch_or_record<RefreshInverseReg64<T>, 128>(k_refresh_inverse_reg64<T>, dim3((W + 1) / 2), dim3(128), 0,
                                                         st, gm, ginv, scal, status, n, W, check_drift, drift_tol,
                                                         ginv64);
  }
  if (n > 32 && inplace_smem <= kRefreshSmemMax) {
    return launch_or_record<RefreshInverseInplace<T>, 512>(k_refresh_inverse_inplace<T>, dim3(W), dim3(256),
                                                           inplace_smem, st, gm, ginv, scal, status, n, n, check_drift,
                                                           drift_tol, ginv64);
  }
  if (n > 32) {
    // as many leading rows in shared memory as fit in kRefreshSmemMax (which
    // also keeps one CTA per SM), the rest in global memory
    const int rs = static_cast<int>((kRefreshSmemMax - aux) / ((size_t)(n + 1) * sizeof(double)));
    const size_t smem = (size_t)rs * (n + 1) * sizeof(double) + aux;
    return launch_or_record<RefreshInverseInplace<T>, 512>(k_refresh_inverse_inplace<T>, dim3(W), dim3(512), smem, st,
                                                           gm, ginv, scal, status, n, rs, check_drift, drift_tol,
                                                           ginv64);
  }
  if (n <= 32) {
    // 4 warps per CTA, 32 / NM walkers per warp
    if (n <= 8)
      return launch_or_record<RefreshInverseReg<T, 8>, 128>(k_refresh_inverse_reg<T, 8>, dim3((W + 15) / 16),
                                                            dim3(128), 0, st, gm, ginv, scal, status, n, W,
                                                            check_drift, drift_tol, ginv64);
    if (n <= 16)
      return launch_or_record<RefreshInverseReg<T, 16>, 128>(k_refresh_inverse_reg<T, 16>, dim3((W + 7) / 8),
                                                             dim3(128), 0, st, gm, ginv, scal, status, n, W,
                                                             check_drift, drift_tol, ginv64);
    return launch_or_record<RefreshInverseReg<T, 32>, 128>(k_refresh_inverse_reg<T, 32>, dim3((W + 3) / 4), dim3(128),
                                                           0, st, gm, ginv, scal, status, n, W, check_drift,
                                                           drift_tol, ginv64);
  }
  return cudaErrorInvalidValue;
}
template cudaError_t launch_refresh_inverse<double>(double *, double *, double *, int *, int, int, int, double,
                                                    cudaStream_t, double *);
template cudaError_t launch_refresh_inverse<float>(double *, float *, double *, int *, int, int, int, double,
                                                   cudaStream_t, double *);

// ---------------------------------------------------------------------------
// Kinetic-energy contraction vectors.  D = det G~ is linear in row i (up
// electron i) and in column j (down electron j), so
//   grad_i D / D = sum_mu grad phi_mu(r_i) M[i][mu],
//   up:   M[i]       = sum_j Ginv[j][i] Bt[j]      (Bt[j] = lambda phi(r_j^dn) or c^{(l)})
//   down: M[n_up + j] = sum_i Ginv[j][i] A_up[i]   (A_up[i] = phi(r_i^up)^T lambda)
// and the same M with the Laplacians.  One CTA per (walker, 64 columns).
// ---------------------------------------------------------------------------
template <typename T>
struct Mmat {
  static __device__ __forceinline__ void run(DevSystem s, const T *__restrict__ ginv, const T *__restrict__ bt,
                                             const T *__restrict__ a_up, T *__restrict__ mbuf, const uint3 bid,
                                             const uint3 gdim) {
    assume_global(ginv, bt, a_up, mbuf);
    extern __shared__ double smd[];
    T *sm = reinterpret_cast<T *>(smd);
    const int n = s.n_up, nd = s.n_dn, N = s.N, L = s.L;
    const int w = bid.y, c0 = bid.x * 64, tid = threadIdx.x;
    T *Gs = sm;              // n*n
    T *Bs = Gs + n * n;      // n*64
    T *As = Bs + n * 64;     // n*64
    for (int t = tid; t < n * n; t += 256) Gs[t] = ginv[(size_t)w * n * n + t];
    for (int t = tid; t < n * 64; t += 256) {
      const int j = t >> 6, c = t & 63;
      const bool in = c0 + c < L;
      Bs[t] = in ? bt[((size_t)w * n + j) * L + c0 + c] : T(0);
      As[t] = in ? a_up[((size_t)w * n + j) * L + c0 + c] : T(0);
    }
    __syncthreads();
    for (int idx = tid; idx < N * 64; idx += 256) {
      const int e = idx >> 6, c = idx & 63;
      if (c0 + c >= L) continue;
      T acc = T(0);
      if (e < n) {
        for (int j = 0; j < n; ++j) acc = fma(Gs[j * n + e], Bs[j * 64 + c], acc);
      } else {
        const int jj = e - n;
        for (int i = 0; i < n; ++i) acc = fma(Gs[jj * n + i], As[i * 64 + c], acc);
      }
      (void)nd;
      mbuf[((size_t)w * N + e) * L + c0 + c] = acc;
    }
}
};
template <typename T>
__global__ void __launch_bounds__(256) k_mmat(DevSystem s, const T *__restrict__ ginv, const T *__restrict__ bt,
                                              const T *__restrict__ a_up, T *__restrict__ mbuf) {
  Mmat<T>::run(s, ginv, bt, a_up, mbuf, blockIdx, gridDim);
}

// The same contraction for N_up too large to stage G~^{-1} whole: 64 x 64
// output tiles (electrons x basis functions), 4 x 4 per thread, the sum over
// j (or i) in chunks of 16 in the same order as above.  Up tiles come first in
// blockIdx.y, then down tiles, so that no tile mixes the two formulas.
template <typename T>
struct MmatTiled {
  static __device__ __forceinline__ void run(DevSystem s, const T *__restrict__ ginv, const T *__restrict__ bt,
                                             const T *__restrict__ a_up, T *__restrict__ mbuf, const uint3 bid,
                                             const uint3 gdim) {
    assume_global(ginv, bt, a_up, mbuf);
    __shared__ T Xs[16][64];  // Xs[k][e]: G~^{-1}[k][e] (up) or G~^{-1}[e][k] (down)
    __shared__ T Ys[16][64];  // Ys[k][c]: Bt[k][c] (up) or A_up[k][c] (down)
    const int n = s.n_up, N = s.N, L = s.L;
    const int w = bid.z, c0 = bid.x * 64, tid = threadIdx.x;
    const int up_tiles = (n + 63) / 64;
    const bool up = (int)bid.y < up_tiles;
    const int e0 = up ? bid.y * 64 : (bid.y - up_tiles) * 64;  // within the species
    const int ne = up ? n : s.n_dn;
    const T *G = ginv + (size_t)w * n * n;
    const T *Y = (up ? bt : a_up) + (size_t)w * n * L;
    const int tx = tid & 15, ty = tid >> 4;
    T acc[4][4];
  #pragma unroll
    for (int a = 0; a < 4; ++a)
  #pragma unroll
      for (int b = 0; b < 4; ++b) acc[a][b] = T(0);
    for (int k0 = 0; k0 < n; k0 += 16) {
  #pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int idx = tid + q * 256;
        const int kk = idx >> 6, col = idx & 63, k = k0 + kk;
        T xv = T(0), yv = T(0);
        if (k < n) {
          const int e = e0 + col;
          if (e < ne) xv = up ? G[(size_t)k * n + e] : G[(size_t)e * n + k];
          if (c0 + col < L) yv = Y[(size_t)k * L + c0 + col];
        }
        Xs[kk][col] = xv;
        Ys[kk][col] = yv;
      }
      __syncthreads();
  #pragma unroll
      for (int kk = 0; kk < 16; ++kk) {
        T xa[4], yb[4];
  #pragma unroll
        for (int a = 0; a < 4; ++a) xa[a] = Xs[kk][ty * 4 + a];
  #pragma unroll
        for (int b = 0; b < 4; ++b) yb[b] = Ys[kk][tx * 4 + b];
  #pragma unroll
        for (int a = 0; a < 4; ++a)
  #pragma unroll
          for (int b = 0; b < 4; ++b) acc[a][b] = fma(xa[a], yb[b], acc[a][b]);
      }
      __syncthreads();
    }
    const int ebase = up ? 0 : n;
  #pragma unroll
    for (int a = 0; a < 4; ++a) {
      const int e = e0 + ty * 4 + a;
      if (e >= ne) continue;
      T *o = mbuf + ((size_t)w * N + ebase + e) * L;
  #pragma unroll
      for (int b = 0; b < 4; ++b) {
        const int c = c0 + tx * 4 + b;
        if (c < L) o[c] = acc[a][b];
      }
    }
}
};
template <typename T>
__global__ void __launch_bounds__(256) k_mmat_tiled(DevSystem s, const T *__restrict__ ginv, const T *__restrict__ bt,
                                                    const T *__restrict__ a_up, T *__restrict__ mbuf) {
  MmatTiled<T>::run(s, ginv, bt, a_up, mbuf, blockIdx, gridDim);
}

// The mixed path's M vectors for small N_up on the CUDA cores: the sums of
// k_mmat with the FP64 inverse of the last refresh (split into two floats)
// against the two-float tables, as compensated dot products (error-free
// products and sums, the errors summed apart; Ogita, Rump and Oishi 2005) with
// the cross terms of the low parts, so that M + M_lo keeps about twice the
// FP32 precision.  One CTA per (walker, 64 columns).
struct MmatDw {
  static __device__ __forceinline__ void run(DevSystem s, const double *__restrict__ ginv64,
                                             const float *__restrict__ bt, const float *__restrict__ bt_lo,
                                             const float *__restrict__ a_up, const float *__restrict__ a_lo,
                                             float *__restrict__ mbuf, float *__restrict__ mlo, const uint3 bid,
                                             const uint3 gdim) {
    assume_global(ginv64, bt, bt_lo, a_up, a_lo, mbuf, mlo);
    extern __shared__ float smf[];
    const int n = s.n_up, N = s.N, L = s.L;
    const int w = bid.y, c0 = bid.x * 64, tid = threadIdx.x;
    float *Gh = smf, *Gl = Gh + n * n;              // n*n each
    float *Bh = Gl + n * n, *Bl = Bh + n * 64;       // n*64 each
    float *Ah = Bl + n * 64, *Al = Ah + n * 64;      // n*64 each
    for (int t = tid; t < n * n; t += 256) {
      const fdw v = dw_of(ginv64[(size_t)w * n * n + t]);
      Gh[t] = v.hi;
      Gl[t] = v.lo;
    }
    for (int t = tid; t < n * 64; t += 256) {
      const int j = t >> 6, c = t & 63;
      const bool in = c0 + c < L;
      const size_t src = ((size_t)w * n + j) * L + c0 + c;
      Bh[t] = in ? bt[src] : 0.0f;
      Bl[t] = in ? bt_lo[src] : 0.0f;
      Ah[t] = in ? a_up[src] : 0.0f;
      Al[t] = in ? a_lo[src] : 0.0f;
    }
    __syncthreads();
    for (int idx = tid; idx < N * 64; idx += 256) {
      const int e = idx >> 6, c = idx & 63;
      if (c0 + c >= L) continue;
      float sh = 0.0f, err = 0.0f;
      const bool upe = e < n;
      const int jj = e - n;
      for (int j = 0; j < n; ++j) {
        // up: Ginv[j][e] Bt[j][c]; down: Ginv[jj][j] A_up[j][c]
        const int gi = upe ? j * n + e : jj * n + j;
        const float gh = Gh[gi], gl = Gl[gi];
        const float bh = upe ? Bh[j * 64 + c] : Ah[j * 64 + c], bl = upe ? Bl[j * 64 + c] : Al[j * 64 + c];
        const fdw p = two_prod(gh, bh);
        const fdw q = two_sum(sh, p.hi);
        sh = q.hi;
        err = __fadd_rn(err, __fadd_rn(q.lo, __fadd_rn(p.lo, __fmaf_rn(gh, bl, __fmul_rn(gl, bh)))));
      }
      const fdw r = fast_two_sum(sh, err);
      const size_t o = ((size_t)w * N + e) * L + c0 + c;
      mbuf[o] = r.hi;
      mlo[o] = r.lo;
    }
}
};
__global__ void __launch_bounds__(256) k_mmat_dw(DevSystem s, const double *__restrict__ ginv64,
                                                 const float *__restrict__ bt, const float *__restrict__ bt_lo,
                                                 const float *__restrict__ a_up, const float *__restrict__ a_lo,
                                                 float *__restrict__ mbuf, float *__restrict__ mlo) {
  MmatDw::run(s, ginv64, bt, bt_lo, a_up, a_lo, mbuf, mlo, blockIdx, gridDim);
}

cudaError_t launch_mmat_dw(const DevSystem &s, const double *ginv64, const float *bt, const float *bt_lo,
                           const float *a_up, const float *a_lo, float *mbuf, float *mlo, int W, cudaStream_t st) {
  if (W <= 0) return cudaSuccess;
  const int n = s.n_up;
  const size_t smem = (size_t)(2 * n * n + 4 * n * 64) * sizeof(float);
  if (smem > kMmatSmemMax) return cudaErrorInvalidValue;
  dim3 grid((s.L + 63) / 64, W);
  return launch_or_record<MmatDw, 256>(k_mmat_dw, grid, dim3(256), smem, st, s, ginv64, bt, bt_lo, a_up, a_lo, mbuf,
                                       mlo);
}

template <typename T>
cudaError_t launch_mmat(const DevSystem &s, const T *ginv, const T *bt, const T *a_up, T *mbuf, int W,
                        cudaStream_t st) {
  if (W <= 0) return cudaSuccess;
  const int n = s.n_up;
  const size_t smem = (size_t)(n * n + 2 * n * 64) * sizeof(T);
  if (smem > kMmatSmemMax) {
    dim3 grid((s.L + 63) / 64, (n + 63) / 64 + (s.n_dn + 63) / 64, W);
    return launch_or_record<MmatTiled<T>, 256>(k_mmat_tiled<T>, grid, dim3(256), 0, st, s, ginv, bt, a_up, mbuf);
  }
  dim3 grid((s.L + 63) / 64, W);
  return launch_or_record<Mmat<T>, 256>(k_mmat<T>, grid, dim3(256), smem, st, s, ginv, bt, a_up, mbuf);
}
template cudaError_t launch_mmat<double>(const DevSystem &, const double *, const double *, const double *, double *,
                                         int, cudaStream_t);
template cudaError_t launch_mmat<float>(const DevSystem &, const float *, const float *, const float *, float *, int,
                                        cudaStream_t);

// the kernels of this file raise their shared-memory limit when first
// launched (launch_or_record)
cudaError_t setup_kernel_attributes() { return cudaSuccess; }

}  // namespace jagp
