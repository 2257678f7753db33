// k_forces.cu -- the finite-variance force estimator of Sec. "Atomic forces":
//   * the space-warp coordinate transformation (an electron at r moves with
//     nucleus a by Delta R_a omega_a(r), omega_a = kappa_a / sum_b kappa_b,
//     kappa(d) = 1/d^4), added to the adjoint's per-walker derivatives;
//   * the guiding function's regularisation ratio R(x) = (S sum |G~^{-1}|^2)^-theta
//     (Eq. R_r, S = min_i sum_j |G~_ij|^2) and the reweighting factor
//     W(x) = (R / max(R, eps))^2 (Eqs. regularization, reweighting);
//   * the seeds of the reweighted estimator <W F> / <W> for the adjoint.
// FP64 throughout, sums in a fixed order.
#include "jagp_launch.h"

namespace jagp {

namespace {

constexpr int kThreads = 128;

// Per walker: rbar_at[w][a] += sum_i omega_a(r_i) rbar[w][i] + sL_w / 2 sum_i grad omega_a(r_i)
// (the warp applied to the vector-Jacobian product sL d ln|Psi| + sE d e_L: the
// d/dr_i terms move with the nuclei, the Jacobian's half-log derivative carries sL)
__global__ void __launch_bounds__(kThreads) k_space_warp(DevSystem s, const double *__restrict__ r,
                                                          const double *__restrict__ rbar,
                                                          const double *__restrict__ sL,
                                                          double *__restrict__ rbar_at) {
  extern __shared__ double sm[];
  const int w = blockIdx.x, N = s.N, na = s.n_atoms, tid = threadIdx.x;
  double *xs = sm, *rb = xs + 3 * N, *ks = rb + 3 * N, *gs = ks + N;  // positions, rbar, sum kappa, sum grad kappa
  for (int t = tid; t < 3 * N; t += kThreads) {
    xs[t] = r[(size_t)w * N * 3 + t];
    rb[t] = rbar[(size_t)w * N * 3 + t];
  }
  __syncthreads();
  for (int i = tid; i < N; i += kThreads) {
    double k = 0.0, g0 = 0.0, g1 = 0.0, g2 = 0.0;
    for (int b = 0; b < na; ++b) {
      const double d0 = xs[3 * i] - s.R[3 * b], d1 = xs[3 * i + 1] - s.R[3 * b + 1], d2 = xs[3 * i + 2] - s.R[3 * b + 2];
      const double q = d0 * d0 + d1 * d1 + d2 * d2;
      const double k4 = 1.0 / (q * q), k6 = -4.0 / (q * q * q);
      k += k4;
      g0 = fma(k6, d0, g0);
      g1 = fma(k6, d1, g1);
      g2 = fma(k6, d2, g2);
    }
    ks[i] = k;
    gs[3 * i] = g0;
    gs[3 * i + 1] = g1;
    gs[3 * i + 2] = g2;
  }
  __syncthreads();
  const double hl = sL ? 0.5 * sL[w] : 0.0;
  for (int a = tid; a < na; a += kThreads) {
    double acc0 = 0.0, acc1 = 0.0, acc2 = 0.0;
    for (int i = 0; i < N; ++i) {
      const double d0 = xs[3 * i] - s.R[3 * a], d1 = xs[3 * i + 1] - s.R[3 * a + 1], d2 = xs[3 * i + 2] - s.R[3 * a + 2];
      const double q = d0 * d0 + d1 * d1 + d2 * d2;
      const double k4 = 1.0 / (q * q), k6 = -4.0 / (q * q * q);
      const double S = ks[i], iS = 1.0 / S;
      const double om = k4 * iS;
      // grad omega_a = (grad kappa_a S - kappa_a sum_b grad kappa_b) / S^2
      const double w0 = (k6 * d0 - om * gs[3 * i]) * iS, w1 = (k6 * d1 - om * gs[3 * i + 1]) * iS,
                   w2 = (k6 * d2 - om * gs[3 * i + 2]) * iS;
      acc0 += om * rb[3 * i] + hl * w0;
      acc1 += om * rb[3 * i + 1] + hl * w1;
      acc2 += om * rb[3 * i + 2] + hl * w2;
    }
    double *o = rbar_at + ((size_t)w * na + a) * 3;
    o[0] += acc0;
    o[1] += acc1;
    o[2] += acc2;
  }
}

// out[k] = sum_w in[w][k], k < n (fixed order over walkers)
__global__ void k_walker_sum(const double *__restrict__ in, int W, int n, double *__restrict__ out) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  double a = 0.0;
  for (int w = 0; w < W; ++w) a += in[(size_t)w * n + k];
  out[k] = a;
}

// R(x) and W(x) per walker from G~ (g, FP64) and G~^{-1} (ginv):
//   F = sum_jk Ginv_jk^2, S = min_i sum_j G_ij^2, R = (S F)^-theta,
//   W = (R / max(R, eps))^2.
template <typename T>
__global__ void __launch_bounds__(kThreads) k_guiding(const double *__restrict__ g, const T *__restrict__ ginv, int n,
                                                      double theta, double eps, double *__restrict__ Rout,
                                                      double *__restrict__ Wout) {
  __shared__ double red[kThreads];
  __shared__ double rmin[kThreads];
  const int w = blockIdx.x, tid = threadIdx.x;
  const double *G = g + (size_t)w * n * n;
  const T *A = ginv + (size_t)w * n * n;
  double f = 0.0;
  for (int t = tid; t < n * n; t += kThreads) {
    const double v = static_cast<double>(A[t]);
    f = fma(v, v, f);
  }
  double mn = INFINITY;
  for (int i = tid; i < n; i += kThreads) {
    double rs = 0.0;
    for (int j = 0; j < n; ++j) rs = fma(G[(size_t)i * n + j], G[(size_t)i * n + j], rs);
    mn = fmin(mn, rs);
  }
  red[tid] = f;
  rmin[tid] = mn;
  __syncthreads();
  for (int o = kThreads / 2; o > 0; o >>= 1) {
    if (tid < o) {
      red[tid] += red[tid + o];
      rmin[tid] = fmin(rmin[tid], rmin[tid + o]);
    }
    __syncthreads();
  }
  if (tid == 0) {
    const double R = pow(rmin[0] * red[0], -theta);
    const double q = R / fmax(R, eps);
    if (Rout) Rout[w] = R;
    if (Wout) Wout[w] = q * q;
  }
}

// Seeds of the reweighted force estimator <W F>_G / <W>_G (Eq. reweighting)
// for the adjoint: with weights u_w (NULL: all 1), ubar = sum u, E = sum u e / ubar,
//   sE_w = u_w / ubar,  sL_w = 2 u_w (e_w - E) / ubar.
__global__ void __launch_bounds__(kThreads) k_force_seeds(const double *__restrict__ e, const double *__restrict__ u,
                                                          int M, double *__restrict__ sL, double *__restrict__ sE,
                                                          double *__restrict__ mean_out) {
  __shared__ double a[kThreads], b[kThreads];
  const int tid = threadIdx.x;
  double su = 0.0, sue = 0.0;
  for (int i = tid; i < M; i += kThreads) {
    const double ui = u ? u[i] : 1.0;
    su += ui;
    sue = fma(ui, e[i], sue);
  }
  a[tid] = su;
  b[tid] = sue;
  __syncthreads();
  for (int o = kThreads / 2; o > 0; o >>= 1) {
    if (tid < o) {
      a[tid] += a[tid + o];
      b[tid] += b[tid + o];
    }
    __syncthreads();
  }
  const double ubar = a[0], E = b[0] / ubar;
  for (int i = tid; i < M; i += kThreads) {
    const double ui = u ? u[i] : 1.0;
    sE[i] = ui / ubar;
    sL[i] = 2.0 * ui * (e[i] - E) / ubar;
  }
  if (tid == 0 && mean_out) {
    mean_out[0] = E;
    mean_out[1] = ubar / M;
  }
}

}  // namespace

cudaError_t launch_space_warp(const DevSystem &s, const double *r, const double *rbar, const double *sL,
                              double *rbar_at, double *dR, int W, cudaStream_t st) {
  if (W <= 0) return cudaSuccess;
  // positions (3N), rbar (3N), sum kappa (N) and sum grad kappa (3N) per electron
  const size_t smem = (size_t)s.N * 10 * sizeof(double);
  if (smem > 200 * 1024) return cudaErrorInvalidValue;
  k_space_warp<<<W, kThreads, smem, st>>>(s, r, rbar, sL, rbar_at);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess || !dR) return e;
  const int n = 3 * s.n_atoms;
  k_walker_sum<<<(n + 127) / 128, 128, 0, st>>>(rbar_at, W, n, dR);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_guiding(const double *g, const T *ginv, int n, int W, double theta, double eps, double *R,
                           double *Wt, cudaStream_t st) {
  if (W <= 0) return cudaSuccess;
  k_guiding<T><<<W, kThreads, 0, st>>>(g, ginv, n, theta, eps, R, Wt);
  return cudaGetLastError();
}
template cudaError_t launch_guiding<double>(const double *, const double *, int, int, double, double, double *,
                                            double *, cudaStream_t);
template cudaError_t launch_guiding<float>(const double *, const float *, int, int, double, double, double *,
                                           double *, cudaStream_t);

cudaError_t launch_force_seeds(const double *e, const double *u, int M, double *sL, double *sE, double *mean_out,
                               cudaStream_t st) {
  if (M <= 0) return cudaSuccess;
  k_force_seeds<<<1, kThreads, 0, st>>>(e, u, M, sL, sE, mean_out);
  return cudaGetLastError();
}

cudaError_t setup_forces_attributes() {
  return cudaFuncSetAttribute(k_space_warp, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
}

}  // namespace jagp
