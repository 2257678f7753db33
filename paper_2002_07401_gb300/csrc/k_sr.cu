// k_sr.cu -- stochastic reconfiguration (Sec. "Stochastic reconfiguration",
// Eqs. SRupdate, sr and the diagonal shift of S) on the GPU:
//   * per-walker log-derivatives O_k = d ln|Psi| / d alpha_k (Sec.
//     "Derivatives with respect to variational parameters") for every entry
//     of lambda and the three Jastrow parameters;
//   * the regularised SR step dalpha = Delta (S + eps diag S)^{-1} f with
//     S = cov(O, O), f = -2 cov(e_L, O), solved by conjugate gradients without
//     forming S: every product S v is two passes over the M x P samples,
//     (1/M) O_c^T (O_c v) with O_c = O - Obar (the paper's matrix-free solve).
// FP64 throughout; every sum in a fixed order, so repeated calls agree bit for
// bit.  The passes over O are bound by HBM bandwidth.
#include "jagp_launch.h"

namespace jagp {

namespace {

constexpr int kThreads = 256;

// fixed-order tree sum over a CTA of kThreads threads
__device__ double cta_sum(double v, double *sh) {
  sh[threadIdx.x] = v;
  __syncthreads();
  for (int o = kThreads / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
    __syncthreads();
  }
  const double r = sh[0];
  __syncthreads();
  return r;
}

// ---------------------------------------------------------------------------
// Per-walker products with a shared leading (contraction) index:
//   Out[w][a][b] = sum_{k < K} X[w][k][a] Y[w][k][b],  a < Ma, b < Nb.
// X rows have pitch ldx, Y rows pitch ldy, Out rows pitch ldo; walker w's
// blocks start at X + w xw, Y + w yw, Out + w ow.  64 x 64 output tiles, 4 x 4
// per thread, the sum over k in chunks of 16 staged through shared memory
// (coalesced row reads of X and Y).
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kThreads) k_bgemm_tn(const double *__restrict__ X, size_t xw, int ldx,
                                                       const double *__restrict__ Y, size_t yw, int ldy, int K,
                                                       int Ma, int Nb, double *__restrict__ Out, size_t ow,
                                                       long long ldo) {
  __shared__ double Xs[16][64];
  __shared__ double Ys[16][64];
  const int w = blockIdx.z, a0 = blockIdx.y * 64, b0 = blockIdx.x * 64, tid = threadIdx.x;
  const int tx = tid & 15, ty = tid >> 4;
  const double *Xw = X + (size_t)w * xw, *Yw = Y + (size_t)w * yw;
  double acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0.0;
  for (int k0 = 0; k0 < K; k0 += 16) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int idx = tid + q * kThreads, kk = idx >> 6, col = idx & 63, k = k0 + kk;
      Xs[kk][col] = (k < K && a0 + col < Ma) ? Xw[(size_t)k * ldx + a0 + col] : 0.0;
      Ys[kk][col] = (k < K && b0 + col < Nb) ? Yw[(size_t)k * ldy + b0 + col] : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < 16; ++kk) {
      double xa[4], yb[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) xa[i] = Xs[kk][ty * 4 + i];
#pragma unroll
      for (int j = 0; j < 4; ++j) yb[j] = Ys[kk][tx * 4 + j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fma(xa[i], yb[j], acc[i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int a = a0 + ty * 4 + i;
    if (a >= Ma) continue;
    double *o = Out + (size_t)w * ow + (size_t)a * ldo;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int b = b0 + tx * 4 + j;
      if (b < Nb) o[b] = acc[i][j];
    }
  }
}

// d ln|Psi| / d (b_ea, b_para, b_anti) of each walker into O[w][off + 0..2]
__global__ void __launch_bounds__(128) k_sr_jastrow(DevSystem s, const double *__restrict__ r, double *__restrict__ O,
                                                    long long ldo, long long off) {
  __shared__ double red[3][4];
  const int w = blockIdx.x, N = s.N, tid = threadIdx.x;
  const double *x = r + (size_t)w * N * 3;
  double pe = 0.0, pp = 0.0, pa = 0.0;
  for (int e = tid; e < N; e += blockDim.x) {
    const double ex = x[3 * e], ey = x[3 * e + 1], ez = x[3 * e + 2];
    if (s.use_j1)
      for (int a = 0; a < s.n_atoms; ++a) {
        const double dx = ex - s.R[3 * a], dy = ey - s.R[3 * a + 1], dz = ez - s.R[3 * a + 2];
        pe += j1_db(s.c1[a], s.b_ea, sqrt(dx * dx + dy * dy + dz * dz));
      }
    if (s.use_j2)
      for (int k = e + 1; k < N; ++k) {
        const double dx = ex - x[3 * k], dy = ey - x[3 * k + 1], dz = ez - x[3 * k + 2];
        const double rr = sqrt(dx * dx + dy * dy + dz * dz);
        const bool same = (e < s.n_up) == (k < s.n_up);
        double kk, bb;
        j2_params(s, same, &kk, &bb);
        const double q = 1.0 + bb * rr;
        const double vdb = -rr * rr / (kk * q * q);
        if (same && !s.j2_si)
          pp += vdb;
        else
          pa += vdb;
      }
  }
  pe = warp_sum(pe);
  pp = warp_sum(pp);
  pa = warp_sum(pa);
  if ((tid & 31) == 0) {
    red[0][tid >> 5] = pe;
    red[1][tid >> 5] = pp;
    red[2][tid >> 5] = pa;
  }
  __syncthreads();
  if (tid < 3) {
    double t = 0.0;
    for (int q = 0; q < (int)(blockDim.x >> 5); ++q) t += red[tid][q];
    O[(size_t)w * ldo + off + tid] = t;
  }
}

// ---------------------------------------------------------------------------
// Column reductions over the M samples (rows) of O [M][ldo]:
//   mode 0: out_k = sum_i t_i O_ik                       (t = NULL: t_i = 1)
//   mode 1: out_k = sum_i (O_ik - c_k)^2
// Rows are split into kRowChunks slabs (partials [kRowChunks][P]) summed in a
// fixed order by k_sr_colsum_finish, which also scales by `scale` and, in
// mode 0, subtracts c_k * tsum (the centred form sum_i t_i (O_ik - c_k)).
// Threads take consecutive columns, so every row read is coalesced.
// ---------------------------------------------------------------------------
constexpr int kRowChunks = 16;

__global__ void __launch_bounds__(kThreads) k_sr_colsum(const double *__restrict__ O, long long ldo, int M, int P,
                                                        const double *__restrict__ t, const double *__restrict__ c,
                                                        int mode, double *__restrict__ part) {
  const int k = blockIdx.x * kThreads + threadIdx.x, z = blockIdx.y;
  if (k >= P) return;
  const int rows = (M + kRowChunks - 1) / kRowChunks, i0 = z * rows, i1 = min(M, i0 + rows);
  double a = 0.0;
  if (mode == 0) {
    for (int i = i0; i < i1; ++i) a = fma(t ? t[i] : 1.0, O[(size_t)i * ldo + k], a);
  } else {
    const double ck = c[k];
    for (int i = i0; i < i1; ++i) {
      const double d = O[(size_t)i * ldo + k] - ck;
      a = fma(d, d, a);
    }
  }
  part[(size_t)z * P + k] = a;
}

__global__ void k_sr_colsum_finish(const double *__restrict__ part, int P, double scale, const double *__restrict__ c,
                                   const double *__restrict__ tsum, double *__restrict__ out) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= P) return;
  double a = 0.0;
  for (int z = 0; z < kRowChunks; ++z) a += part[(size_t)z * P + k];
  if (c && tsum) a -= c[k] * tsum[0];
  out[k] = a * scale;
}

// t_i = sum_k O_ik v_k - (Obar . v): one CTA per sample row; the scalar
// Obar . v (in dotc[0]) is formed once beforehand
__global__ void __launch_bounds__(kThreads) k_sr_rowdot(const double *__restrict__ O, long long ldo, int P,
                                                        const double *__restrict__ v, const double *__restrict__ dotc,
                                                        double *__restrict__ t) {
  __shared__ double sh[kThreads];
  const int i = blockIdx.x;
  const double *row = O + (size_t)i * ldo;
  double a = 0.0;
  for (int k = threadIdx.x; k < P; k += kThreads) a = fma(row[k], v[k], a);
  const double s = cta_sum(a, sh);
  if (threadIdx.x == 0) t[i] = s - (dotc ? dotc[0] : 0.0);
}

// out[0] = sum_k x_k y_k (z given: sum_k x_k y_k z_k), one CTA, fixed order
__global__ void __launch_bounds__(kThreads) k_sr_dot(const double *__restrict__ x, const double *__restrict__ y,
                                                     const double *__restrict__ z, int n, double *__restrict__ out) {
  __shared__ double sh[kThreads];
  double a = 0.0;
  for (int k = threadIdx.x; k < n; k += kThreads) a = fma(x[k], z ? y[k] * z[k] : y[k], a);
  const double s = cta_sum(a, sh);
  if (threadIdx.x == 0) out[0] = s;
}

// out[0] = sum_i x_i, one CTA, fixed order
__global__ void __launch_bounds__(kThreads) k_sr_sum(const double *__restrict__ x, int n, double *__restrict__ out) {
  __shared__ double sh[kThreads];
  double a = 0.0;
  for (int k = threadIdx.x; k < n; k += kThreads) a += x[k];
  const double s = cta_sum(a, sh);
  if (threadIdx.x == 0) out[0] = s;
}

// the new r.z becomes the old one for the next iteration
__global__ void k_sr_roll(double *sc) {
  if (threadIdx.x == 0) sc[0] = sc[2];
}

// local energies: ebar = mean, ec_i = e_i - ebar, and sum_i ec_i (for the centred form)
__global__ void __launch_bounds__(kThreads) k_sr_center(const double *__restrict__ e, int M, double *__restrict__ ec,
                                                        double *__restrict__ scal) {
  __shared__ double sh[kThreads];
  double a = 0.0;
  for (int i = threadIdx.x; i < M; i += kThreads) a += e[i];
  const double mean = cta_sum(a, sh) / M;
  double b = 0.0;
  for (int i = threadIdx.x; i < M; i += kThreads) {
    ec[i] = e[i] - mean;
    b += ec[i];
  }
  const double s = cta_sum(b, sh);
  if (threadIdx.x == 0) {
    scal[0] = mean;
    scal[1] = s;
  }
}

// preconditioned CG vector updates.  dinv_k = 1 / S'_kk (0 for a parameter
// whose samples do not vary: it stays at 0)
__global__ void k_sr_cg_init(const double *__restrict__ f, const double *__restrict__ diag, double eps, int P,
                             double *__restrict__ dinv, double *__restrict__ x, double *__restrict__ r,
                             double *__restrict__ z, double *__restrict__ p) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= P) return;
  const double d = diag[k] * (1.0 + eps);
  const double di = d > 0.0 ? 1.0 / d : 0.0;
  dinv[k] = di;
  x[k] = 0.0;
  r[k] = di > 0.0 ? f[k] : 0.0;
  z[k] = r[k] * di;
  p[k] = z[k];
}

// q = S' p from u = (1/M) O_c^T t:  q_k = u_k + eps diag_k p_k (0 where dinv = 0)
__global__ void k_sr_cg_apply(const double *__restrict__ u, const double *__restrict__ diag,
                              const double *__restrict__ dinv, const double *__restrict__ p, double eps, int P,
                              double *__restrict__ q) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= P) return;
  q[k] = dinv[k] > 0.0 ? u[k] + eps * diag[k] * p[k] : 0.0;
}

// x += a p, r -= a q, z = dinv r with a = rz / pq (device scalars)
__global__ void k_sr_cg_step(const double *__restrict__ p, const double *__restrict__ q,
                             const double *__restrict__ dinv, const double *__restrict__ sc, int P,
                             double *__restrict__ x, double *__restrict__ r, double *__restrict__ z) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= P) return;
  const double a = sc[1] != 0.0 ? sc[0] / sc[1] : 0.0;  // rz / pq
  x[k] = fma(a, p[k], x[k]);
  r[k] = fma(-a, q[k], r[k]);
  z[k] = r[k] * dinv[k];
}

// p = z + (rz_new / rz_old) p
__global__ void k_sr_cg_dir(const double *__restrict__ z, const double *__restrict__ sc, int P,
                            double *__restrict__ p) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= P) return;
  const double beta = sc[0] != 0.0 ? sc[2] / sc[0] : 0.0;
  p[k] = fma(beta, p[k], z[k]);
}

__global__ void k_sr_scale(const double *__restrict__ x, double delta, int P, double *__restrict__ out) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k < P) out[k] = delta * x[k];
}

inline int blocks_for(long n) { return (int)((n + kThreads - 1) / kThreads); }

}  // namespace

cudaError_t launch_bgemm_tn(const double *X, size_t xw, int ldx, const double *Y, size_t yw, int ldy, int K, int Ma,
                            int Nb, double *Out, size_t ow, long long ldo, int W, cudaStream_t st) {
  if (W <= 0 || Ma <= 0 || Nb <= 0) return cudaSuccess;
  dim3 grid((Nb + 63) / 64, (Ma + 63) / 64, W);
  k_bgemm_tn<<<grid, kThreads, 0, st>>>(X, xw, ldx, Y, yw, ldy, K, Ma, Nb, Out, ow, ldo);
  return cudaGetLastError();
}

cudaError_t launch_sr_jastrow(const DevSystem &s, const double *r, double *O, long long ldo, long long off, int W,
                              cudaStream_t st) {
  if (W <= 0) return cudaSuccess;
  k_sr_jastrow<<<W, 128, 0, st>>>(s, r, O, ldo, off);
  return cudaGetLastError();
}

// workspace of the SR solve (doubles)
SrLayout sr_layout(int M, int P) {
  SrLayout l;
  size_t o = 0;
  auto take = [&](size_t n) { size_t r = o; o += (n + 31) / 32 * 32; return r; };
  l.obar = take(P);
  l.diag = take(P);
  l.dinv = take(P);
  l.x = take(P);
  l.r = take(P);
  l.z = take(P);
  l.p = take(P);
  l.q = take(P);
  l.u = take(P);
  l.part = take((size_t)kRowChunks * P);
  l.ec = take(M);
  l.t = take(M);
  l.sc = take(32);
  l.total = o;
  return l;
}

cudaError_t sr_prepare(const double *O, long long ldo, const double *e, int M, int P, double *w, const SrLayout &L,
                       double *f, cudaStream_t st) {
  const dim3 cgrid(blocks_for(P), kRowChunks);
  // Obar_k = (1/M) sum_i O_ik
  k_sr_colsum<<<cgrid, kThreads, 0, st>>>(O, ldo, M, P, nullptr, nullptr, 0, w + L.part);
  k_sr_colsum_finish<<<blocks_for(P), kThreads, 0, st>>>(w + L.part, P, 1.0 / M, nullptr, nullptr, w + L.obar);
  // diag S_kk = (1/M) sum_i (O_ik - Obar_k)^2
  k_sr_colsum<<<cgrid, kThreads, 0, st>>>(O, ldo, M, P, nullptr, w + L.obar, 1, w + L.part);
  k_sr_colsum_finish<<<blocks_for(P), kThreads, 0, st>>>(w + L.part, P, 1.0 / M, nullptr, nullptr, w + L.diag);
  // f_k = -(2/M) sum_i (e_i - ebar)(O_ik - Obar_k)
  k_sr_center<<<1, kThreads, 0, st>>>(e, M, w + L.ec, w + L.sc + 8);
  k_sr_colsum<<<cgrid, kThreads, 0, st>>>(O, ldo, M, P, w + L.ec, nullptr, 0, w + L.part);
  k_sr_colsum_finish<<<blocks_for(P), kThreads, 0, st>>>(w + L.part, P, -2.0 / M, w + L.obar, w + L.sc + 9, f);
  return cudaGetLastError();
}

cudaError_t sr_cg_init(const double *f, double eps, int P, double *w, const SrLayout &L, cudaStream_t st) {
  k_sr_cg_init<<<blocks_for(P), kThreads, 0, st>>>(f, w + L.diag, eps, P, w + L.dinv, w + L.x, w + L.r, w + L.z,
                                                    w + L.p);
  // sc[0] = r . z, sc[3] = r . r at the start
  k_sr_dot<<<1, kThreads, 0, st>>>(w + L.r, w + L.z, nullptr, P, w + L.sc);
  k_sr_dot<<<1, kThreads, 0, st>>>(w + L.r, w + L.r, nullptr, P, w + L.sc + 3);
  return cudaGetLastError();
}

// One preconditioned CG iteration on S' x = f, S' v = (1/M) O_c^T (O_c v) +
// eps diag(S) v.  Device scalars sc: [0] r.z, [1] p.q, [2] new r.z, [3] new
// r.r, [4] Obar.p, [5] sum_i t_i.
cudaError_t sr_cg_iter(const double *O, long long ldo, int M, int P, double eps, double *w, const SrLayout &L,
                       cudaStream_t st) {
  double *sc = w + L.sc;
  const dim3 cgrid(blocks_for(P), kRowChunks);
  // t = O_c p = O p - (Obar . p)
  k_sr_dot<<<1, kThreads, 0, st>>>(w + L.obar, w + L.p, nullptr, P, sc + 4);
  k_sr_rowdot<<<M, kThreads, 0, st>>>(O, ldo, P, w + L.p, sc + 4, w + L.t);
  // u = (1/M) O_c^T t = (1/M) (O^T t - Obar sum_i t_i)
  k_sr_sum<<<1, kThreads, 0, st>>>(w + L.t, M, sc + 5);
  k_sr_colsum<<<cgrid, kThreads, 0, st>>>(O, ldo, M, P, w + L.t, nullptr, 0, w + L.part);
  k_sr_colsum_finish<<<blocks_for(P), kThreads, 0, st>>>(w + L.part, P, 1.0 / M, w + L.obar, sc + 5, w + L.u);
  // q = S' p; a = r.z / p.q; x += a p, r -= a q, z = dinv r
  k_sr_cg_apply<<<blocks_for(P), kThreads, 0, st>>>(w + L.u, w + L.diag, w + L.dinv, w + L.p, eps, P, w + L.q);
  k_sr_dot<<<1, kThreads, 0, st>>>(w + L.p, w + L.q, nullptr, P, sc + 1);
  k_sr_cg_step<<<blocks_for(P), kThreads, 0, st>>>(w + L.p, w + L.q, w + L.dinv, sc, P, w + L.x, w + L.r, w + L.z);
  k_sr_dot<<<1, kThreads, 0, st>>>(w + L.r, w + L.z, nullptr, P, sc + 2);
  k_sr_dot<<<1, kThreads, 0, st>>>(w + L.r, w + L.r, nullptr, P, sc + 3);
  // p = z + (new r.z / old r.z) p
  k_sr_cg_dir<<<blocks_for(P), kThreads, 0, st>>>(w + L.z, sc, P, w + L.p);
  k_sr_roll<<<1, 32, 0, st>>>(sc);
  return cudaGetLastError();
}

cudaError_t sr_finish(double delta, int P, const double *w, const SrLayout &L, double *dalpha, cudaStream_t st) {
  k_sr_scale<<<blocks_for(P), kThreads, 0, st>>>(w + L.x, delta, P, dalpha);
  return cudaGetLastError();
}

}  // namespace jagp
