// k_adjoint.cu -- reverse-mode derivatives (Sec. "Derivatives of energy":
// algorithmic adjoint differentiation) of log|Psi| and of the local energy
// with respect to the pairing matrix lambda, the Jastrow parameters, the
// nuclear positions R_a and the electron positions r_i, for the force of
// Eq. forces:aad (without the space warp).
//
// Notation per walker: Bt_j = lambda phi(r_j^dn) (then the unpaired orbitals),
// A_i = lambda^T phi(r_i^up), G~ = Phi_up Bt^T, M_e the kinetic contraction
// vector of electron e (M_i = sum_j Ginv[j][i] Bt_j, M_{n+j} = sum_i Ginv[j][i] A_i),
// gD_e = grad phi(r_e)^T M_e, lD_e = lap phi(r_e) . M_e.  With seeds sL (on
// log|Psi|) and sE (on e_L) the adjoints are
//   Mbar_e = sE (-1/2 lap phi(r_e) - grad phi(r_e) . grad J_e)
//   H_ij   = Mbar_i . Bt_j + A_i . Mbar_{n+j}
//   Gbar   = -(Ginv H Ginv)^T + sL Ginv^T
//   Btbar_j = sum_i Gbar_ij phi_i + sum_i Ginv_ji Mbar_i,   Abar_i = sum_j Ginv_ji Mbar_{n+j}
//   phibar_i = sum_j Gbar_ij Bt_j + lambda Abar_i (up),     phibar_{n+j} = lambda^T Btbar_j (down)
//   lambdabar = sum_j Btbar_j phi_{n+j}^T + sum_i phi_i Abar_i^T
// and the orbital tables carry them to the positions through the orbital
// gradients, Hessians and gradients of the Laplacian.
#include <math.h>

#include "jagp_launch.h"

namespace jagp {

// ---------------------------------------------------------------------------
// orbital values, gradients, Hessians (xx, yy, zz, xy, yz, zx) and gradients
// of the Laplacian of one shell at displacement d (FP64)
// ---------------------------------------------------------------------------
__device__ __forceinline__ int shell_third(int info, double zeta, double dx, double dy, double dz, double val[5],
                                           double grad[5][3], double hess[5][6], double glap[5][3]) {
  const int l = shell_l(info);
  const double d[3] = {dx, dy, dz};
  const double r2 = dx * dx + dy * dy + dz * dz;
  double g, gg[3], Hg[3][3], lapg, glg[3];
  if (shell_rad(info)) {
    const double r = sqrt(r2);
    g = exp(-zeta * r);
    for (int a = 0; a < 3; ++a) gg[a] = -zeta * d[a] / r * g;
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 3; ++b)
        Hg[a][b] = (zeta * zeta * d[a] * d[b] / r2 + zeta * d[a] * d[b] / (r2 * r) - (a == b ? zeta / r : 0.0)) * g;
    lapg = (zeta * zeta - 2.0 * zeta / r) * g;
    const double q = (2.0 * zeta / (r2 * r) - zeta * (zeta * zeta - 2.0 * zeta / r) / r) * g;
    for (int a = 0; a < 3; ++a) glg[a] = q * d[a];
  } else {
    g = exp(-zeta * r2);
    for (int a = 0; a < 3; ++a) gg[a] = -2.0 * zeta * d[a] * g;
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 3; ++b) Hg[a][b] = (4.0 * zeta * zeta * d[a] * d[b] - (a == b ? 2.0 * zeta : 0.0)) * g;
    lapg = (4.0 * zeta * zeta * r2 - 6.0 * zeta) * g;
    const double q = (8.0 * zeta * zeta - 2.0 * zeta * (4.0 * zeta * zeta * r2 - 6.0 * zeta)) * g;
    for (int a = 0; a < 3; ++a) glg[a] = q * d[a];
  }
  const int nc = 2 * l + 1;
  for (int c = 0; c < nc; ++c) {
    double P, gP[3] = {0.0, 0.0, 0.0}, HP[3][3] = {{0.0, 0.0, 0.0}, {0.0, 0.0, 0.0}, {0.0, 0.0, 0.0}};
    if (l == 0) {
      P = 1.0;
    } else if (l == 1) {
      P = d[c];
      gP[c] = 1.0;
    } else if (c == 0) {
      P = dx * dy; gP[0] = dy; gP[1] = dx; HP[0][1] = HP[1][0] = 1.0;
    } else if (c == 1) {
      P = dy * dz; gP[1] = dz; gP[2] = dy; HP[1][2] = HP[2][1] = 1.0;
    } else if (c == 2) {
      P = dz * dx; gP[0] = dz; gP[2] = dx; HP[0][2] = HP[2][0] = 1.0;
    } else if (c == 3) {
      P = dx * dx - dy * dy; gP[0] = 2.0 * dx; gP[1] = -2.0 * dy; HP[0][0] = 2.0; HP[1][1] = -2.0;
    } else {
      P = 3.0 * dz * dz - r2; gP[0] = -2.0 * dx; gP[1] = -2.0 * dy; gP[2] = 4.0 * dz;
      HP[0][0] = -2.0; HP[1][1] = -2.0; HP[2][2] = 4.0;
    }
    val[c] = P * g;
    for (int q = 0; q < 3; ++q) grad[c][q] = gP[q] * g + P * gg[q];
    const int pa[6] = {0, 1, 2, 0, 1, 2}, pb[6] = {0, 1, 2, 1, 2, 0};
    for (int k = 0; k < 6; ++k) {
      const int a = pa[k], b = pb[k];
      hess[c][k] = HP[a][b] * g + gP[a] * gg[b] + gP[b] * gg[a] + P * Hg[a][b];
    }
    for (int q = 0; q < 3; ++q) {
      double t = 0.0;
      for (int p = 0; p < 3; ++p) t += HP[q][p] * gg[p] + gP[p] * Hg[q][p];
      glap[c][q] = 2.0 * t + gP[q] * lapg + P * glg[q];
    }
  }
  return nc;
}

// ---------------------------------------------------------------------------
// Jastrow derivatives of one radial function F(r), r = |d|: F', F'', F''' .
// J1 term of an atom: F = -c^3 u(c r), u = (1 - e^{-b s}) / (2b);
// J2 pair term: F = r / (k (1 + b r)).
// ---------------------------------------------------------------------------
__device__ __forceinline__ void j1_d3(double c, double b, double r, double *f1, double *f2, double *f3) {
  const double c4 = c * c * c * c;
  if (b == 0.0) {
    *f1 = -0.5 * c4;
    *f2 = 0.0;
    *f3 = 0.0;
    return;
  }
  const double e = exp(-b * c * r);
  *f1 = -0.5 * c4 * e;
  *f2 = 0.5 * c4 * c * b * e;
  *f3 = -0.5 * c4 * c * c * b * b * e;
}
__device__ __forceinline__ void j2_d3(double k, double b, double r, double *v1, double *v2, double *v3) {
  const double q = 1.0 + b * r;
  *v1 = 1.0 / (k * q * q);
  *v2 = -2.0 * b / (k * q * q * q);
  *v3 = 6.0 * b * b / (k * q * q * q * q);
}

// gradient F' dhat, Hessian-vector product H v, and gradient of the Laplacian
// (F''' + 2F''/r - 2F'/r^2) dhat of F(|d|)
__device__ __forceinline__ void radial_adj(double f1, double f2, double f3, const double d[3], double r,
                                           const double v[3], double hv[3], double glap[3]) {
  const double dh[3] = {d[0] / r, d[1] / r, d[2] / r};
  const double dv = dh[0] * v[0] + dh[1] * v[1] + dh[2] * v[2];
  const double gl = f3 + 2.0 * f2 / r - 2.0 * f1 / (r * r);
  for (int q = 0; q < 3; ++q) {
    hv[q] = f2 * dh[q] * dv + (f1 / r) * (v[q] - dh[q] * dv);
    glap[q] = gl * dh[q];
  }
}

// ---------------------------------------------------------------------------
// 1. Jastrow gradient at every electron and the kinetic adjoint vectors
//    Mbar_e = sE (-1/2 lap phi - grad phi . grad J_e); also the orbital values
//    at the down electrons (rows of dnphi).  One warp per electron.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_adj_kvec(DevSystem s, const double *__restrict__ r,
                                                  const double *__restrict__ sE, double *__restrict__ jg,
                                                  double *__restrict__ kbar, double *__restrict__ dnphi, int W) {
  extern __shared__ double4 sh_geo[];
  int *sh_info = reinterpret_cast<int *>(sh_geo + s.n_shells);
  for (int k = threadIdx.x; k < s.n_shells; k += blockDim.x) {
    sh_geo[k] = s.shell_geo[k];
    sh_info[k] = s.shell_info[k];
  }
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const long nwarps = (long)gridDim.x * (blockDim.x >> 5);
  const long total = (long)W * s.N;
  for (long pt = (long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); pt < total; pt += nwarps) {
    const int w = (int)(pt / s.N), e = (int)(pt % s.N);
    const double *xw = r + (size_t)w * s.N * 3;
    const double ex = xw[3 * e], ey = xw[3 * e + 1], ez = xw[3 * e + 2];
    // grad J_e (lanes over atoms and other electrons)
    double gx = 0.0, gy = 0.0, gz = 0.0;
    if (s.use_j1)
      for (int a = lane; a < s.n_atoms; a += 32) {
        const double dx = ex - s.R[3 * a], dy = ey - s.R[3 * a + 1], dz = ez - s.R[3 * a + 2];
        const double rr = sqrt(dx * dx + dy * dy + dz * dz);
        double fp, fpp;
        j1_d(s.c1[a], s.b_ea, rr, &fp, &fpp);
        gx += fp * dx / rr;
        gy += fp * dy / rr;
        gz += fp * dz / rr;
      }
    if (s.use_j2)
      for (int k = lane; k < s.N; k += 32) {
        if (k == e) continue;
        const double dx = ex - xw[3 * k], dy = ey - xw[3 * k + 1], dz = ez - xw[3 * k + 2];
        const double rr = sqrt(dx * dx + dy * dy + dz * dz);
        double kk, bb;
        j2_params(s, (e < s.n_up) == (k < s.n_up), &kk, &bb);
        const double q1 = 1.0 + bb * rr;
        const double vp = 1.0 / (kk * q1 * q1);
        gx += vp * dx / rr;
        gy += vp * dy / rr;
        gz += vp * dz / rr;
      }
    gx = warp_sum(gx);
    gy = warp_sum(gy);
    gz = warp_sum(gz);
    if (lane == 0) {
      jg[pt * 3] = gx;
      jg[pt * 3 + 1] = gy;
      jg[pt * 3 + 2] = gz;
    }
    const double se = sE ? sE[w] : 0.0;
    double *kb = kbar + pt * s.L;
    double *dp = (e >= s.n_up) ? dnphi + ((size_t)w * s.n_up + (e - s.n_up)) * s.L : nullptr;
    for (int k = lane; k < s.n_shells; k += 32) {
      const double4 g = sh_geo[k];
      const int info = sh_info[k];
      double o[5][5];
      const int nc = shell_derivs(info, g.w, ex - g.x, ey - g.y, ez - g.z, o);
      const int off = shell_off(info);
      for (int c = 0; c < nc; ++c) {
        kb[off + c] = se * (-0.5 * o[c][4] - (o[c][1] * gx + o[c][2] * gy + o[c][3] * gz));
        if (dp) dp[off + c] = o[c][0];
      }
    }
  }
}

// ---------------------------------------------------------------------------
// 2. Gbar = -(Ginv H Ginv)^T + sL Ginv^T with H = H1 + H2 (H2 only in the
//    first n_dn columns).  One CTA per walker, everything in shared memory.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_adj_gbar(const double *__restrict__ ginv, const double *__restrict__ h1,
                                                  const double *__restrict__ h2, const double *__restrict__ sL, int n,
                                                  int nd, double *__restrict__ gbar) {
  extern __shared__ double sm[];
  const int w = blockIdx.x, tid = threadIdx.x, bs = blockDim.x, nn = n * n;
  double *Gi = sm, *Hm = Gi + nn, *T = Hm + nn;
  const double *gw = ginv + (size_t)w * nn;
  for (int t = tid; t < nn; t += bs) {
    Gi[t] = gw[t];
    const int i = t / n, j = t - i * n;
    Hm[t] = h1[(size_t)w * nn + t] + (j < nd ? h2[(size_t)w * nn + (size_t)i * n + j] : 0.0);
  }
  __syncthreads();
  for (int t = tid; t < nn; t += bs) {  // T = Ginv H
    const int i = t / n, j = t - i * n;
    double a = 0.0;
    for (int k = 0; k < n; ++k) a = fma(Gi[i * n + k], Hm[k * n + j], a);
    T[t] = a;
  }
  __syncthreads();
  const double s = sL ? sL[w] : 0.0;
  for (int t = tid; t < nn; t += bs) {  // Gbar_ij = -(T Ginv)_ji + s Ginv_ji
    const int i = t / n, j = t - i * n;
    double a = 0.0;
    for (int k = 0; k < n; ++k) a = fma(T[j * n + k], Gi[k * n + i], a);
    gbar[(size_t)w * nn + t] = -a + s * Gi[j * n + i];
  }
}

// ---------------------------------------------------------------------------
// 3. row adjoints, per (walker, 64 columns):
//    Btbar_j = sum_i Gbar_ij phi_i + sum_i Ginv_ji Mbar_i        (j < n_dn)
//    Abar_i  = sum_j Ginv_ji Mbar_{n+j}                          (i < n)
//    phibar_i (partial) = sum_j Gbar_ij Bt_j                     (i < n)
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_adj_rows(DevSystem s, const double *__restrict__ ginv,
                                                  const double *__restrict__ gbar, const double *__restrict__ phi_up,
                                                  const double *__restrict__ bt, const double *__restrict__ kbar,
                                                  double *__restrict__ btbar, double *__restrict__ abar,
                                                  double *__restrict__ phibar) {
  extern __shared__ double sm[];
  const int n = s.n_up, nd = s.n_dn, N = s.N, L = s.L, nn = n * n;
  const int w = blockIdx.y, c0 = blockIdx.x * 64, tid = threadIdx.x;
  double *Gi = sm, *Gb = Gi + nn, *Ph = Gb + nn, *Bs = Ph + n * 64, *Ku = Bs + n * 64, *Kd = Ku + n * 64;
  for (int t = tid; t < nn; t += 256) {
    Gi[t] = ginv[(size_t)w * nn + t];
    Gb[t] = gbar[(size_t)w * nn + t];
  }
  for (int t = tid; t < n * 64; t += 256) {
    const int j = t >> 6, c = t & 63;
    const bool in = c0 + c < L;
    Ph[t] = in ? phi_up[((size_t)w * n + j) * L + c0 + c] : 0.0;
    Bs[t] = in ? bt[((size_t)w * n + j) * L + c0 + c] : 0.0;
    Ku[t] = in ? kbar[((size_t)w * N + j) * L + c0 + c] : 0.0;
    Kd[t] = (in && j < nd) ? kbar[((size_t)w * N + n + j) * L + c0 + c] : 0.0;
  }
  __syncthreads();
  for (int idx = tid; idx < n * 64; idx += 256) {
    const int i = idx >> 6, c = idx & 63;
    if (c0 + c >= L) continue;
    double pb = 0.0, ab = 0.0, bb = 0.0;
    for (int j = 0; j < n; ++j) pb = fma(Gb[i * n + j], Bs[j * 64 + c], pb);
    for (int j = 0; j < nd; ++j) ab = fma(Gi[j * n + i], Kd[j * 64 + c], ab);
    if (i < nd) {
      for (int k = 0; k < n; ++k) bb = fma(Gb[k * n + i], Ph[k * 64 + c], bb);
      for (int k = 0; k < n; ++k) bb = fma(Gi[i * n + k], Ku[k * 64 + c], bb);
      btbar[((size_t)w * n + i) * L + c0 + c] = bb;
    }
    abar[((size_t)w * n + i) * L + c0 + c] = ab;
    phibar[((size_t)w * n + i) * L + c0 + c] = pb;
  }
}

// ---------------------------------------------------------------------------
// 4. orbital tables -> positions.  One warp per electron e; per orbital mu:
//    c = phibar_mu grad phi_mu + M_mu (Hess phi_mu) gbarD + lbarD M_mu grad(lap phi_mu)
//    with gbarD = -sE grad J_e, lbarD = -sE / 2; rbar_e += c, Rbar_atom(mu) -= c.
//    The per-atom sums of the CTA's electrons go to part[w][blockIdx.x][atom].
// ---------------------------------------------------------------------------
constexpr int kAdjWarps = 8;

__global__ void __launch_bounds__(kAdjWarps * 32) k_adj_positions(
    DevSystem s, const double *__restrict__ r, const double *__restrict__ sE, const double *__restrict__ jg,
    const double *__restrict__ mbuf, const double *__restrict__ phibar_a, const double *__restrict__ phibar_b,
    const double *__restrict__ phibar_dn, const int *__restrict__ shell_atom, double *__restrict__ rbar,
    double *__restrict__ part) {
  extern __shared__ double sm[];
  double *Rb = sm;                                           // n_atoms * 3
  int *s_atom = reinterpret_cast<int *>(Rb + 3 * s.n_atoms);   // n_shells
  for (int t = threadIdx.x; t < 3 * s.n_atoms; t += blockDim.x) Rb[t] = 0.0;
  for (int t = threadIdx.x; t < s.n_shells; t += blockDim.x) s_atom[t] = shell_atom[t];
  __syncthreads();
  const int w = blockIdx.y, lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int e = blockIdx.x * kAdjWarps + warp;
  if (e < s.N) {
    const size_t pt = (size_t)w * s.N + e;
    const double ex = r[pt * 3], ey = r[pt * 3 + 1], ez = r[pt * 3 + 2];
    const double se = sE ? sE[w] : 0.0;
    const double gb[3] = {-se * jg[pt * 3], -se * jg[pt * 3 + 1], -se * jg[pt * 3 + 2]};
    const double lb = -0.5 * se;
    const double *M = mbuf + pt * s.L;
    const bool up = e < s.n_up;
    const double *pa = up ? phibar_a + ((size_t)w * s.n_up + e) * s.L : phibar_dn + ((size_t)w * s.n_up + e - s.n_up) * s.L;
    const double *pb2 = up ? phibar_b + ((size_t)w * s.n_up + e) * s.L : nullptr;
    double re[3] = {0.0, 0.0, 0.0};
    for (int k = lane; k < s.n_shells; k += 32) {
      const double4 g = s.shell_geo[k];
      const int info = s.shell_info[k];
      double val[5], grad[5][3], hs[5][6], gl[5][3];
      const int nc = shell_third(info, g.w, ex - g.x, ey - g.y, ez - g.z, val, grad, hs, gl);
      const int off = shell_off(info);
      double c[3] = {0.0, 0.0, 0.0};
      for (int q = 0; q < nc; ++q) {
        const double pbar = pa[off + q] + (pb2 ? pb2[off + q] : 0.0);
        const double m = M[off + q];
        // Hessian (xx, yy, zz, xy, yz, zx) times gb
        const double h0 = hs[q][0] * gb[0] + hs[q][3] * gb[1] + hs[q][5] * gb[2];
        const double h1 = hs[q][3] * gb[0] + hs[q][1] * gb[1] + hs[q][4] * gb[2];
        const double h2 = hs[q][5] * gb[0] + hs[q][4] * gb[1] + hs[q][2] * gb[2];
        c[0] += pbar * grad[q][0] + m * h0 + lb * m * gl[q][0];
        c[1] += pbar * grad[q][1] + m * h1 + lb * m * gl[q][1];
        c[2] += pbar * grad[q][2] + m * h2 + lb * m * gl[q][2];
      }
      const int a = s_atom[k];
      atomicAdd(&Rb[3 * a], -c[0]);
      atomicAdd(&Rb[3 * a + 1], -c[1]);
      atomicAdd(&Rb[3 * a + 2], -c[2]);
      re[0] += c[0];
      re[1] += c[1];
      re[2] += c[2];
    }
    re[0] = warp_sum(re[0]);
    re[1] = warp_sum(re[1]);
    re[2] = warp_sum(re[2]);
    if (lane == 0) {
      rbar[pt * 3] = re[0];
      rbar[pt * 3 + 1] = re[1];
      rbar[pt * 3 + 2] = re[2];
    }
  }
  __syncthreads();
  double *po = part + ((size_t)w * gridDim.x + blockIdx.x) * 3 * s.n_atoms;
  for (int t = threadIdx.x; t < 3 * s.n_atoms; t += blockDim.x) po[t] = Rb[t];
}

// ---------------------------------------------------------------------------
// 5. Jastrow and Coulomb adjoints, Jastrow parameter derivatives.  One CTA per
//    walker; electrons first (their grad J adjoints in shared memory), then
//    atoms.  rbar[e] += ..., rbar_at[w][a] = ..., jpar[w][3] = ...
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(128) k_adj_jastrow(DevSystem s, const double *__restrict__ r,
                                                     const double *__restrict__ sL, const double *__restrict__ sE,
                                                     const double *__restrict__ jg, const double *__restrict__ kin,
                                                     double *__restrict__ rbar, double *__restrict__ rbar_at,
                                                     double *__restrict__ jpar) {
  extern __shared__ double sm[];
  const int w = blockIdx.x, N = s.N, tid = threadIdx.x, bs = blockDim.x;
  double *xs = sm, *gJb = xs + 3 * N;  // electron positions; adjoint of grad J_e
  const double sl = sL ? sL[w] : 0.0, se = sE ? sE[w] : 0.0;
  const double lJb = -0.5 * se;        // adjoint of lap J_e (the same for all e)
  for (int t = tid; t < 3 * N; t += bs) {
    xs[t] = r[(size_t)w * N * 3 + t];
    // gbarJ_e = -sE (gD_e + gJ_e)
    const int e = t / 3, q = t - 3 * e;
    gJb[t] = -se * (kin[((size_t)w * N + e) * 4 + q] + jg[((size_t)w * N + e) * 3 + q]);
  }
  __syncthreads();
  double pb_ea = 0.0, pb_para = 0.0, pb_anti = 0.0;
  for (int e = tid; e < N; e += bs) {
    const double *xe = xs + 3 * e;
    const double gje[3] = {jg[((size_t)w * N + e) * 3], jg[((size_t)w * N + e) * 3 + 1], jg[((size_t)w * N + e) * 3 + 2]};
    double re[3] = {sl * gje[0], sl * gje[1], sl * gje[2]};  // from J itself
    for (int a = 0; a < s.n_atoms; ++a) {
      const double d[3] = {xe[0] - s.R[3 * a], xe[1] - s.R[3 * a + 1], xe[2] - s.R[3 * a + 2]};
      const double rr = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
      const double z3 = s.Z[a] / (rr * rr * rr);
      for (int q = 0; q < 3; ++q) re[q] += se * z3 * d[q];  // V_ei
      if (s.use_j1) {
        double f1, f2, f3, hv[3], gl[3];
        j1_d3(s.c1[a], s.b_ea, rr, &f1, &f2, &f3);
        radial_adj(f1, f2, f3, d, rr, gJb + 3 * e, hv, gl);
        for (int q = 0; q < 3; ++q) re[q] += hv[q] + lJb * gl[q];
        pb_ea += sl * j1_db(s.c1[a], s.b_ea, rr);
      }
    }
    for (int k = 0; k < N; ++k) {
      if (k == e) continue;
      const double d[3] = {xe[0] - xs[3 * k], xe[1] - xs[3 * k + 1], xe[2] - xs[3 * k + 2]};
      const double rr = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
      const double r3 = 1.0 / (rr * rr * rr);
      for (int q = 0; q < 3; ++q) re[q] -= se * r3 * d[q];  // V_ee
      if (s.use_j2) {
        const bool same = (e < s.n_up) == (k < s.n_up);
        double kk, bb, v1, v2, v3, hv[3], gl[3];
        j2_params(s, same, &kk, &bb);
        j2_d3(kk, bb, rr, &v1, &v2, &v3);
        const double dg[3] = {gJb[3 * e] - gJb[3 * k], gJb[3 * e + 1] - gJb[3 * k + 1], gJb[3 * e + 2] - gJb[3 * k + 2]};
        radial_adj(v1, v2, v3, d, rr, dg, hv, gl);
        for (int q = 0; q < 3; ++q) re[q] += hv[q] + 2.0 * lJb * gl[q];
        if (k > e) {
          const double q1 = 1.0 + bb * rr;
          const double vdb = -rr * rr / (kk * q1 * q1);
          if (same && !s.j2_si) pb_para += sl * vdb;
          else pb_anti += sl * vdb;
        }
      }
    }
    for (int q = 0; q < 3; ++q) rbar[((size_t)w * N + e) * 3 + q] += re[q];
  }
  for (int a = tid; a < s.n_atoms; a += bs) {
    double ra[3] = {0.0, 0.0, 0.0};
    for (int e = 0; e < N; ++e) {
      const double *xe = xs + 3 * e;
      const double d[3] = {xe[0] - s.R[3 * a], xe[1] - s.R[3 * a + 1], xe[2] - s.R[3 * a + 2]};
      const double rr = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
      const double z3 = s.Z[a] / (rr * rr * rr);
      for (int q = 0; q < 3; ++q) ra[q] -= se * z3 * d[q];
      if (s.use_j1) {
        double f1, f2, f3, hv[3], gl[3];
        j1_d3(s.c1[a], s.b_ea, rr, &f1, &f2, &f3);
        radial_adj(f1, f2, f3, d, rr, gJb + 3 * e, hv, gl);
        for (int q = 0; q < 3; ++q) ra[q] -= hv[q] + lJb * gl[q] + sl * f1 * d[q] / rr;
      }
    }
    for (int b = 0; b < s.n_atoms; ++b) {  // V_ii
      if (b == a) continue;
      const double d[3] = {s.R[3 * a] - s.R[3 * b], s.R[3 * a + 1] - s.R[3 * b + 1], s.R[3 * a + 2] - s.R[3 * b + 2]};
      const double rr = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
      for (int q = 0; q < 3; ++q) ra[q] -= se * s.Z[a] * s.Z[b] * d[q] / (rr * rr * rr);
    }
    for (int q = 0; q < 3; ++q) rbar_at[((size_t)w * s.n_atoms + a) * 3 + q] = ra[q];
  }
  // Jastrow parameter adjoints (from log|Psi| only): block sums
  __shared__ double red[3][4];
  pb_ea = warp_sum(pb_ea);
  pb_para = warp_sum(pb_para);
  pb_anti = warp_sum(pb_anti);
  if ((tid & 31) == 0) {
    red[0][tid >> 5] = pb_ea;
    red[1][tid >> 5] = pb_para;
    red[2][tid >> 5] = pb_anti;
  }
  __syncthreads();
  if (tid == 0) {
    double a0 = 0.0, a1 = 0.0, a2 = 0.0;
    for (int q = 0; q < (bs >> 5); ++q) {
      a0 += red[0][q];
      a1 += red[1][q];
      a2 += red[2][q];
    }
    jpar[(size_t)w * 3] = a0;
    jpar[(size_t)w * 3 + 1] = a1;
    jpar[(size_t)w * 3 + 2] = a2;
  }
}

// ---------------------------------------------------------------------------
// 6. per-walker nuclear adjoints: rbar_at[w] += sum of the orbital partials;
//    then the totals over walkers (fixed order) for R and the Jastrow params.
// ---------------------------------------------------------------------------
__global__ void k_adj_reduce_walker(const double *__restrict__ part, int nparts, int n_atoms,
                                    double *__restrict__ rbar_at, int W) {
  const long total = (long)W * n_atoms * 3;
  for (long t = blockIdx.x * (long)blockDim.x + threadIdx.x; t < total; t += (long)gridDim.x * blockDim.x) {
    const long w = t / (n_atoms * 3), q = t % (n_atoms * 3);
    double a = rbar_at[t];
    for (int p = 0; p < nparts; ++p) a += part[((size_t)w * nparts + p) * 3 * n_atoms + q];
    rbar_at[t] = a;
  }
}

__global__ void k_adj_reduce_total(const double *__restrict__ per_w, int W, int width, double *__restrict__ out) {
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < width; q += gridDim.x * blockDim.x) {
    double a = 0.0;
    for (int w = 0; w < W; ++w) a += per_w[(size_t)w * width + q];
    out[q] = a;
  }
}

// ---------------------------------------------------------------------------
// 7. lambdabar = sum_rows U[row]^T V[row] for two stacked row sets; split over
//    row ranges (blockIdx.z), partial sums to part[z][L][L].
//    Set 1: U = Btbar rows (w, j < n_dn), V = phi(r_j^dn) rows;
//    set 2: U = Phi_up rows (w, i < n_up), V = Abar rows.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_adj_lambda(const double *__restrict__ btbar,
                                                    const double *__restrict__ dnphi,
                                                    const double *__restrict__ phi_up, const double *__restrict__ abar,
                                                    int W, int n, int nd, int L, int rows_per_z,
                                                    double *__restrict__ part) {
  __shared__ double Us[16][64], Vs[16][64];
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int m0 = blockIdx.y * 64, n0 = blockIdx.x * 64;
  const long rows1 = (long)W * nd, rows_all = rows1 + (long)W * n;
  const long r0 = (long)blockIdx.z * rows_per_z;
  const long r1 = min(rows_all, r0 + rows_per_z);
  double acc[4][4] = {};
  for (long rb = r0; rb < r1; rb += 16) {
    for (int t = tid; t < 16 * 64; t += 256) {
      const int rr = t >> 6, c = t & 63;
      const long row = rb + rr;
      double u = 0.0, v = 0.0;
      if (row < r1) {
        const double *U, *V;
        if (row < rows1) {
          const long w = row / nd, j = row % nd;
          U = btbar + ((size_t)w * n + j) * L;
          V = dnphi + ((size_t)w * n + j) * L;
        } else {
          const long q = row - rows1, w = q / n, i = q % n;
          U = phi_up + ((size_t)w * n + i) * L;
          V = abar + ((size_t)w * n + i) * L;
        }
        if (m0 + c < L) u = U[m0 + c];
        if (n0 + c < L) v = V[n0 + c];
      }
      Us[rr][c] = u;
      Vs[rr][c] = v;
    }
    __syncthreads();
    for (int k = 0; k < 16; ++k) {
      double a[4], b[4];
      for (int i = 0; i < 4; ++i) a[i] = Us[k][ty + 16 * i];
      for (int j = 0; j < 4; ++j) b[j] = Vs[k][tx + 16 * j];
      for (int i = 0; i < 4; ++i)
        for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }
  double *po = part + (size_t)blockIdx.z * L * L;
  for (int i = 0; i < 4; ++i)
    for (int j = 0; j < 4; ++j) {
      const int mu = m0 + ty + 16 * i, nu = n0 + tx + 16 * j;
      if (mu < L && nu < L) po[(size_t)mu * L + nu] = acc[i][j];
    }
}

__global__ void k_adj_lambda_sum(const double *__restrict__ part, int nz, int LL, double *__restrict__ out) {
  for (long t = blockIdx.x * (long)blockDim.x + threadIdx.x; t < LL; t += (long)gridDim.x * blockDim.x) {
    double a = 0.0;
    for (int z = 0; z < nz; ++z) a += part[(size_t)z * LL + t];
    out[t] = a;
  }
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
cudaError_t launch_adj_kvec(const DevSystem &s, const double *r, const double *sE, double *jg, double *kbar,
                            double *dnphi, int W, cudaStream_t st) {
  const long total = (long)W * s.N;
  long blocks = (total + 7) / 8;
  if (blocks > 152 * 16) blocks = 152 * 16;
  const size_t smem = (size_t)s.n_shells * (sizeof(double4) + sizeof(int));
  k_adj_kvec<<<(int)blocks, 256, smem, st>>>(s, r, sE, jg, kbar, dnphi, W);
  return cudaGetLastError();
}

cudaError_t launch_adj_gbar(const double *ginv, const double *h1, const double *h2, const double *sL, int n, int nd,
                            double *gbar, int W, cudaStream_t st) {
  const size_t smem = (size_t)3 * n * n * sizeof(double);
  k_adj_gbar<<<W, 256, smem, st>>>(ginv, h1, h2, sL, n, nd, gbar);
  return cudaGetLastError();
}

cudaError_t launch_adj_rows(const DevSystem &s, const double *ginv, const double *gbar, const double *phi_up,
                            const double *bt, const double *kbar, double *btbar, double *abar, double *phibar, int W,
                            cudaStream_t st) {
  const int n = s.n_up;
  const size_t smem = (size_t)(2 * n * n + 4 * n * 64) * sizeof(double);
  dim3 grid((s.L + 63) / 64, W);
  k_adj_rows<<<grid, 256, smem, st>>>(s, ginv, gbar, phi_up, bt, kbar, btbar, abar, phibar);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// N_up beyond shared-memory staging: the same adjoints of steps 2 and 3 as
// per-walker GEMMs (k_bgemm below) with Gbar kept transposed,
//   GbarT = sL Ginv - (Ginv H) Ginv,
//   Btbar = GbarT Phi_up + Ginv Mbar_up,   Abar = Ginv^T Mbar_dn,
//   phibar = GbarT^T Bt.
// ---------------------------------------------------------------------------
// C[w] = alpha op(A[w]) B[w] (+ C[w] when accumulate), op(A) = A or A^T, all
// row-major: op(A) M x K, B K x N, C M x N.  64 x 64 output tiles, 4 x 4 per
// thread, k in chunks of 16 (the k order of every output is 0, 1, ..., K-1).
template <bool TA>
__global__ void __launch_bounds__(256) k_bgemm(const double *__restrict__ A, size_t sa, int lda,
                                               const double *__restrict__ B, size_t sb, int ldb,
                                               double *__restrict__ C, size_t sc, int ldc, int M, int N, int K,
                                               double alpha, int accumulate) {
  __shared__ double As[16][65];  // As[k][i] = op(A)[i0 + i][k0 + k]
  __shared__ double Bs[16][65];  // Bs[k][c] = B[k0 + k][c0 + c]
  const int w = blockIdx.z, i0 = blockIdx.y * 64, c0 = blockIdx.x * 64, tid = threadIdx.x;
  const int tx = tid & 15, ty = tid >> 4;
  const double *Aw = A + (size_t)w * sa, *Bw = B + (size_t)w * sb;
  double acc[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) acc[a][b] = 0.0;
  for (int k0 = 0; k0 < K; k0 += 16) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int idx = tid + q * 256;
      double av = 0.0, bv = 0.0;
      if (TA) {  // op(A)[i][k] = A[k][i]: consecutive threads take consecutive i
        const int kk = idx >> 6, i = idx & 63;
        if (k0 + kk < K && i0 + i < M) av = Aw[(size_t)(k0 + kk) * lda + i0 + i];
        As[kk][i] = av;
      } else {   // op(A)[i][k] = A[i][k]: consecutive threads take consecutive k
        const int i = idx >> 4, kk = idx & 15;
        if (k0 + kk < K && i0 + i < M) av = Aw[(size_t)(i0 + i) * lda + k0 + kk];
        As[kk][i] = av;
      }
      const int kk = idx >> 6, c = idx & 63;
      if (k0 + kk < K && c0 + c < N) bv = Bw[(size_t)(k0 + kk) * ldb + c0 + c];
      Bs[kk][c] = bv;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < 16; ++kk) {
      double xa[4], yb[4];
#pragma unroll
      for (int a = 0; a < 4; ++a) xa[a] = As[kk][ty * 4 + a];
#pragma unroll
      for (int b = 0; b < 4; ++b) yb[b] = Bs[kk][tx * 4 + b];
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = fma(xa[a], yb[b], acc[a][b]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    const int i = i0 + ty * 4 + a;
    if (i >= M) continue;
    double *Cr = C + (size_t)w * sc + (size_t)i * ldc;
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      const int c = c0 + tx * 4 + b;
      if (c >= N) continue;
      Cr[c] = accumulate ? fma(alpha, acc[a][b], Cr[c]) : alpha * acc[a][b];
    }
  }
}

static cudaError_t bgemm(bool ta, const double *A, size_t sa, int lda, const double *B, size_t sb, int ldb, double *C,
                         size_t sc, int ldc, int M, int N, int K, double alpha, int accumulate, int W,
                         cudaStream_t st) {
  if (W <= 0 || M <= 0 || N <= 0) return cudaSuccess;
  dim3 grid((N + 63) / 64, (M + 63) / 64, W);
  if (ta)
    k_bgemm<true><<<grid, 256, 0, st>>>(A, sa, lda, B, sb, ldb, C, sc, ldc, M, N, K, alpha, accumulate);
  else
    k_bgemm<false><<<grid, 256, 0, st>>>(A, sa, lda, B, sb, ldb, C, sc, ldc, M, N, K, alpha, accumulate);
  return cudaGetLastError();
}

// H = H1 + H2 (H2 only in the first n_dn columns), in place in h1; GbarT = sL Ginv
__global__ void k_adj_gbar_init(const double *__restrict__ ginv, double *__restrict__ h1,
                                const double *__restrict__ h2, const double *__restrict__ sL, int n, int nd, int W,
                                double *__restrict__ gbarT) {
  const long nn = (long)n * n, total = (long)W * nn;
  for (long t = blockIdx.x * (long)blockDim.x + threadIdx.x; t < total; t += (long)gridDim.x * blockDim.x) {
    const int w = (int)(t / nn), j = (int)(t % n);
    if (j < nd) h1[t] += h2[t];
    gbarT[t] = (sL ? sL[w] : 0.0) * ginv[t];
  }
}

cudaError_t launch_adj_rows_gemm(const DevSystem &s, const double *ginv, double *h1, double *h2, const double *sL,
                                 const double *phi_up, const double *bt, const double *kbar, double *gbarT,
                                 double *btbar, double *abar, double *phibar, int W, cudaStream_t st) {
  const int n = s.n_up, nd = s.n_dn, N = s.N, L = s.L;
  const size_t nn = (size_t)n * n, nL = (size_t)n * L, NL = (size_t)N * L;
  long blocks = ((long)W * nn + 255) / 256;
  if (blocks > 152 * 16) blocks = 152 * 16;
  k_adj_gbar_init<<<(int)blocks, 256, 0, st>>>(ginv, h1, h2, sL, n, nd, W, gbarT);
  cudaError_t e = cudaGetLastError();
  // T = Ginv H (into h2), GbarT -= T Ginv
  if (!e) e = bgemm(false, ginv, nn, n, h1, nn, n, h2, nn, n, n, n, n, 1.0, 0, W, st);
  if (!e) e = bgemm(false, h2, nn, n, ginv, nn, n, gbarT, nn, n, n, n, n, -1.0, 1, W, st);
  // Btbar (rows j < n_dn) = GbarT Phi_up + Ginv Mbar_up
  if (!e && nd > 0) e = bgemm(false, gbarT, nn, n, phi_up, nL, L, btbar, nL, L, nd, L, n, 1.0, 0, W, st);
  if (!e && nd > 0) e = bgemm(false, ginv, nn, n, kbar, NL, L, btbar, nL, L, nd, L, n, 1.0, 1, W, st);
  // Abar = Ginv^T Mbar_dn (zero without down electrons)
  if (!e && nd > 0) e = bgemm(true, ginv, nn, n, kbar + nL, NL, L, abar, nL, L, n, L, nd, 1.0, 0, W, st);
  if (!e && nd == 0) e = cudaMemsetAsync(abar, 0, (size_t)W * nL * sizeof(double), st);
  // phibar = GbarT^T Bt
  if (!e) e = bgemm(true, gbarT, nn, n, bt, nL, L, phibar, nL, L, n, L, n, 1.0, 0, W, st);
  return e;
}

int adj_position_parts(const DevSystem &s) { return (s.N + kAdjWarps - 1) / kAdjWarps; }

cudaError_t launch_adj_positions(const DevSystem &s, const double *r, const double *sE, const double *jg,
                                 const double *mbuf, const double *phibar_a, const double *phibar_b,
                                 const double *phibar_dn, const int *shell_atom, double *rbar, double *part, int W,
                                 cudaStream_t st) {
  dim3 grid(adj_position_parts(s), W);
  const size_t smem = (size_t)3 * s.n_atoms * sizeof(double) + (size_t)s.n_shells * sizeof(int);
  k_adj_positions<<<grid, kAdjWarps * 32, smem, st>>>(s, r, sE, jg, mbuf, phibar_a, phibar_b, phibar_dn, shell_atom,
                                                      rbar, part);
  return cudaGetLastError();
}

cudaError_t launch_adj_jastrow(const DevSystem &s, const double *r, const double *sL, const double *sE,
                               const double *jg, const double *kin, double *rbar, double *rbar_at, double *jpar, int W,
                               cudaStream_t st) {
  const size_t smem = (size_t)6 * s.N * sizeof(double);
  k_adj_jastrow<<<W, 128, smem, st>>>(s, r, sL, sE, jg, kin, rbar, rbar_at, jpar);
  return cudaGetLastError();
}

cudaError_t launch_adj_reduce(const double *part, int nparts, int n_atoms, double *rbar_at, const double *jpar,
                              int W, double *dR, double *djas, cudaStream_t st) {
  const long total = (long)W * n_atoms * 3;
  long blocks = (total + 255) / 256;
  if (blocks > 152 * 8) blocks = 152 * 8;
  k_adj_reduce_walker<<<(int)blocks, 256, 0, st>>>(part, nparts, n_atoms, rbar_at, W);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  if (dR) {
    k_adj_reduce_total<<<(3 * n_atoms + 255) / 256, 256, 0, st>>>(rbar_at, W, 3 * n_atoms, dR);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  if (djas) {
    k_adj_reduce_total<<<1, 32, 0, st>>>(jpar, W, 3, djas);
    e = cudaGetLastError();
  }
  return e;
}

cudaError_t launch_adj_lambda(const double *btbar, const double *dnphi, const double *phi_up, const double *abar,
                              int W, int n, int nd, int L, double *part, int nz, double *dlam, cudaStream_t st) {
  const long rows = (long)W * (n + nd);
  const int rows_per_z = (int)(((rows + nz - 1) / nz + 15) / 16 * 16);
  dim3 grid((L + 63) / 64, (L + 63) / 64, nz);
  k_adj_lambda<<<grid, 256, 0, st>>>(btbar, dnphi, phi_up, abar, W, n, nd, L, rows_per_z, part);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const long LL = (long)L * L;
  long blocks = (LL + 255) / 256;
  if (blocks > 152 * 8) blocks = 152 * 8;
  k_adj_lambda_sum<<<(int)blocks, 256, 0, st>>>(part, nz, (int)LL, dlam);
  return cudaGetLastError();
}

cudaError_t launch_adj_lambda_sum(const double *part, int nz, int L, double *dlam, cudaStream_t st) {
  const long LL = (long)L * L;
  long blocks = (LL + 255) / 256;
  if (blocks > 152 * 8) blocks = 152 * 8;
  k_adj_lambda_sum<<<(int)blocks, 256, 0, st>>>(part, nz, (int)LL, dlam);
  return cudaGetLastError();
}

cudaError_t setup_adjoint_attributes() {
  const int big = 200 * 1024;
  cudaError_t e;
  if ((e = cudaFuncSetAttribute(k_adj_kvec, cudaFuncAttributeMaxDynamicSharedMemorySize, big))) return e;
  if ((e = cudaFuncSetAttribute(k_adj_gbar, cudaFuncAttributeMaxDynamicSharedMemorySize, big))) return e;
  if ((e = cudaFuncSetAttribute(k_adj_rows, cudaFuncAttributeMaxDynamicSharedMemorySize, big))) return e;
  return cudaFuncSetAttribute(k_adj_positions, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
}

}  // namespace jagp
