// k_energy.cu -- local energy e_L = H Psi / Psi (Sec. VMC, Eq. 1) for
// Psi = det(G~) exp(J):
//   lap_i Psi / Psi = lap_i D/D + 2 grad_i D/D . grad_i J + lap_i J + |grad_i J|^2,
//   e_L = -1/2 sum_i lap_i Psi/Psi - sum_{i,a} Z_a/r_ia + sum_{i<j} 1/r_ij + sum_{a<b} Z_a Z_b/R_ab.
#include <math.h>

#include "jagp_launch.h"

namespace jagp {

// ---------------------------------------------------------------------------
// Orbital gradients and Laplacians at every electron contracted with that
// electron's M vector (see k_mmat): one warp per electron, lanes over shells;
// the derivative tables are never stored.
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(256) k_kinetic(DevSystem s, const double *__restrict__ r,
                                                 const T *__restrict__ mbuf, double *__restrict__ kin,
                                                 int W) {
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
    const double *rr = r + pt * 3;
    const double px = rr[0], py = rr[1], pz = rr[2];
    const T *M = mbuf + pt * s.L;
    T tx = T(0), ty = T(0), tz = T(0), tl = T(0);
    for (int k = lane; k < s.n_shells; k += 32) {
      const double4 g = sh_geo[k];
      const int info = sh_info[k];
      T o[5][5];
      const int nc = shell_derivs<T>(info, g.w, px - g.x, py - g.y, pz - g.z, o);
      const int off = shell_off(info);
#pragma unroll
      for (int c = 0; c < 5; ++c) {
        if (c >= nc) break;
        const T m = M[off + c];
        tx = fma(o[c][1], m, tx);
        ty = fma(o[c][2], m, ty);
        tz = fma(o[c][3], m, tz);
        tl = fma(o[c][4], m, tl);
      }
    }
    // lane partials are summed in FP64
    const double gx = warp_sum(static_cast<double>(tx));
    const double gy = warp_sum(static_cast<double>(ty));
    const double gz = warp_sum(static_cast<double>(tz));
    const double lp = warp_sum(static_cast<double>(tl));
    if (lane == 0) {
      double *o = kin + pt * 4;
      o[0] = gx;
      o[1] = gy;
      o[2] = gz;
      o[3] = lp;
    }
  }
}

template <typename T>
cudaError_t launch_kinetic(const DevSystem &s, const double *r, const T *mbuf, double *kin, int W, cudaStream_t st) {
  if (W <= 0) return cudaSuccess;
  const long total = (long)W * s.N;
  long blocks = (total + 7) / 8;
  if (blocks > 152 * 16) blocks = 152 * 16;
  const size_t smem = (size_t)s.n_shells * (sizeof(double4) + sizeof(int));
  k_kinetic<T><<<(int)blocks, 256, smem, st>>>(s, r, mbuf, kin, W);
  return cudaGetLastError();
}
template cudaError_t launch_kinetic<double>(const DevSystem &, const double *, const double *, double *, int,
                                            cudaStream_t);
template cudaError_t launch_kinetic<float>(const DevSystem &, const double *, const float *, double *, int,
                                           cudaStream_t);

// ---------------------------------------------------------------------------
// Jastrow derivatives, kinetic assembly and the Coulomb terms: one CTA per walker.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(128) k_elocal(DevSystem s, const double *__restrict__ r,
                                                const double *__restrict__ kin, double *__restrict__ eL,
                                                double *__restrict__ parts) {
  const int w = blockIdx.x, N = s.N, tid = threadIdx.x;
  extern __shared__ double xs[];
  for (int t = tid; t < N * 3; t += blockDim.x) xs[t] = r[(size_t)w * N * 3 + t];
  __syncthreads();
  double tkin = 0.0, vee = 0.0, vei = 0.0;
  for (int e = tid; e < N; e += blockDim.x) {
    const double ex = xs[3 * e], ey = xs[3 * e + 1], ez = xs[3 * e + 2];
    double gJx = 0.0, gJy = 0.0, gJz = 0.0, lJ = 0.0;
    for (int a = 0; a < s.n_atoms; ++a) {
      const double dx = ex - s.R[3 * a], dy = ey - s.R[3 * a + 1], dz = ez - s.R[3 * a + 2];
      const double rr = sqrt(dx * dx + dy * dy + dz * dz);
      vei -= s.Z[a] / rr;
      if (s.use_j1) {
        double fp, fpp;
        j1_d(s.c1[a], s.b_ea, rr, &fp, &fpp);
        const double q = fp / rr;
        gJx += q * dx;
        gJy += q * dy;
        gJz += q * dz;
        lJ += fpp + 2.0 * q;
      }
    }
    for (int k = 0; k < N; ++k) {
      if (k == e) continue;
      const double dx = ex - xs[3 * k], dy = ey - xs[3 * k + 1], dz = ez - xs[3 * k + 2];
      const double rr = sqrt(dx * dx + dy * dy + dz * dz);
      if (k > e) vee += 1.0 / rr;
      if (s.use_j2) {
        double kk, bb;
        j2_params(s, (e < s.n_up) == (k < s.n_up), &kk, &bb);
        const double q1 = 1.0 + bb * rr;
        const double vp = 1.0 / (kk * q1 * q1);
        const double vpp = -2.0 * bb / (kk * q1 * q1 * q1);
        const double q = vp / rr;
        gJx += q * dx;
        gJy += q * dy;
        gJz += q * dz;
        lJ += vpp + 2.0 * q;
      }
    }
    const double *kd = kin + ((size_t)w * N + e) * 4;
    const double t = kd[3] + lJ + 2.0 * (kd[0] * gJx + kd[1] * gJy + kd[2] * gJz) +
                     (gJx * gJx + gJy * gJy + gJz * gJz);
    tkin += -0.5 * t;
  }
  __shared__ double red[3][4];
  tkin = warp_sum(tkin);
  vee = warp_sum(vee);
  vei = warp_sum(vei);
  if ((tid & 31) == 0) {
    red[0][tid >> 5] = tkin;
    red[1][tid >> 5] = vee;
    red[2][tid >> 5] = vei;
  }
  __syncthreads();
  if (tid == 0) {
    double a = 0.0, b = 0.0, c = 0.0;
    for (int q = 0; q < (int)(blockDim.x >> 5); ++q) {
      a += red[0][q];
      b += red[1][q];
      c += red[2][q];
    }
    eL[w] = a + b + c + s.v_ii;
    if (parts) {
      parts[(size_t)w * 4 + 0] = a;
      parts[(size_t)w * 4 + 1] = b;
      parts[(size_t)w * 4 + 2] = c;
      parts[(size_t)w * 4 + 3] = s.v_ii;
    }
  }
}

cudaError_t launch_elocal(const DevSystem &s, const double *r, const double *kin, double *eL, double *parts, int W,
                          cudaStream_t st) {
  if (W <= 0) return cudaSuccess;
  k_elocal<<<W, 128, (size_t)s.N * 3 * sizeof(double), st>>>(s, r, kin, eL, parts);
  return cudaGetLastError();
}

cudaError_t setup_energy_attributes() {
  cudaError_t e = cudaFuncSetAttribute(k_kinetic<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(k_kinetic<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
}

}  // namespace jagp
