// k_energy.cu -- local energy e_L = H Psi / Psi (Sec. VMC, Eq. 1) for
// Psi = det(G~) exp(J):
//   lap_i Psi / Psi = lap_i D/D + 2 grad_i D/D . grad_i J + lap_i J + |grad_i J|^2,
//   e_L = -1/2 sum_i lap_i Psi/Psi - sum_{i,a} Z_a/r_ia + sum_{i<j} 1/r_ij + sum_{a<b} Z_a Z_b/R_ab.
#include <math.h>

#include <type_traits>

#include "j3.cuh"
#include "jagp_group.cuh"
#include "jagp_launch.h"

namespace jagp {

// ---------------------------------------------------------------------------
// Orbital gradients and Laplacians at every electron contracted with that
// electron's M vector (see k_mmat): one warp per electron, lanes over shells;
// the derivative tables are never stored.
//
// Per shell the contraction needs only S0 = sum_c M_c P_c and Sg = sum_c M_c
// grad P_c: the angular polynomials are harmonic and homogeneous of degree l
// (grad P . d = l P), so for the Gaussian g = e^{-zeta r^2}
//   sum_c M_c grad(P_c g) = g (Sg - 2 zeta S0 d),
//   sum_c M_c lap(P_c g)  = g S0 (4 zeta^2 r^2 - (4l + 6) zeta),
// and for the Slater g = e^{-zeta r}
//   sum_c M_c grad(P_c g) = g (Sg - zeta S0 d / r),
//   sum_c M_c lap(P_c g)  = g S0 (zeta^2 - 2 zeta (l + 1) / r).
//
// FP64 path: FP64 throughout.  FP32 path: the displacement, r^2 and the radial
// factor in double-word (FP32 instructions only, see dword.cuh) so that g is
// accurate before its rounding; the polynomial contraction in FP32.
// ---------------------------------------------------------------------------
template <typename T>
struct Kinetic {
  static __device__ __forceinline__ void run(DevSystem s, const double *__restrict__ r, const T *__restrict__ mbuf,
                                             double *__restrict__ kin, int W, const uint3 bid, const uint3 gdim) {
    assume_global(r, mbuf, kin);
    constexpr bool kDw = std::is_same<T, float>::value;
    extern __shared__ double4 sh_geo[];
    int *sh_info = reinterpret_cast<int *>(sh_geo + s.n_shells);
    float4 *sh_dw = reinterpret_cast<float4 *>(sh_geo);
    for (int k = threadIdx.x; k < s.n_shells; k += blockDim.x) {
      if constexpr (kDw) {
        sh_dw[2 * k] = s.shell_dw[2 * k];
        sh_dw[2 * k + 1] = s.shell_dw[2 * k + 1];
      } else {
        sh_geo[k] = s.shell_geo[k];
      }
      sh_info[k] = s.shell_info[k];
    }
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const long nwarps = (long)gdim.x * (blockDim.x >> 5);
    const long total = (long)W * s.N;
    for (long pt = (long)bid.x * (blockDim.x >> 5) + (threadIdx.x >> 5); pt < total; pt += nwarps) {
      const double *rr = r + pt * 3;
      const double px = rr[0], py = rr[1], pz = rr[2];
      fdw pd[3];
      if constexpr (kDw) {
        // one FP64 -> double-word conversion per lane, shared by shuffles
        const int kc = lane < 3 ? lane : 2;
        const fdw mine = dw_of(kc == 0 ? px : (kc == 1 ? py : pz));
  #pragma unroll
        for (int k = 0; k < 3; ++k)
          pd[k] = fdw{__shfl_sync(0xffffffffu, mine.hi, k), __shfl_sync(0xffffffffu, mine.lo, k)};
      }
      const T *M = mbuf + pt * s.L;
      T tx = T(0), ty = T(0), tz = T(0), tl = T(0);
      for (int k = lane; k < s.n_shells; k += 32) {
        const int info = sh_info[k];
        const int l = shell_l(info), off = shell_off(info), rad = shell_rad(info);
        T g, dx, dy, dz, r2, zeta, rinv = T(0);
        if constexpr (kDw) {
          const float4 gh = sh_dw[2 * k], gl = sh_dw[2 * k + 1];
          const DwDisp d = dw_displacement(pd, gh, gl);
          const fdw zw{gh.w, gl.w};
          const fdw rw = rad ? dw_sqrt(d.r2) : fdw{0.0f, 0.0f};
          g = dw_exp_neg(dw_neg(dw_mul(zw, rad ? rw : d.r2))).hi;
          dx = d.x.hi;
          dy = d.y.hi;
          dz = d.z.hi;
          r2 = d.r2.hi;
          zeta = gh.w;
          if (rad) rinv = 1.0f / rw.hi;
        } else {
          const double4 g4 = sh_geo[k];
          dx = px - g4.x;
          dy = py - g4.y;
          dz = pz - g4.z;
          r2 = dx * dx + dy * dy + dz * dz;
          zeta = g4.w;
          g = radial_factor(rad, zeta, r2);
          if (rad) rinv = 1.0 / sqrt(r2);
        }
        T S0, Sx, Sy, Sz;
        if (l == 0) {
          S0 = M[off];
          Sx = Sy = Sz = T(0);
        } else if (l == 1) {
          const T m0 = M[off], m1 = M[off + 1], m2 = M[off + 2];
          S0 = m0 * dx + m1 * dy + m2 * dz;
          Sx = m0;
          Sy = m1;
          Sz = m2;
        } else {
          const T m0 = M[off], m1 = M[off + 1], m2 = M[off + 2], m3 = M[off + 3], m4 = M[off + 4];
          S0 = m0 * dx * dy + m1 * dy * dz + m2 * dz * dx + m3 * (dx * dx - dy * dy) + m4 * (T(3) * dz * dz - r2);
          Sx = m0 * dy + m2 * dz + T(2) * (m3 - m4) * dx;
          Sy = m0 * dx + m1 * dz - T(2) * (m3 + m4) * dy;
          Sz = m1 * dy + m2 * dx + T(4) * m4 * dz;
        }
        T f, lapfac;
        if (rad) {
          f = -zeta * S0 * rinv;
          lapfac = zeta * zeta - T(2) * zeta * static_cast<T>(l + 1) * rinv;
        } else {
          f = T(-2) * zeta * S0;
          lapfac = T(4) * zeta * zeta * r2 - static_cast<T>(4 * l + 6) * zeta;
        }
        tx = fma(g, fma(f, dx, Sx), tx);
        ty = fma(g, fma(f, dy, Sy), ty);
        tz = fma(g, fma(f, dz, Sz), tz);
        tl = fma(g * S0, lapfac, tl);
      }
      // lane partials summed in FP64, or (FP32 partials) as double-words with
      // FP32 instructions only
      double gx, gy, gz, lp;
      if constexpr (kDw) {
        fdw sx{static_cast<float>(tx), 0.0f}, sy{static_cast<float>(ty), 0.0f}, sz{static_cast<float>(tz), 0.0f},
            sl{static_cast<float>(tl), 0.0f};
  #pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
          sx = dw_add(sx, fdw{__shfl_xor_sync(0xffffffffu, sx.hi, o), __shfl_xor_sync(0xffffffffu, sx.lo, o)});
          sy = dw_add(sy, fdw{__shfl_xor_sync(0xffffffffu, sy.hi, o), __shfl_xor_sync(0xffffffffu, sy.lo, o)});
          sz = dw_add(sz, fdw{__shfl_xor_sync(0xffffffffu, sz.hi, o), __shfl_xor_sync(0xffffffffu, sz.lo, o)});
          sl = dw_add(sl, fdw{__shfl_xor_sync(0xffffffffu, sl.hi, o), __shfl_xor_sync(0xffffffffu, sl.lo, o)});
        }
        gx = static_cast<double>(sx.hi) + sx.lo;
        gy = static_cast<double>(sy.hi) + sy.lo;
        gz = static_cast<double>(sz.hi) + sz.lo;
        lp = static_cast<double>(sl.hi) + sl.lo;
      } else {
        gx = warp_sum(static_cast<double>(tx));
        gy = warp_sum(static_cast<double>(ty));
        gz = warp_sum(static_cast<double>(tz));
        lp = warp_sum(static_cast<double>(tl));
      }
      if (lane == 0) {
        double *o = kin + pt * 4;
        o[0] = gx;
        o[1] = gy;
        o[2] = gz;
        o[3] = lp;
      }
    }
}
};
template <typename T>
__global__ void __launch_bounds__(256) k_kinetic(DevSystem s, const double *__restrict__ r,
                                                 const T *__restrict__ mbuf, double *__restrict__ kin, int W) {
  Kinetic<T>::run(s, r, mbuf, kin, W, blockIdx, gridDim);
}

template <typename T>
cudaError_t launch_kinetic(const DevSystem &s, const double *r, const T *mbuf, double *kin, int W, cudaStream_t st) {
  if (W <= 0) return cudaSuccess;
  const long total = (long)W * s.N;
  long blocks = (total + 7) / 8;
  if (blocks > 152 * 16) blocks = 152 * 16;
  const size_t smem = (size_t)s.n_shells * (sizeof(double4) + sizeof(int));
  return launch_or_record<Kinetic<T>, 256>(k_kinetic<T>, dim3((int)blocks), dim3(256), smem, st, s, r, mbuf, kin, W);
}
template cudaError_t launch_kinetic<double>(const DevSystem &, const double *, const double *, double *, int,
                                            cudaStream_t);
template cudaError_t launch_kinetic<float>(const DevSystem &, const double *, const float *, double *, int,
                                           cudaStream_t);

// ---------------------------------------------------------------------------
// The mixed path's contraction with two-float M vectors (M + M_lo: exact
// fixed-point tensor-core products of the FP64 inverse with the two-float
// tables): the same per-shell formulas as k_kinetic with every step in
// double-word arithmetic (FP32 instructions only), so that the result keeps
// the M vectors' accuracy.  Rounding the shells' terms to FP32 would not: the
// shells' contributions cancel to a sum that is smaller by about cond(G~),
// which makes their FP32 rounding the dominant error of e_L at large N_up.
// ---------------------------------------------------------------------------
struct KineticM2 {
  static __device__ __forceinline__ void run(DevSystem s, const double *__restrict__ r,
                                             const float *__restrict__ mbuf, const float *__restrict__ mlo,
                                             double *__restrict__ kin, int W, const uint3 bid, const uint3 gdim) {
    assume_global(r, mbuf, mlo, kin);
    extern __shared__ double4 sh_geo[];
    int *sh_info = reinterpret_cast<int *>(sh_geo + s.n_shells);
    float4 *sh_dw = reinterpret_cast<float4 *>(sh_geo);
    for (int k = threadIdx.x; k < s.n_shells; k += blockDim.x) {
      sh_dw[2 * k] = s.shell_dw[2 * k];
      sh_dw[2 * k + 1] = s.shell_dw[2 * k + 1];
      sh_info[k] = s.shell_info[k];
    }
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const long nwarps = (long)gdim.x * (blockDim.x >> 5);
    const long total = (long)W * s.N;
    const fdw zero{0.0f, 0.0f};
    for (long pt = (long)bid.x * (blockDim.x >> 5) + (threadIdx.x >> 5); pt < total; pt += nwarps) {
      const double *rr = r + pt * 3;
      fdw pd[3];
      {
        const int kc = lane < 3 ? lane : 2;
        const fdw mine = dw_of(rr[kc]);
  #pragma unroll
        for (int k = 0; k < 3; ++k)
          pd[k] = fdw{__shfl_sync(0xffffffffu, mine.hi, k), __shfl_sync(0xffffffffu, mine.lo, k)};
      }
      const float *M = mbuf + pt * s.L, *Ml = mlo + pt * s.L;
      fdw tx = zero, ty = zero, tz = zero, tl = zero;
      for (int k = lane; k < s.n_shells; k += 32) {
        const int info = sh_info[k];
        const int l = shell_l(info), off = shell_off(info), rad = shell_rad(info);
        const float4 gh = sh_dw[2 * k], gl = sh_dw[2 * k + 1];
        const DwDisp d = dw_displacement(pd, gh, gl);
        const fdw zw{gh.w, gl.w};
        fdw g, rinv = zero;
        if (rad) {
          const fdw rw = dw_sqrt(d.r2);
          g = dw_exp_neg(dw_neg(dw_mul(zw, rw)));
          rinv = dw_recip(rw);
        } else {
          g = dw_exp_neg(dw_neg(dw_mul(zw, d.r2)));
        }
        fdw S0, Sx = zero, Sy = zero, Sz = zero;
        const fdw m0{M[off], Ml[off]};
        if (l == 0) {
          S0 = m0;
        } else if (l == 1) {
          const fdw m1{M[off + 1], Ml[off + 1]}, m2{M[off + 2], Ml[off + 2]};
          S0 = dw_add(dw_add(dw_mul(m0, d.x), dw_mul(m1, d.y)), dw_mul(m2, d.z));
          Sx = m0;
          Sy = m1;
          Sz = m2;
        } else {
          const fdw m1{M[off + 1], Ml[off + 1]}, m2{M[off + 2], Ml[off + 2]}, m3{M[off + 3], Ml[off + 3]},
              m4{M[off + 4], Ml[off + 4]};
          const fdw xx = dw_mul(d.x, d.x), yy = dw_mul(d.y, d.y), zz = dw_mul(d.z, d.z);
          S0 = dw_add(dw_add(dw_mul(m0, dw_mul(d.x, d.y)), dw_mul(m1, dw_mul(d.y, d.z))),
                      dw_add(dw_mul(m2, dw_mul(d.z, d.x)), dw_mul(m3, dw_add(xx, dw_neg(yy)))));
          S0 = dw_add(S0, dw_mul(m4, dw_add(dw_mul_f(zz, 3.0f), dw_neg(d.r2))));
          const fdw d34 = dw_add(m3, dw_neg(m4)), s34 = dw_add(m3, m4);
          Sx = dw_add(dw_add(dw_mul(m0, d.y), dw_mul(m2, d.z)), dw_mul_f(dw_mul(d34, d.x), 2.0f));
          Sy = dw_add(dw_add(dw_mul(m0, d.x), dw_mul(m1, d.z)), dw_neg(dw_mul_f(dw_mul(s34, d.y), 2.0f)));
          Sz = dw_add(dw_add(dw_mul(m1, d.y), dw_mul(m2, d.x)), dw_mul_f(dw_mul(m4, d.z), 4.0f));
        }
        fdw f, lapfac;
        const fdw zz2 = dw_mul(zw, zw);
        if (rad) {
          f = dw_neg(dw_mul(dw_mul(zw, S0), rinv));
          lapfac = dw_add(zz2, dw_neg(dw_mul_f(dw_mul(zw, rinv), static_cast<float>(2 * (l + 1)))));
        } else {
          f = dw_neg(dw_mul_f(dw_mul(zw, S0), 2.0f));
          lapfac = dw_add(dw_mul_f(dw_mul(zz2, d.r2), 4.0f), dw_neg(dw_mul_f(zw, static_cast<float>(4 * l + 6))));
        }
        tx = dw_add(tx, dw_mul(g, dw_add(Sx, dw_mul(f, d.x))));
        ty = dw_add(ty, dw_mul(g, dw_add(Sy, dw_mul(f, d.y))));
        tz = dw_add(tz, dw_mul(g, dw_add(Sz, dw_mul(f, d.z))));
        tl = dw_add(tl, dw_mul(dw_mul(g, S0), lapfac));
      }
  #pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        tx = dw_add(tx, fdw{__shfl_xor_sync(0xffffffffu, tx.hi, o), __shfl_xor_sync(0xffffffffu, tx.lo, o)});
        ty = dw_add(ty, fdw{__shfl_xor_sync(0xffffffffu, ty.hi, o), __shfl_xor_sync(0xffffffffu, ty.lo, o)});
        tz = dw_add(tz, fdw{__shfl_xor_sync(0xffffffffu, tz.hi, o), __shfl_xor_sync(0xffffffffu, tz.lo, o)});
        tl = dw_add(tl, fdw{__shfl_xor_sync(0xffffffffu, tl.hi, o), __shfl_xor_sync(0xffffffffu, tl.lo, o)});
      }
      if (lane == 0) {
        double *o = kin + pt * 4;
        o[0] = static_cast<double>(tx.hi) + tx.lo;
        o[1] = static_cast<double>(ty.hi) + ty.lo;
        o[2] = static_cast<double>(tz.hi) + tz.lo;
        o[3] = static_cast<double>(tl.hi) + tl.lo;
      }
    }
}
};
__global__ void __launch_bounds__(256) k_kinetic_m2(DevSystem s, const double *__restrict__ r,
                                                    const float *__restrict__ mbuf, const float *__restrict__ mlo,
                                                    double *__restrict__ kin, int W) {
  KineticM2::run(s, r, mbuf, mlo, kin, W, blockIdx, gridDim);
}

cudaError_t launch_kinetic_m2(const DevSystem &s, const double *r, const float *mbuf, const float *mlo, double *kin,
                              int W, cudaStream_t st) {
  if (W <= 0) return cudaSuccess;
  const long total = (long)W * s.N;
  long blocks = (total + 7) / 8;
  if (blocks > 152 * 16) blocks = 152 * 16;
  const size_t smem = (size_t)s.n_shells * (sizeof(double4) + sizeof(int));
  return launch_or_record<KineticM2, 256>(k_kinetic_m2, dim3((int)blocks), dim3(256), smem, st, s, r, mbuf, mlo, kin,
                                          W);
}

// ---------------------------------------------------------------------------
// Jastrow value and derivatives, kinetic assembly and the Coulomb terms: one
// CTA per walker.  With scal given, J = J1 + J2 is written too (the sweep then
// needs no separate Jastrow pass).
// ---------------------------------------------------------------------------
struct Elocal {
  static __device__ __forceinline__ void run(DevSystem s, const double *__restrict__ r,
                                             const double *__restrict__ kin, double *__restrict__ eL,
                                             double *__restrict__ parts, double *__restrict__ scal,
                                             const double *__restrict__ j3buf, const uint3 bid, const uint3 gdim) {
    assume_global(r, kin, eL);
    const int w = bid.x, N = s.N, tid = threadIdx.x;
    extern __shared__ double xs[];
    for (int t = tid; t < N * 3; t += blockDim.x) xs[t] = r[(size_t)w * N * 3 + t];
    __syncthreads();
    double tkin = 0.0, vee = 0.0, vei = 0.0, jv = 0.0;
    for (int e = tid; e < N; e += blockDim.x) {
      const double ex = xs[3 * e], ey = xs[3 * e + 1], ez = xs[3 * e + 2];
      double gJx = 0.0, gJy = 0.0, gJz = 0.0, lJ = 0.0;
      for (int a = 0; a < s.n_atoms; ++a) {
        const double dx = ex - s.R[3 * a], dy = ey - s.R[3 * a + 1], dz = ez - s.R[3 * a + 2];
        const double r2 = dx * dx + dy * dy + dz * dz;
        const double rinv = rsqrt(r2), rr = r2 * rinv;
        vei -= s.Z[a] * rinv;
        if (s.use_j1) {
          // f = -c^3 u(c r), u = (1 - e^{-b s}) / (2b); f' = -c^4 e / 2, f'' = c^5 b e / 2
          const double c = s.c1[a], c3 = c * c * c, c4 = c3 * c, b = s.b_ea;
          double f, fp, fpp;
          if (b == 0.0) {
            f = -0.5 * c4 * rr;
            fp = -0.5 * c4;
            fpp = 0.0;
          } else {
            const double ex1 = exp(-b * c * rr);
            f = -c3 * (1.0 - ex1) / (2.0 * b);
            fp = -0.5 * c4 * ex1;
            fpp = 0.5 * c4 * c * b * ex1;
          }
          jv += f;
          const double q = fp * rinv;
          gJx += q * dx;
          gJy += q * dy;
          gJz += q * dz;
          lJ += fpp + 2.0 * q;
        }
      }
      for (int k = 0; k < N; ++k) {
        if (k == e) continue;
        const double dx = ex - xs[3 * k], dy = ey - xs[3 * k + 1], dz = ez - xs[3 * k + 2];
        const double r2 = dx * dx + dy * dy + dz * dz;
        const double rinv = rsqrt(r2), rr = r2 * rinv;
        if (k > e) vee += rinv;
        if (s.use_j2) {
          double kk, bb;
          j2_params(s, (e < s.n_up) == (k < s.n_up), &kk, &bb);
          const double ik = 1.0 / kk;  // exact: k is 2 or 4
          const double iq = 1.0 / (1.0 + bb * rr);
          const double vp = ik * iq * iq;
          const double vpp = -2.0 * bb * vp * iq;
          if (k > e) jv += rr * ik * iq;
          const double q = vp * rinv;
          gJx += q * dx;
          gJy += q * dy;
          gJz += q * dz;
          lJ += vpp + 2.0 * q;
        }
      }
      if (s.use_j3 && j3buf) {
        // three/four-body Jastrow: 1/2 chi^T Q to J, (grad chi)^T Q, (lap chi)^T Q
        double g3[3] = {0.0, 0.0, 0.0};
        j3_electron(s, j3buf + (size_t)w * 6 * s.LJ, e < s.n_up, ex, ey, ez, &jv, g3, &lJ);
        gJx += g3[0];
        gJy += g3[1];
        gJz += g3[2];
      }
      const double *kd = kin + ((size_t)w * N + e) * 4;
      const double t = kd[3] + lJ + 2.0 * (kd[0] * gJx + kd[1] * gJy + kd[2] * gJz) +
                       (gJx * gJx + gJy * gJy + gJz * gJz);
      tkin += -0.5 * t;
    }
    __shared__ double red[4][4];
    tkin = warp_sum(tkin);
    vee = warp_sum(vee);
    vei = warp_sum(vei);
    jv = warp_sum(jv);
    if ((tid & 31) == 0) {
      red[0][tid >> 5] = tkin;
      red[1][tid >> 5] = vee;
      red[2][tid >> 5] = vei;
      red[3][tid >> 5] = jv;
    }
    __syncthreads();
    if (tid == 0) {
      double a = 0.0, b = 0.0, c = 0.0, j = 0.0;
      for (int q = 0; q < (int)(blockDim.x >> 5); ++q) {
        a += red[0][q];
        b += red[1][q];
        c += red[2][q];
        j += red[3][q];
      }
      eL[w] = a + b + c + s.v_ii;
      if (parts) {
        parts[(size_t)w * 4 + 0] = a;
        parts[(size_t)w * 4 + 1] = b;
        parts[(size_t)w * 4 + 2] = c;
        parts[(size_t)w * 4 + 3] = s.v_ii;
      }
      if (scal) scal[(size_t)w * S_STRIDE + S_J] = j;
    }
}
};
__global__ void __launch_bounds__(128) k_elocal(DevSystem s, const double *__restrict__ r,
                                                const double *__restrict__ kin, double *__restrict__ eL,
                                                double *__restrict__ parts, double *__restrict__ scal,
                                                const double *__restrict__ j3buf) {
  Elocal::run(s, r, kin, eL, parts, scal, j3buf, blockIdx, gridDim);
}

// ---------------------------------------------------------------------------
// The same local-energy assembly for the FP32 path with FP32 instructions:
// distances, 1/r, the Coulomb sums and the Jastrow values in double-word
// arithmetic (dword.cuh; ~1e-14 relative, so V, J and the Jastrow gradients
// and Laplacians keep FP64-level accuracy without the FP64 pipe; the Jastrow
// gradient multiplies grad D / D in the kinetic term, so FP32 there was not
// enough).  One CTA per walker; the per-thread sums are double-words,
// combined in FP64 at the end.
// ---------------------------------------------------------------------------
struct ElocalDw {
  static __device__ __forceinline__ void run(DevSystem s, const double *__restrict__ r,
                                             const double *__restrict__ kin, double *__restrict__ eL,
                                             double *__restrict__ parts, double *__restrict__ scal,
                                             const double *__restrict__ j3buf, const uint3 bid, const uint3 gdim) {
    assume_global(r, kin, eL);
    const int w = bid.x, N = s.N, tid = threadIdx.x, na = s.n_atoms;
    const int lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
    extern __shared__ float sf[];
    float *xh = sf, *xl = xh + 3 * N;           // electron coordinates as double-words
    float *ah = xl + 3 * N, *al = ah + 3 * na;  // atom coordinates
    // per atom, as double-words: -Z, and for J1 -c^4/2, c^3/(2b), -b c
    float *ac = al + 3 * na;
    // two-body Jastrow constants [same spin, opposite spin]: b k (dw), k, -2 b (dw)
    __shared__ float j2c[2][5];
    for (int t = tid; t < N * 3; t += blockDim.x) {
      const fdw v = dw_of(r[(size_t)w * N * 3 + t]);
      xh[t] = v.hi;
      xl[t] = v.lo;
    }
    for (int t = tid; t < na * 3; t += blockDim.x) {
      const fdw v = dw_of(s.R[t]);
      ah[t] = v.hi;
      al[t] = v.lo;
    }
    for (int a = tid; a < na; a += blockDim.x) {
      const double c = s.c1[a], b = s.b_ea;
      const fdw z = dw_of(-s.Z[a]), c4 = dw_of(-0.5 * c * c * c * c);
      const fdw c3 = dw_of(b == 0.0 ? 0.0 : c * c * c / (2.0 * b)), bc = dw_of(-b * c);
      float *q = ac + 8 * a;
      q[0] = z.hi;
      q[1] = z.lo;
      q[2] = c4.hi;
      q[3] = c4.lo;
      q[4] = c3.hi;
      q[5] = c3.lo;
      q[6] = bc.hi;
      q[7] = bc.lo;
    }
    if (tid < 2) {
      double kk, bb;
      j2_params(s, tid == 0, &kk, &bb);
      const fdw bk = dw_of(bb * kk), m2b = dw_of(-2.0 * bb);
      j2c[tid][0] = bk.hi;
      j2c[tid][1] = bk.lo;
      j2c[tid][2] = static_cast<float>(kk);  // 2 or 4, exact
      j2c[tid][3] = m2b.hi;
      j2c[tid][4] = m2b.lo;
    }
    __syncthreads();
    // a warp per electron, its lanes over the partners (atoms, then electrons);
    // every constant comes from shared memory, so the loops are FP32 only
    fdw tkin{0.0f, 0.0f}, vee{0.0f, 0.0f}, vei{0.0f, 0.0f}, jv{0.0f, 0.0f};
    const int P = na + N;
    // lane j keeps the Jastrow gradient and Laplacian of the warp's j-th electron
    // of the current group of 32, so that the FP64 assembly of the kinetic term
    // is issued once per group instead of once per electron
    fdw kx{0.0f, 0.0f}, ky{0.0f, 0.0f}, kz{0.0f, 0.0f}, kl{0.0f, 0.0f};
    int mine = -1, slot = 0;
    for (int e = warp; e < N; e += nw) {
      const fdw pe[3] = {{xh[3 * e], xl[3 * e]}, {xh[3 * e + 1], xl[3 * e + 1]}, {xh[3 * e + 2], xl[3 * e + 2]}};
      const bool eup = e < s.n_up;
      fdw gJx{0.0f, 0.0f}, gJy{0.0f, 0.0f}, gJz{0.0f, 0.0f}, lJ{0.0f, 0.0f};
      for (int p = lane; p < P; p += 32) {
        if (p < na) {
          const int a = p;
          const float *q = ac + 8 * a;
          const fdw dx = dw_add(pe[0], fdw{-ah[3 * a], -al[3 * a]});
          const fdw dy = dw_add(pe[1], fdw{-ah[3 * a + 1], -al[3 * a + 1]});
          const fdw dz = dw_add(pe[2], fdw{-ah[3 * a + 2], -al[3 * a + 2]});
          const fdw r2 = dw_add(dw_add(dw_mul(dx, dx), dw_mul(dy, dy)), dw_mul(dz, dz));
          const fdw rr = dw_sqrt(r2), rinv = dw_recip(rr);
          vei = dw_add(vei, dw_mul(rinv, fdw{q[0], q[1]}));
          if (s.use_j1) {
            // f = -c^3 u(c r), u = (1 - e^{-b c r}) / (2b); f' = -c^4 e / 2, f'' = c^5 b e / 2
            const fdw c4{q[2], q[3]}, bc{q[6], q[7]};
            fdw ex{1.0f, 0.0f};
            if (s.b_ea == 0.0) {
              jv = dw_add(jv, dw_mul(rr, c4));
            } else {
              ex = dw_exp_neg(dw_mul(rr, bc));
              // -c^3 (1 - e) / (2b) = c^3 / (2b) (e - 1)
              jv = dw_add(jv, dw_mul(dw_add_f(ex, -1.0f), fdw{q[4], q[5]}));
            }
            const fdw fp = dw_mul(ex, c4);   // f'
            const fdw fpp = dw_mul(fp, bc);  // f'' = -b c f'
            const fdw qq = dw_mul(fp, rinv);
            gJx = dw_add(gJx, dw_mul(qq, dx));
            gJy = dw_add(gJy, dw_mul(qq, dy));
            gJz = dw_add(gJz, dw_mul(qq, dz));
            lJ = dw_add(lJ, dw_add(fpp, dw_add(qq, qq)));
          }
          continue;
        }
        const int k = p - na;
        if (k == e) continue;
        const fdw dx = dw_add(pe[0], fdw{-xh[3 * k], -xl[3 * k]});
        const fdw dy = dw_add(pe[1], fdw{-xh[3 * k + 1], -xl[3 * k + 1]});
        const fdw dz = dw_add(pe[2], fdw{-xh[3 * k + 2], -xl[3 * k + 2]});
        const fdw r2 = dw_add(dw_add(dw_mul(dx, dx), dw_mul(dy, dy)), dw_mul(dz, dz));
        const fdw rr = dw_sqrt(r2), rinv = dw_recip(rr);
        if (k > e) vee = dw_add(vee, rinv);
        if (s.use_j2) {
          const float *jc = j2c[eup == (k < s.n_up) ? 0 : 1];
          const float kk = jc[2];
          const fdw den = dw_add_f(dw_mul(rr, fdw{jc[0], jc[1]}), kk);  // k (1 + b r), k exact
          const fdw iq = dw_recip(den);                                  // 1 / (k (1 + b r))
          if (k > e) jv = dw_add(jv, dw_mul(rr, iq));
          const fdw qi = dw_mul_f(iq, kk);                               // 1/q (k exact)
          const fdw vp = dw_mul(iq, qi);                                 // 1 / (k q^2)
          const fdw vpp = dw_mul(dw_mul(vp, qi), fdw{jc[3], jc[4]});      // -2b / (k q^3)
          const fdw qq = dw_mul(vp, rinv);
          gJx = dw_add(gJx, dw_mul(qq, dx));
          gJy = dw_add(gJy, dw_mul(qq, dy));
          gJz = dw_add(gJz, dw_mul(qq, dz));
          lJ = dw_add(lJ, dw_add(vpp, dw_add(qq, qq)));
        }
      }
      // the electron's Jastrow gradient and Laplacian over the warp
  #pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        gJx = dw_add(gJx, fdw{__shfl_xor_sync(0xffffffffu, gJx.hi, o), __shfl_xor_sync(0xffffffffu, gJx.lo, o)});
        gJy = dw_add(gJy, fdw{__shfl_xor_sync(0xffffffffu, gJy.hi, o), __shfl_xor_sync(0xffffffffu, gJy.lo, o)});
        gJz = dw_add(gJz, fdw{__shfl_xor_sync(0xffffffffu, gJz.hi, o), __shfl_xor_sync(0xffffffffu, gJz.lo, o)});
        lJ = dw_add(lJ, fdw{__shfl_xor_sync(0xffffffffu, lJ.hi, o), __shfl_xor_sync(0xffffffffu, lJ.lo, o)});
      }
      if (s.use_j3 && j3buf) {
        // three/four-body Jastrow of this electron in FP64 on one lane (its
        // value to J, gradient and Laplacian to the Jastrow sums of every lane)
        double v3 = 0.0, g3[3] = {0.0, 0.0, 0.0}, l3 = 0.0;
        if (lane == 0) {
          const double *pr = r + ((size_t)w * N + e) * 3;
          j3_electron(s, j3buf + (size_t)w * 6 * s.LJ, eup, pr[0], pr[1], pr[2], &v3, g3, &l3);
          jv = dw_add(jv, dw_of(v3));
        }
        gJx = dw_add(gJx, dw_of(__shfl_sync(0xffffffffu, g3[0], 0)));
        gJy = dw_add(gJy, dw_of(__shfl_sync(0xffffffffu, g3[1], 0)));
        gJz = dw_add(gJz, dw_of(__shfl_sync(0xffffffffu, g3[2], 0)));
        lJ = dw_add(lJ, dw_of(__shfl_sync(0xffffffffu, l3, 0)));
      }
      if (lane == slot) {
        kx = gJx;
        ky = gJy;
        kz = gJz;
        kl = lJ;
        mine = e;
      }
      if (++slot == 32 || e + nw >= N) {  // warp-uniform
        if (mine >= 0) {
          const double *kd = kin + ((size_t)w * N + mine) * 4;
          const double gx = static_cast<double>(kx.hi) + kx.lo, gy = static_cast<double>(ky.hi) + ky.lo,
                       gz = static_cast<double>(kz.hi) + kz.lo, lj = static_cast<double>(kl.hi) + kl.lo;
          const double t =
              kd[3] + lj + 2.0 * (kd[0] * gx + kd[1] * gy + kd[2] * gz) + (gx * gx + gy * gy + gz * gz);
          tkin = dw_add(tkin, dw_of(-0.5 * t));
        }
        mine = -1;
        slot = 0;
      }
    }
    // the four sums over the block as double-words (FP32 instructions), FP64 at the end
    __shared__ float red[4][4][2];
    fdw a4[4] = {tkin, vee, vei, jv};
  #pragma unroll
    for (int q = 0; q < 4; ++q)
  #pragma unroll
      for (int o = 16; o > 0; o >>= 1)
        a4[q] = dw_add(a4[q], fdw{__shfl_xor_sync(0xffffffffu, a4[q].hi, o), __shfl_xor_sync(0xffffffffu, a4[q].lo, o)});
    if (lane == 0)
  #pragma unroll
      for (int q = 0; q < 4; ++q) {
        red[q][warp][0] = a4[q].hi;
        red[q][warp][1] = a4[q].lo;
      }
    __syncthreads();
    if (tid == 0) {
      fdw sum[4];
      for (int q = 0; q < 4; ++q) {
        sum[q] = fdw{red[q][0][0], red[q][0][1]};
        for (int k = 1; k < nw; ++k) sum[q] = dw_add(sum[q], fdw{red[q][k][0], red[q][k][1]});
      }
      const double a = static_cast<double>(sum[0].hi) + sum[0].lo, b = static_cast<double>(sum[1].hi) + sum[1].lo,
                   c = static_cast<double>(sum[2].hi) + sum[2].lo, j = static_cast<double>(sum[3].hi) + sum[3].lo;
      eL[w] = a + b + c + s.v_ii;
      if (parts) {
        parts[(size_t)w * 4 + 0] = a;
        parts[(size_t)w * 4 + 1] = b;
        parts[(size_t)w * 4 + 2] = c;
        parts[(size_t)w * 4 + 3] = s.v_ii;
      }
      if (scal) scal[(size_t)w * S_STRIDE + S_J] = j;
    }
}
};
__global__ void __launch_bounds__(128) k_elocal_dw(DevSystem s, const double *__restrict__ r,
                                                   const double *__restrict__ kin, double *__restrict__ eL,
                                                   double *__restrict__ parts, double *__restrict__ scal,
                                                   const double *__restrict__ j3buf) {
  ElocalDw::run(s, r, kin, eL, parts, scal, j3buf, blockIdx, gridDim);
}

cudaError_t launch_elocal_dw(const DevSystem &s, const double *r, const double *kin, double *eL, double *parts, int W,
                             cudaStream_t st, double *scal, const double *j3buf) {
  if (W <= 0) return cudaSuccess;
  if (s.use_j3 && !j3buf) return cudaErrorInvalidValue;
  const size_t smem = ((size_t)(s.N + s.n_atoms) * 6 + (size_t)s.n_atoms * 8) * sizeof(float);
  return launch_or_record<ElocalDw, 128>(k_elocal_dw, dim3(W), dim3(128), smem, st, s, r, kin, eL, parts, scal,
                                         j3buf);
}

cudaError_t launch_elocal(const DevSystem &s, const double *r, const double *kin, double *eL, double *parts, int W,
                          cudaStream_t st, double *scal, const double *j3buf) {
  if (W <= 0) return cudaSuccess;
  if (s.use_j3 && !j3buf) return cudaErrorInvalidValue;
  return launch_or_record<Elocal, 128>(k_elocal, dim3(W), dim3(128), (size_t)s.N * 3 * sizeof(double), st, s, r, kin,
                                       eL, parts, scal, j3buf);
}

// the kernels of this file raise their shared-memory limit when first
// launched (launch_or_record)
cudaError_t setup_energy_attributes() { return cudaSuccess; }

}  // namespace jagp
