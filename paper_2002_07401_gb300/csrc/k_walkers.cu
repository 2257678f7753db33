// k_walkers.cu -- per-electron and per-walker kernels of the VMC sweep:
// orbital evaluation at electrons / proposals, the sequential Metropolis
// acceptance with Sherman-Morrison updates, the full Jastrow, bookkeeping.
#include <math.h>

#include <type_traits>

#include "j3.cuh"
#include "jagp_group.cuh"
#include "jagp_launch.h"

namespace jagp {

// ---------------------------------------------------------------------------
// Orbitals at points: one warp per point, lanes stride over shells.  The shell
// table (32-byte centre+exponent records and packed info words; in the FP32
// path the double-word split records instead) is staged in shared memory once
// per CTA; CTAs then grid-stride over points.
// (Sec. "Atomic basis set", Eqs. gaussian, slater.)
// FP64 path: FP64 values.  FP32 path: double-word values (FP32 arithmetic
// only, see shell_values_dw); the FP32 table gets hi, out_lo (when given) lo.
// With PROPOSE the point is the Metropolis proposal of the electron, and the
// one-body Jastrow change of the move is taken here as well (FP32 distances in
// the FP32 path: it only enters the acceptance test).
// ---------------------------------------------------------------------------
// Mixed path: FP32 instructions only, from the positions and atoms rounded to
// FP32 (the change only enters the acceptance test); every lane gets the sum.
__device__ __forceinline__ double j1_move_change_f(const DevSystem &s, const float *rp, const float *rr, int lane) {
  float dj1 = 0.0f;
  const float b = s.b_ea_f;
  for (int q = lane; q < 2 * s.n_atoms; q += 32) {
    const float4 A = s.atom_f[q >> 1];
    const float *pos = (q & 1) ? rr : rp;
    const float ax = pos[0] - A.x, ay = pos[1] - A.y, az = pos[2] - A.z;
    const float c = A.w;
    const float sc = c * sqrtf(ax * ax + ay * ay + az * az);
    const float u = (b == 0.0f) ? 0.5f * sc : -expm1f(-b * sc) / (2.0f * b);
    const float v = -c * c * c * u;
    dj1 += (q & 1) ? -v : v;
  }
  return static_cast<double>(warp_sum(dj1));
}

template <bool PROPOSE, typename T>
struct BasisPoints {
  static __device__ __forceinline__ void run(DevSystem s, const double *__restrict__ r, int W, int e0, int npts,
                                             T *__restrict__ out, float *__restrict__ out_lo,
                                             double *__restrict__ rprop, uint32_t walker0, uint32_t sweep,
                                             const uint32_t *__restrict__ sweep_dev, const uint3 bid,
                                             const uint3 gdim) {
    assume_global(r, out);
    constexpr bool kDw = std::is_same<T, float>::value;
    if (PROPOSE && sweep_dev) sweep += *sweep_dev;  // graph replays read the sweep index from the device
    extern __shared__ double4 sh_geo[];
    int *sh_info = reinterpret_cast<int *>(sh_geo + s.n_shells);
    float4 *sh_dw = reinterpret_cast<float4 *>(sh_geo);  // FP32 path: two float4 per shell in place of the double4
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
    const long total = (long)W * npts;
    for (long pt = (long)bid.x * (blockDim.x >> 5) + (threadIdx.x >> 5); pt < total; pt += nwarps) {
      const int w = (int)(pt / npts), i = (int)(pt % npts);
      const double *rr = r + ((size_t)w * s.N + e0 + i) * 3;
      double p[3] = {rr[0], rr[1], rr[2]};
      const int kc = lane < 3 ? lane : 2;  // the coordinate this lane converts
      if (PROPOSE) {
        double rp[3], u, rpk;
        move_draw_coord(s, walker0 + (uint32_t)w, sweep, (uint32_t)(e0 + i), p[kc], kc, &rpk, &u);
  #pragma unroll
        for (int k = 0; k < 3; ++k) rp[k] = __shfl_sync(0xffffffffu, rpk, k);
        p[0] = rp[0];
        p[1] = rp[1];
        p[2] = rp[2];
        // change of the one-body Jastrow for this move: it depends only on the
        // electron's own old and new positions, so it is taken here, in parallel
        double dj1 = 0.0;
        if (s.use_j1) {
          if constexpr (kDw) {
            // new and old position in FP32, one coordinate converted per lane
            const float pk = static_cast<float>(rpk), ok = static_cast<float>(rr[kc]);
            float pf[3], of[3];
  #pragma unroll
            for (int k = 0; k < 3; ++k) {
              pf[k] = __shfl_sync(0xffffffffu, pk, k);
              of[k] = __shfl_sync(0xffffffffu, ok, k);
            }
            dj1 = j1_move_change_f(s, pf, of, lane);
          } else {
            dj1 = j1_move_change(s, rp, rr, lane);
          }
        }
        double *rec = rprop + ((size_t)w * s.n_up + i) * kPropStride;
        if (lane < 4) rec[lane] = lane < 3 ? rp[lane] : u;
        if (lane == 0) rec[4] = dj1;
      }
      T *o = out + ((size_t)w * s.n_up + i) * s.L;
      if constexpr (kDw) {
        const fdw mine = dw_of(p[kc]);  // one conversion per lane, shared by shuffles
        fdw pd[3];
  #pragma unroll
        for (int k = 0; k < 3; ++k)
          pd[k] = fdw{__shfl_sync(0xffffffffu, mine.hi, k), __shfl_sync(0xffffffffu, mine.lo, k)};
        float *ol = out_lo ? out_lo + ((size_t)w * s.n_up + i) * s.L : nullptr;
        for (int k = lane; k < s.n_shells; k += 32) {
          const float4 gh = sh_dw[2 * k], gl = sh_dw[2 * k + 1];
          const int info = sh_info[k];
          const DwDisp d = dw_displacement(pd, gh, gl);
          float v[5], vl[5];
          const int nc = shell_values_dw(info, fdw{gh.w, gl.w}, d, v, vl);
          const int off = shell_off(info);
  #pragma unroll
          for (int c = 0; c < 5; ++c)
            if (c < nc) {
              o[off + c] = v[c];
              if (ol) ol[off + c] = vl[c];
            }
        }
      } else {
        for (int k = lane; k < s.n_shells; k += 32) {
          const double4 g = sh_geo[k];
          const int info = sh_info[k];
          double v[5];
          const int nc = shell_values(info, g.w, p[0] - g.x, p[1] - g.y, p[2] - g.z, v);
          const int off = shell_off(info);
  #pragma unroll
          for (int c = 0; c < 5; ++c)
            if (c < nc) o[off + c] = v[c];
        }
      }
    }
}
};
template <bool PROPOSE, typename T>
__global__ void __launch_bounds__(256) k_basis_points(DevSystem s, const double *__restrict__ r, int W, int e0,
                                                      int npts, T *__restrict__ out, float *__restrict__ out_lo,
                                                      double *__restrict__ rprop, uint32_t walker0, uint32_t sweep,
                                                      const uint32_t *__restrict__ sweep_dev) {
  BasisPoints<PROPOSE, T>::run(s, r, W, e0, npts, out, out_lo, rprop, walker0, sweep, sweep_dev, blockIdx, gridDim);
}

template <typename T>
cudaError_t launch_basis_points(const DevSystem &s, bool propose, const double *r, int W, int e0, int npts,
                                T *out, float *out_lo, double *rprop, uint32_t walker0, uint32_t sweep,
                                cudaStream_t st, const uint32_t *sweep_dev) {
  if (W <= 0 || npts <= 0) return cudaSuccess;
  const long total = (long)W * npts;
  const int warps = 8;
  long blocks = (total + warps - 1) / warps;
  if (blocks > 152 * 16) blocks = 152 * 16;
  const size_t smem = (size_t)s.n_shells * (sizeof(double4) + sizeof(int));
  if (propose)
    return launch_or_record<BasisPoints<true, T>, 256>(k_basis_points<true, T>, dim3((int)blocks), dim3(warps * 32), smem, st, s, r, W, e0,
                                                       npts, out, out_lo, rprop, walker0, sweep, sweep_dev);
  return launch_or_record<BasisPoints<false, T>, 256>(k_basis_points<false, T>, dim3((int)blocks), dim3(warps * 32), smem, st, s, r, W, e0,
                                                      npts, out, out_lo, rprop, walker0, sweep,
                                                      (const uint32_t *)nullptr);
}
template cudaError_t launch_basis_points<double>(const DevSystem &, bool, const double *, int, int, int, double *,
                                                 float *, double *, uint32_t, uint32_t, cudaStream_t,
                                                 const uint32_t *);
template cudaError_t launch_basis_points<float>(const DevSystem &, bool, const double *, int, int, int, float *,
                                                float *, double *, uint32_t, uint32_t, cudaStream_t,
                                                const uint32_t *);

// ---------------------------------------------------------------------------
// Block reduction of two doubles (blockDim.x <= 1024); result valid in thread 0.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void block_sum2(double &a, double &b, double *red) {
  a = warp_sum(a);
  b = warp_sum(b);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  __syncthreads();
  if (lane == 0) {
    red[2 * warp] = a;
    red[2 * warp + 1] = b;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int q = 1; q < nw; ++q) {
      a += red[2 * q];
      b += red[2 * q + 1];
    }
  }
}

// ---------------------------------------------------------------------------
// Sequential single-electron Metropolis for one spin species (Sec. VMC).
// One CTA per walker; G~^{-1} lives in shared memory for the whole
// half-sweep (in global memory, L2-resident, when it does not fit).  Move m of an up electron replaces row m of G~ by the proposed
// row g' (already computed from the frozen down-spin table):
//   ratio R = g' . G~^{-1}[:, m],
//   G~^{-1} <- G~^{-1} - G~^{-1}[:, m] (g'^T G~^{-1} - e_m^T) / R   (Sherman-Morrison);
// a down electron replaces column m, with the transposed formulas.  The
// Jastrow factor contributes exp(2 dJ), dJ summed over the atoms (J1) and the
// other electrons at their current positions (J2).  Accept iff u < R^2 e^{2 dJ}.
// log|det| is not tracked move by move: the refresh that ends every
// half-sweep or sweep recomputes it from the tables.
// ---------------------------------------------------------------------------
// Acceptance probability R^2 e^{2 dJ}.  The mixed path (T = float) takes the
// exponential in FP32, like the rest of its acceptance test; FP64 where
// |2 dJ| >= 80 (FP32's range) and in the FP64 path.
template <typename T>
__device__ __forceinline__ double accept_prob(double pr, double pj) {
  if constexpr (std::is_same<T, float>::value) {
    const float x = static_cast<float>(2.0 * pj);
    if (fabsf(x) < 80.0f) return pr * pr * static_cast<double>(expf(x));
  }
  return pr * pr * exp(2.0 * pj);
}

template <typename T>
__host__ __device__ inline size_t metro_smem_per_walker(int n, int N) {
  // positions (FP64), G~^{-1}, three n-vectors, and in the mixed path the FP32
  // mirror of the positions
  const size_t mirror = std::is_same<T, float>::value ? (size_t)N * 3 * sizeof(float) : 0;
  return ((size_t)N * 3 * sizeof(double) + (size_t)(n * n + 3 * n) * sizeof(T) + mirror + 15) & ~size_t(15);
}

template <bool UP, typename T, bool GLOB>
struct Metropolis {
  static __device__ __forceinline__ void run(DevSystem s, double *__restrict__ r, const double *__restrict__ rprop,
                                             const T *__restrict__ gprop, T *__restrict__ ginv,
                                             double *__restrict__ scal, int *__restrict__ status,
                                             const T *__restrict__ pprop, T *__restrict__ phi_up,
                                             int *__restrict__ list, int *__restrict__ count,
                                             const float *__restrict__ pprop_lo, float *__restrict__ phi_lo,
                                             int m_begin, int m_end, int *__restrict__ total,
                                             double *__restrict__ j3buf, const uint3 bid, const uint3 gdim) {
    assume_global(r, rprop, gprop, ginv, scal, status, pprop, phi_up, list, count);
    extern __shared__ double sm[];
    const int n = s.n_up, N = s.N, tid = threadIdx.x, bs = blockDim.x;
    const int w = bid.x;
    T *gw = ginv + (size_t)w * n * n;
    double *xs = sm;                                  // N * 3 positions (FP64)
    // G~^{-1} in shared memory, or (GLOB, too large for it) in place in global
    // memory, where a CTA's n x n block stays resident in L2 for the half-sweep
    T *Gi = GLOB ? gw : reinterpret_cast<T *>(xs + N * 3);
    T *gp = GLOB ? reinterpret_cast<T *>(xs + N * 3) : Gi + n * n;  // n
    T *vv = gp + n;                                   // n
    T *cc = vv + n;                                   // n
    float *xf = reinterpret_cast<float *>(cc + n);    // mixed path: N * 3 positions rounded to FP32
    constexpr bool kF32 = std::is_same<T, float>::value;
    // three-body Jastrow (G~^{-1} in shared memory; its change in FP64 in both
    // paths): the walker's j3 vectors [6][LJ] and chi at the old and the
    // proposed position, chi change, after the per-walker block
    const bool j3 = !GLOB && s.use_j3 && j3buf;
    const int LJ = s.LJ;
    double *j3v = reinterpret_cast<double *>(reinterpret_cast<char *>(sm) + metro_smem_per_walker<T>(n, N));
    double *chi_o = j3v + 6 * LJ, *chi_n = chi_o + LJ, *dchi = chi_n + LJ;
    if (j3)
      for (int t = tid; t < 6 * LJ; t += bs) j3v[t] = j3buf[(size_t)w * 6 * LJ + t];
    __shared__ double red[64];
    __shared__ int s_acc;
    __shared__ double s_R;
    if (!GLOB)
      for (int t = tid; t < n * n; t += bs) Gi[t] = gw[t];
    for (int t = tid; t < N * 3; t += bs) {
      xs[t] = r[(size_t)w * N * 3 + t];
      if constexpr (kF32) xf[t] = static_cast<float>(xs[t]);
    }
    double sgn = 1.0, J = 0.0, nacc = 0.0;
    int st_bits = 0;
    if (tid == 0) {
      sgn = scal[(size_t)w * S_STRIDE + S_SIGN];
      J = scal[(size_t)w * S_STRIDE + S_J];
      nacc = scal[(size_t)w * S_STRIDE + S_NACC];
      st_bits = status[w];
    }
    const int nmoves = m_end < (UP ? s.n_up : s.n_dn) ? m_end : (UP ? s.n_up : s.n_dn);
    const int e0 = UP ? 0 : s.n_up;
    __syncthreads();
    for (int m = m_begin; m < nmoves; ++m) {
      const int e = e0 + m;
      const double *rp4 = rprop + ((size_t)w * n + m) * kPropStride;
      const double px = rp4[0], py = rp4[1], pz = rp4[2];
      for (int t = tid; t < n; t += bs) gp[t] = gprop[((size_t)w * n + m) * n + t];
      __syncthreads();
      T prt = T(0);
      double pj = 0.0;
      for (int t = tid; t < n; t += bs) prt += UP ? gp[t] * Gi[t * n + m] : Gi[m * n + t] * gp[t];
      double pr = static_cast<double>(prt);
      const double ox = xs[3 * e], oy = xs[3 * e + 1], oz = xs[3 * e + 2];
      if (tid == 0) pj = rp4[4];   // one-body Jastrow change, from the proposal kernel
      if (s.use_j2) {
        if constexpr (kF32) {
          const float pf[3] = {static_cast<float>(px), static_cast<float>(py), static_cast<float>(pz)};
          const float of[3] = {xf[3 * e], xf[3 * e + 1], xf[3 * e + 2]};
          pj += static_cast<double>(j2_move_change_f<UP>(s, xf, e, pf, of, tid, bs));
        } else {
          pj += j2_move_change<T, UP>(s, xs, e, px, py, pz, ox, oy, oz, tid, bs);
        }
      }
      if (j3) {
        // chi at the old and the proposed position (threads over the Jastrow's shells)
        for (int k = tid; k < s.n_jshells; k += bs) {
          const double4 g = s.jshell_geo[k];
          const int info = s.jshell_info[k], off = shell_off(info);
          double vo[5], vn[5];
          const int nc = shell_values(info, g.w, ox - g.x, oy - g.y, oz - g.z, vo);
          shell_values(info, g.w, px - g.x, py - g.y, pz - g.z, vn);
          for (int c = 0; c < nc; ++c) {
            chi_o[off + c] = vo[c];
            chi_n[off + c] = vn[c];
          }
        }
        __syncthreads();
        // d J3 = (chi' - chi)^T Q, Q = M_p U_s + M_a U_s' - M_p chi
        const double *Vs = j3v + (UP ? 2 : 3) * LJ, *Va = j3v + (UP ? 5 : 4) * LJ;
        for (int mu = tid; mu < LJ; mu += bs) {
          double mc = 0.0;
          for (int nu = 0; nu < LJ; ++nu) mc = fma(s.j3p[(size_t)mu * LJ + nu], chi_o[nu], mc);
          pj = fma(chi_n[mu] - chi_o[mu], Vs[mu] + Va[mu] - mc, pj);
        }
      }
      block_sum2(pr, pj, red);
      if (tid == 0) {
        const double u = rp4[3];
        const double p = accept_prob<T>(pr, pj);
        int acc = 0;
        if (!isfinite(p) || !isfinite(pr)) {
          st_bits |= JAGP_WS_NONFINITE;
        } else if (pr != 0.0 && u < p) {
          acc = 1;
          if (pr < 0.0) sgn = -sgn;
          J += pj;
          nacc += 1.0;
          list[atomicAdd(count, 1)] = w * n + m;
          if (total) atomicAdd(total, 1);
        }
        s_acc = acc;
        s_R = pr;
      }
      __syncthreads();
      if (s_acc) {
        if (GLOB && !UP) {
          // rows of G~^{-1} against g': one warp per row, coalesced loads
          const int lane = tid & 31, nw = bs >> 5;
          for (int t = tid >> 5; t < n; t += nw) {
            T a = T(0);
            for (int i = lane; i < n; i += 32) a += Gi[t * n + i] * gp[i];
            a = warp_sum(a);
            if (lane == 0) vv[t] = a;
          }
          for (int t = tid; t < n; t += bs) cc[t] = Gi[m * n + t];
        } else {
          for (int t = tid; t < n; t += bs) {
            T a = T(0);
            if (UP) {
              for (int j = 0; j < n; ++j) a += gp[j] * Gi[j * n + t];
              cc[t] = Gi[t * n + m];
            } else {
              for (int i = 0; i < n; ++i) a += Gi[t * n + i] * gp[i];
              cc[t] = Gi[m * n + t];
            }
            vv[t] = a;
          }
        }
        __syncthreads();
        const T invR = T(1) / static_cast<T>(s_R);
        for (int idx = tid; idx < n * n; idx += bs) {
          const int j = idx / n, k = idx - j * n;
          if (UP)
            Gi[idx] -= cc[j] * (vv[k] - (k == m ? T(1) : T(0))) * invR;
          else
            Gi[idx] -= (vv[j] - (j == m ? T(1) : T(0))) * cc[k] * invR;
        }
        if (tid == 0) {
          xs[3 * e] = px;
          xs[3 * e + 1] = py;
          xs[3 * e + 2] = pz;
          if constexpr (kF32) {
            xf[3 * e] = static_cast<float>(px);
            xf[3 * e + 1] = static_cast<float>(py);
            xf[3 * e + 2] = static_cast<float>(pz);
          }
        }
        if (UP) {
          const size_t row = ((size_t)w * n + m) * s.L;
          for (int t = tid; t < s.L; t += bs) phi_up[row + t] = pprop[row + t];
          if (phi_lo)
            for (int t = tid; t < s.L; t += bs) phi_lo[row + t] = pprop_lo[row + t];
        }
        if (j3) {
          // the spin sum and its two products follow the moved electron
          for (int t = tid; t < LJ; t += bs) dchi[t] = chi_n[t] - chi_o[t];
          __syncthreads();
          double *U = j3v + (UP ? 0 : 1) * LJ, *Up = j3v + (UP ? 2 : 3) * LJ, *Ua = j3v + (UP ? 4 : 5) * LJ;
          for (int mu = tid; mu < LJ; mu += bs) {
            double ap = 0.0, aa = 0.0;
            for (int nu = 0; nu < LJ; ++nu) {
              ap = fma(s.j3p[(size_t)mu * LJ + nu], dchi[nu], ap);
              aa = fma(s.j3a[(size_t)mu * LJ + nu], dchi[nu], aa);
            }
            U[mu] += dchi[mu];
            Up[mu] += ap;
            Ua[mu] += aa;
          }
        }
      }
      __syncthreads();
    }
    if (j3)
      for (int t = tid; t < 6 * LJ; t += bs) j3buf[(size_t)w * 6 * LJ + t] = j3v[t];
    if (!GLOB)
      for (int t = tid; t < n * n; t += bs) gw[t] = Gi[t];
    for (int t = tid; t < N * 3; t += bs) r[(size_t)w * N * 3 + t] = xs[t];
    if (tid == 0) {
      scal[(size_t)w * S_STRIDE + S_SIGN] = sgn;
      scal[(size_t)w * S_STRIDE + S_J] = J;
      scal[(size_t)w * S_STRIDE + S_NACC] = nacc;
      status[w] = st_bits;
    }
}
};
template <bool UP, typename T, bool GLOB>
__global__ void __launch_bounds__(512) k_metropolis(DevSystem s, double *__restrict__ r,
                                                    const double *__restrict__ rprop, const T *__restrict__ gprop,
                                                    T *__restrict__ ginv, double *__restrict__ scal,
                                                    int *__restrict__ status, const T *__restrict__ pprop,
                                                    T *__restrict__ phi_up, int *__restrict__ list,
                                                    int *__restrict__ count, const float *__restrict__ pprop_lo,
                                                    float *__restrict__ phi_lo, int m_begin, int m_end,
                                                    int *__restrict__ total, double *__restrict__ j3buf) {
  Metropolis<UP, T, GLOB>::run(s, r, rprop, gprop, ginv, scal, status, pprop, phi_up, list, count, pprop_lo, phi_lo,
                               m_begin, m_end, total, j3buf, blockIdx, gridDim);
}

// ---------------------------------------------------------------------------
// The same acceptance loop with one warp per walker (N_up <= 32): G~^{-1} in
// the warp's slice of shared memory, reductions by shuffles, no block barriers.
// Every lane takes the accept decision from lane 0's sums so that it is uniform.
// ---------------------------------------------------------------------------
// ---------------------------------------------------------------------------
// Metropolis sampling of the guiding function Psi_G = (max(R, eps) / R) Psi_T
// (Sec. "Atomic forces", Eqs. guiding_function, R_r, regularization) for the
// FP64 path with N_up <= 64: R = (S F)^-theta, F = sum |G~^{-1}|^2,
// S = min_i sum_j |G~_ij|^2, and a move is accepted with probability
// |Psi_T(x')/Psi_T(x)|^2 W(x) / W(x'), W = (R / max(R, eps))^2.  One CTA per
// walker with G~^{-1} and G~ in shared memory.  For the proposed replacement
// of row (up) or column (down) m by g' with ratio R_d, the Sherman-Morrison
// form A' = A - c (v - e_m)^T / R_d (up; the transpose for down) gives
//   |A'|^2 = |A|^2 - 2 (w . (v - e_m)) / R_d + |c|^2 |v - e_m|^2 / R_d^2,
// with w = c^T A (up) or A c (down), so F' costs O(N_up^2) per proposal; the
// row sums of squares of G~ follow the replaced row or column.  F and the row
// sums are recomputed at every launch; G~ is kept current in gmat.
// ---------------------------------------------------------------------------
template <bool UP>
__global__ void __launch_bounds__(128) k_metropolis_guided(DevSystem s, double *__restrict__ r,
                                                           const double *__restrict__ rprop,
                                                           const double *__restrict__ gprop,
                                                           double *__restrict__ ginv, double *__restrict__ scal,
                                                           int *__restrict__ status, const double *__restrict__ pprop,
                                                           double *__restrict__ phi_up, int *__restrict__ list,
                                                           int *__restrict__ count, double *__restrict__ gmat,
                                                           double theta, double eps, int m_begin, int m_end,
                                                           int *__restrict__ total) {
  extern __shared__ double sm[];
  const int n = s.n_up, N = s.N, tid = threadIdx.x, bs = blockDim.x;
  const int w = blockIdx.x;
  double *gw = ginv + (size_t)w * n * n, *gg = gmat + (size_t)w * n * n;
  double *xs = sm;              // N * 3
  double *Gi = xs + N * 3;      // n * n  G~^{-1}
  double *Gm = Gi + n * n;      // n * n  G~
  double *gp = Gm + n * n;      // n      proposed row / column of G~
  double *vv = gp + n;          // n
  double *cc = vv + n;          // n
  double *ww = cc + n;          // n
  double *rn = ww + n;          // n      row sums of squares of G~
  __shared__ double red[8][4];
  __shared__ int s_acc;
  __shared__ double s_R, s_F, s_W;
  for (int t = tid; t < n * n; t += bs) {
    Gi[t] = gw[t];
    Gm[t] = gg[t];
  }
  for (int t = tid; t < N * 3; t += bs) xs[t] = r[(size_t)w * N * 3 + t];
  __syncthreads();
  // F and the row sums of the current configuration
  double f = 0.0;
  for (int t = tid; t < n * n; t += bs) f = fma(Gi[t], Gi[t], f);
  for (int i = tid; i < n; i += bs) {
    double q = 0.0;
    for (int j = 0; j < n; ++j) q = fma(Gm[i * n + j], Gm[i * n + j], q);
    rn[i] = q;
  }
  f = warp_sum(f);
  if ((tid & 31) == 0) red[tid >> 5][0] = f;
  __syncthreads();
  if (tid == 0) {
    double F = 0.0, S = INFINITY;
    for (int q = 0; q < (bs >> 5); ++q) F += red[q][0];
    for (int i = 0; i < n; ++i) S = fmin(S, rn[i]);
    const double R = pow(S * F, -theta), qw = R / fmax(R, eps);
    s_F = F;
    s_W = qw * qw;
  }
  double sgn = 1.0, J = 0.0, nacc = 0.0;
  int st_bits = 0;
  if (tid == 0) {
    sgn = scal[(size_t)w * S_STRIDE + S_SIGN];
    J = scal[(size_t)w * S_STRIDE + S_J];
    nacc = scal[(size_t)w * S_STRIDE + S_NACC];
    st_bits = status[w];
  }
  const int nmoves = m_end < (UP ? s.n_up : s.n_dn) ? m_end : (UP ? s.n_up : s.n_dn);
  const int e0 = UP ? 0 : s.n_up;
  __syncthreads();
  for (int m = m_begin; m < nmoves; ++m) {
    const int e = e0 + m;
    const double *rp4 = rprop + ((size_t)w * n + m) * kPropStride;
    const double px = rp4[0], py = rp4[1], pz = rp4[2];
    for (int t = tid; t < n; t += bs) gp[t] = gprop[((size_t)w * n + m) * n + t];
    __syncthreads();
    double pr = 0.0, pj = 0.0;
    for (int t = tid; t < n; t += bs) pr += UP ? gp[t] * Gi[t * n + m] : Gi[m * n + t] * gp[t];
    const double ox = xs[3 * e], oy = xs[3 * e + 1], oz = xs[3 * e + 2];
    if (tid == 0) pj = rp4[4];
    if (s.use_j2) pj += j2_move_change<double, UP>(s, xs, e, px, py, pz, ox, oy, oz, tid, bs);
    // v, c and w of the Sherman-Morrison form, for the proposal whether or not it is taken
    for (int t = tid; t < n; t += bs) {
      double a = 0.0;
      if (UP) {
        for (int j = 0; j < n; ++j) a = fma(gp[j], Gi[j * n + t], a);
        cc[t] = Gi[t * n + m];
      } else {
        for (int i = 0; i < n; ++i) a = fma(Gi[t * n + i], gp[i], a);
        cc[t] = Gi[m * n + t];
      }
      vv[t] = a;
    }
    __syncthreads();
    for (int t = tid; t < n; t += bs) {
      double a = 0.0;
      if (UP)
        for (int j = 0; j < n; ++j) a = fma(cc[j], Gi[j * n + t], a);
      else
        for (int k = 0; k < n; ++k) a = fma(Gi[t * n + k], cc[k], a);
      ww[t] = a;
    }
    __syncthreads();
    double d1 = 0.0, cn = 0.0, un = 0.0, smin = INFINITY;
    for (int t = tid; t < n; t += bs) {
      const double u = vv[t] - (t == m ? 1.0 : 0.0);
      d1 = fma(ww[t], u, d1);
      cn = fma(cc[t], cc[t], cn);
      un = fma(u, u, un);
      // row sums of G~ after the replacement
      double rt;
      if (!UP) {
        rt = rn[t] - Gm[t * n + m] * Gm[t * n + m] + gp[t] * gp[t];
      } else if (t != m) {
        rt = rn[t];
      } else {
        rt = 0.0;
        for (int j = 0; j < n; ++j) rt = fma(gp[j], gp[j], rt);
      }
      smin = fmin(smin, rt);
    }
    pr = warp_sum(pr);
    pj = warp_sum(pj);
    d1 = warp_sum(d1);
    cn = warp_sum(cn);
    un = warp_sum(un);
    for (int o = 16; o > 0; o >>= 1) smin = fmin(smin, __shfl_xor_sync(0xffffffffu, smin, o));
    const int warp = tid >> 5, lane = tid & 31, nw = bs >> 5;
    __syncthreads();
    if (lane == 0) {
      red[warp][0] = pr;
      red[warp][1] = pj;
      red[warp][2] = d1;
      red[warp][3] = smin;
    }
    __shared__ double red2[8][2];
    if (lane == 0) {
      red2[warp][0] = cn;
      red2[warp][1] = un;
    }
    __syncthreads();
    if (tid == 0) {
      double P = 0.0, PJ = 0.0, D = 0.0, C = 0.0, U = 0.0, Sm = INFINITY;
      for (int q = 0; q < nw; ++q) {
        P += red[q][0];
        PJ += red[q][1];
        D += red[q][2];
        Sm = fmin(Sm, red[q][3]);
        C += red2[q][0];
        U += red2[q][1];
      }
      const double Fp = s_F - 2.0 * D / P + C * U / (P * P);
      const double Rp = pow(Sm * Fp, -theta), qw = Rp / fmax(Rp, eps), Wp = qw * qw;
      const double u = rp4[3];
      const double p = P * P * exp(2.0 * PJ) * (s_W / Wp);
      int acc = 0;
      if (!isfinite(p) || !isfinite(P)) {
        st_bits |= JAGP_WS_NONFINITE;
      } else if (P != 0.0 && u < p) {
        acc = 1;
        if (P < 0.0) sgn = -sgn;
        J += PJ;
        nacc += 1.0;
        list[atomicAdd(count, 1)] = w * n + m;
        if (total) atomicAdd(total, 1);
        s_F = Fp;
        s_W = Wp;
      }
      s_acc = acc;
      s_R = P;
    }
    __syncthreads();
    if (s_acc) {
      const double invR = 1.0 / s_R;
      for (int idx = tid; idx < n * n; idx += bs) {
        const int j = idx / n, k = idx - j * n;
        if (UP)
          Gi[idx] -= cc[j] * (vv[k] - (k == m ? 1.0 : 0.0)) * invR;
        else
          Gi[idx] -= (vv[j] - (j == m ? 1.0 : 0.0)) * cc[k] * invR;
      }
      // G~ and its row sums follow the replaced row / column
      for (int t = tid; t < n; t += bs) {
        if (UP) {
          Gm[m * n + t] = gp[t];
        } else {
          rn[t] = rn[t] - Gm[t * n + m] * Gm[t * n + m] + gp[t] * gp[t];
          Gm[t * n + m] = gp[t];
        }
      }
      if (tid == 0) {
        xs[3 * e] = px;
        xs[3 * e + 1] = py;
        xs[3 * e + 2] = pz;
      }
      if (UP) {
        const size_t row = ((size_t)w * n + m) * s.L;
        for (int t = tid; t < s.L; t += bs) phi_up[row + t] = pprop[row + t];
      }
      __syncthreads();
      if (UP && tid == 0) {
        double q = 0.0;
        for (int j = 0; j < n; ++j) q = fma(gp[j], gp[j], q);
        rn[m] = q;
      }
    }
    __syncthreads();
  }
  for (int t = tid; t < n * n; t += bs) {
    gw[t] = Gi[t];
    gg[t] = Gm[t];
  }
  for (int t = tid; t < N * 3; t += bs) r[(size_t)w * N * 3 + t] = xs[t];
  if (tid == 0) {
    scal[(size_t)w * S_STRIDE + S_SIGN] = sgn;
    scal[(size_t)w * S_STRIDE + S_J] = J;
    scal[(size_t)w * S_STRIDE + S_NACC] = nacc;
    status[w] = st_bits;
  }
}

cudaError_t launch_metropolis_guided(const DevSystem &s, bool up, double *r, const double *rprop,
                                     const double *gprop, double *ginv, double *scal, int *status,
                                     const double *pprop, double *phi_up, int *list, int *count, double *gmat,
                                     double theta, double eps, int W, cudaStream_t st, int m_begin, int m_end,
                                     int *total) {
  if (W <= 0 || (!up && s.n_dn == 0)) return cudaSuccess;
  if (s.n_up > kGuidedMaxUp) return cudaErrorInvalidValue;
  if (m_end < 0) m_end = up ? s.n_up : s.n_dn;
  if (m_begin >= m_end) return cudaSuccess;
  const int n = s.n_up;
  // positions (3N), G~^{-1} and G~ (n^2 each), five n-vectors
  const size_t smem = ((size_t)s.N * 3 + 2 * (size_t)n * n + 5 * (size_t)n + 1) * sizeof(double);
  if (smem > 200 * 1024) return cudaErrorInvalidValue;
  if (up)
    k_metropolis_guided<true><<<W, 128, smem, st>>>(s, r, rprop, gprop, ginv, scal, status, pprop, phi_up, list,
                                                    count, gmat, theta, eps, m_begin, m_end, total);
  else
    k_metropolis_guided<false><<<W, 128, smem, st>>>(s, r, rprop, gprop, ginv, scal, status, pprop, phi_up, list,
                                                     count, gmat, theta, eps, m_begin, m_end, total);
  return cudaGetLastError();
}

constexpr int kMetroWarps = 4;
constexpr size_t kMetroSmemMax = 200 * 1024;  // G~^{-1} kept in shared memory up to this footprint


template <bool UP, typename T>
struct MetropolisWarp {
  // latency-bound (one walker's sequential moves per warp): keep six CTAs of
  // four warps resident per SM
  static constexpr int kMinBlocks = 6;
  static __device__ __forceinline__ void run(DevSystem s, double *__restrict__ r, const double *__restrict__ rprop,
                                             const T *__restrict__ gprop, T *__restrict__ ginv,
                                             double *__restrict__ scal, int *__restrict__ status,
                                             const T *__restrict__ pprop, T *__restrict__ phi_up,
                                             int *__restrict__ list, int *__restrict__ count, int W,
                                             const float *__restrict__ pprop_lo, float *__restrict__ phi_lo,
                                             int m_begin, int m_end, int *__restrict__ total, const uint3 bid,
                                             const uint3 gdim) {
    assume_global(r, rprop, gprop, ginv, scal, status, pprop, phi_up, list, count);
    extern __shared__ double sm[];
    const int n = s.n_up, N = s.N, lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int w = bid.x * kMetroWarps + warp;
    if (w >= W) return;  // warp-uniform; the kernel has no block-wide barrier
    double *xs = reinterpret_cast<double *>(reinterpret_cast<char *>(sm) + warp * metro_smem_per_walker<T>(n, N));
    T *Gi = reinterpret_cast<T *>(xs + N * 3);
    T *gp = Gi + n * n;
    T *vv = gp + n;
    T *cc = vv + n;
    float *xf = reinterpret_cast<float *>(cc + n);  // mixed path: N * 3 positions rounded to FP32
    constexpr bool kF32 = std::is_same<T, float>::value;
    T *gw = ginv + (size_t)w * n * n;
    for (int t = lane; t < n * n; t += 32) Gi[t] = gw[t];
    for (int t = lane; t < N * 3; t += 32) {
      xs[t] = r[(size_t)w * N * 3 + t];
      if constexpr (kF32) xf[t] = static_cast<float>(xs[t]);
    }
    double *sw = scal + (size_t)w * S_STRIDE;
    double sgn = sw[S_SIGN], J = sw[S_J], nacc = sw[S_NACC];
    int st_bits = status[w];
    const int nmoves = m_end < (UP ? s.n_up : s.n_dn) ? m_end : (UP ? s.n_up : s.n_dn);
    const int e0 = UP ? 0 : s.n_up;
    __syncwarp();
    for (int m = m_begin; m < nmoves; ++m) {
      const int e = e0 + m;
      const double *rec = rprop + ((size_t)w * n + m) * kPropStride;
      const double px = rec[0], py = rec[1], pz = rec[2];
      const T *grow = gprop + ((size_t)w * n + m) * n;
      T prt = T(0);
      double pj = 0.0;
      for (int t = lane; t < n; t += 32) {
        const T g = grow[t];
        gp[t] = g;
        prt += UP ? g * Gi[t * n + m] : Gi[m * n + t] * g;
      }
      double pr;
      if constexpr (kF32) {
        // ratio and two-body change summed in FP32 (the acceptance test's precision)
        float pjf = 0.0f;
        if (s.use_j2) {
          const float pf[3] = {static_cast<float>(px), static_cast<float>(py), static_cast<float>(pz)};
          const float of[3] = {xf[3 * e], xf[3 * e + 1], xf[3 * e + 2]};
          pjf = j2_move_change_f<UP>(s, xf, e, pf, of, lane, 32);
        }
        pr = static_cast<double>(__shfl_sync(0xffffffffu, warp_sum(prt), 0));
        pj = rec[4] + static_cast<double>(__shfl_sync(0xffffffffu, warp_sum(pjf), 0));
      } else {
        pr = static_cast<double>(prt);
        if (lane == 0) pj = rec[4];
        if (s.use_j2)
          pj += j2_move_change<T, UP>(s, xs, e, px, py, pz, xs[3 * e], xs[3 * e + 1], xs[3 * e + 2], lane, 32);
        pr = __shfl_sync(0xffffffffu, warp_sum(pr), 0);
        pj = __shfl_sync(0xffffffffu, warp_sum(pj), 0);
      }
      const double p = accept_prob<T>(pr, pj);
      int acc = 0;
      if (!isfinite(p) || !isfinite(pr)) {
        st_bits |= JAGP_WS_NONFINITE;
      } else if (pr != 0.0 && rec[3] < p) {
        acc = 1;
      }
      __syncwarp();
      if (acc) {
        if (pr < 0.0) sgn = -sgn;
        J += pj;
        nacc += 1.0;
        if (lane == 0) {
          list[atomicAdd(count, 1)] = w * n + m;
          if (total) atomicAdd(total, 1);
        }
        for (int t = lane; t < n; t += 32) {
          T a = T(0);
          if (UP) {
            for (int j = 0; j < n; ++j) a = fma(gp[j], Gi[j * n + t], a);
            cc[t] = Gi[t * n + m];
          } else {
            for (int i = 0; i < n; ++i) a = fma(Gi[t * n + i], gp[i], a);
            cc[t] = Gi[m * n + t];
          }
          vv[t] = a;
        }
        __syncwarp();
        const T invR = T(1) / static_cast<T>(pr);
        for (int idx = lane; idx < n * n; idx += 32) {
          const int j = idx / n, k = idx - j * n;
          if (UP)
            Gi[idx] -= cc[j] * (vv[k] - (k == m ? T(1) : T(0))) * invR;
          else
            Gi[idx] -= (vv[j] - (j == m ? T(1) : T(0))) * cc[k] * invR;
        }
        if (lane < 3) {
          const double v = lane == 0 ? px : (lane == 1 ? py : pz);
          xs[3 * e + lane] = v;
          if constexpr (kF32) xf[3 * e + lane] = static_cast<float>(v);
        }
        if (UP) {
          const size_t row = ((size_t)w * n + m) * s.L;
          for (int t = lane; t < s.L; t += 32) phi_up[row + t] = pprop[row + t];
          if (phi_lo)
            for (int t = lane; t < s.L; t += 32) phi_lo[row + t] = pprop_lo[row + t];
        }
        __syncwarp();
      }
    }
    for (int t = lane; t < n * n; t += 32) gw[t] = Gi[t];
    for (int t = lane; t < N * 3; t += 32) r[(size_t)w * N * 3 + t] = xs[t];
    if (lane == 0) {
      sw[S_SIGN] = sgn;
      sw[S_J] = J;
      sw[S_NACC] = nacc;
      status[w] = st_bits;
    }
}
};
template <bool UP, typename T>
__global__ void __launch_bounds__(kMetroWarps * 32) k_metropolis_warp(DevSystem s, double *__restrict__ r,
    const double *__restrict__ rprop, const T *__restrict__ gprop, T *__restrict__ ginv, double *__restrict__ scal,
    int *__restrict__ status, const T *__restrict__ pprop, T *__restrict__ phi_up, int *__restrict__ list,
    int *__restrict__ count, int W, const float *__restrict__ pprop_lo, float *__restrict__ phi_lo, int m_begin,
    int m_end, int *__restrict__ total) {
  MetropolisWarp<UP, T>::run(s, r, rprop, gprop, ginv, scal, status, pprop, phi_up, list, count, W, pprop_lo, phi_lo,
                             m_begin, m_end, total, blockIdx, gridDim);
}

template <typename T>
cudaError_t launch_metropolis(const DevSystem &s, bool up, double *r, const double *rprop, const T *gprop, T *ginv,
                              double *scal, int *status, const T *pprop, T *phi_up, int *list, int *count, int W,
                              cudaStream_t st, const float *pprop_lo, float *phi_lo, int m_begin, int m_end,
                              int *total, double *j3buf) {
  if (W <= 0 || (!up && s.n_dn == 0)) return cudaSuccess;
  if (m_end < 0) m_end = up ? s.n_up : s.n_dn;
  if (m_begin >= m_end) return cudaSuccess;
  const int n = s.n_up;
  // one CTA per walker (threads per CTA, shared memory, G~^{-1} in shared or global memory)
  auto cta = [&](int threads, size_t smem, bool glob, double *j3) -> cudaError_t {
    if (glob) {
      if (up)
        return launch_or_record<Metropolis<true, T, true>, 512>(k_metropolis<true, T, true>, dim3(W), dim3(threads), smem, st, s, r, rprop, gprop,
                                                                ginv, scal, status, pprop, phi_up, list, count,
                                                                pprop_lo, phi_lo, m_begin, m_end, total, j3);
      return launch_or_record<Metropolis<false, T, true>, 512>(k_metropolis<false, T, true>, dim3(W), dim3(threads), smem, st, s, r, rprop, gprop,
                                                               ginv, scal, status, pprop, phi_up, list, count,
                                                               pprop_lo, phi_lo, m_begin, m_end, total, j3);
    }
    if (up)
      return launch_or_record<Metropolis<true, T, false>, 512>(k_metropolis<true, T, false>, dim3(W), dim3(threads), smem, st, s, r, rprop, gprop,
                                                               ginv, scal, status, pprop, phi_up, list, count,
                                                               pprop_lo, phi_lo, m_begin, m_end, total, j3);
    return launch_or_record<Metropolis<false, T, false>, 512>(k_metropolis<false, T, false>, dim3(W), dim3(threads), smem, st, s, r, rprop, gprop,
                                                              ginv, scal, status, pprop, phi_up, list, count,
                                                              pprop_lo, phi_lo, m_begin, m_end, total, j3);
  };
  if (s.use_j3) {
    // the three-body Jastrow's change is formed in the CTA-per-walker kernel
    const size_t per3 = metro_smem_per_walker<T>(n, s.N) + (size_t)9 * s.LJ * sizeof(double);
    if (!j3buf || per3 > kMetroSmemMax) return cudaErrorInvalidValue;
    return cta(n <= 64 ? 128 : 256, per3, false, j3buf);
  }
  const size_t per = metro_smem_per_walker<T>(n, s.N);
  if (n <= 32) {
    const int blocks = (W + kMetroWarps - 1) / kMetroWarps;
    if (up)
      return launch_or_record<MetropolisWarp<true, T>, kMetroWarps * 32>(k_metropolis_warp<true, T>, 
          dim3(blocks), dim3(kMetroWarps * 32), per * kMetroWarps, st, s, r, rprop, gprop, ginv, scal, status, pprop,
          phi_up, list, count, W, pprop_lo, phi_lo, m_begin, m_end, total);
    return launch_or_record<MetropolisWarp<false, T>, kMetroWarps * 32>(k_metropolis_warp<false, T>, 
        dim3(blocks), dim3(kMetroWarps * 32), per * kMetroWarps, st, s, r, rprop, gprop, ginv, scal, status, pprop,
        phi_up, list, count, W, pprop_lo, phi_lo, m_begin, m_end, total);
  }
  if (per <= kMetroSmemMax) return cta(n <= 64 ? 128 : 256, per, false, nullptr);
  const size_t glob = (size_t)s.N * 3 * sizeof(double) + (size_t)3 * n * sizeof(T) +
                      (std::is_same<T, float>::value ? (size_t)s.N * 3 * sizeof(float) : 0);
  return cta(512, glob, true, nullptr);
}
template cudaError_t launch_metropolis<double>(const DevSystem &, bool, double *, const double *, const double *,
                                               double *, double *, int *, const double *, double *, int *, int *,
                                               int, cudaStream_t, const float *, float *, int, int, int *, double *);
template cudaError_t launch_metropolis<float>(const DevSystem &, bool, double *, const double *, const float *,
                                              float *, double *, int *, const float *, float *, int *, int *, int,
                                              cudaStream_t, const float *, float *, int, int, int *, double *);

// ---------------------------------------------------------------------------
// J = J1 + J2 of each walker from scratch (one CTA per walker).
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(128) k_jastrow_full(DevSystem s, const double *__restrict__ r,
                                                      double *__restrict__ scal, const double *__restrict__ j3buf) {
  const int w = blockIdx.x, N = s.N;
  const double *x = r + (size_t)w * N * 3;
  __shared__ double red[64];
  double j1 = 0.0, j2 = 0.0;
  if (s.use_j1)
    for (int idx = threadIdx.x; idx < N * s.n_atoms; idx += blockDim.x) {
      const int i = idx / s.n_atoms, a = idx - i * s.n_atoms;
      const double dx = x[3 * i] - s.R[3 * a], dy = x[3 * i + 1] - s.R[3 * a + 1], dz = x[3 * i + 2] - s.R[3 * a + 2];
      j1 += j1_val(s.c1[a], s.b_ea, sqrt(dx * dx + dy * dy + dz * dz));
    }
  if (s.use_j2)
    for (int idx = threadIdx.x; idx < N * N; idx += blockDim.x) {
      const int i = idx / N, j = idx - i * N;
      if (j <= i) continue;
      double kk, bb;
      j2_params(s, (i < s.n_up) == (j < s.n_up), &kk, &bb);
      const double dx = x[3 * i] - x[3 * j], dy = x[3 * i + 1] - x[3 * j + 1], dz = x[3 * i + 2] - x[3 * j + 2];
      j2 += j2_val(kk, bb, sqrt(dx * dx + dy * dy + dz * dz));
    }
  if (s.use_j3 && j3buf)
    for (int i = threadIdx.x; i < N; i += blockDim.x) {
      double g3[3] = {0.0, 0.0, 0.0}, l3 = 0.0;
      j3_electron(s, j3buf + (size_t)w * 6 * s.LJ, i < s.n_up, x[3 * i], x[3 * i + 1], x[3 * i + 2], &j2, g3, &l3);
    }
  block_sum2(j1, j2, red);
  if (threadIdx.x == 0) scal[(size_t)w * S_STRIDE + S_J] = j1 + j2;
}

cudaError_t launch_jastrow_full(const DevSystem &s, const double *r, double *scal, int W, cudaStream_t st,
                                const double *j3buf) {
  if (W <= 0) return cudaSuccess;
  if (s.use_j3 && !j3buf) return cudaErrorInvalidValue;
  k_jastrow_full<<<W, 128, 0, st>>>(s, r, scal, j3buf);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// bookkeeping
// ---------------------------------------------------------------------------
// clears the counters and flags a walker with a non-finite coordinate
__global__ void k_walker_init(double *scal, int *status, int W, const double *r, int N) {
  const int w = blockIdx.x * blockDim.x + threadIdx.x;
  if (w >= W) return;
  scal[(size_t)w * S_STRIDE + S_NACC] = 0.0;
  scal[(size_t)w * S_STRIDE + S_DRIFT] = 0.0;
  int bits = 0;
  if (r)
    for (int q = 0; q < 3 * N; ++q)
      if (!isfinite(r[(size_t)w * 3 * N + q])) bits = JAGP_WS_NONFINITE;
  status[w] = bits;
}

cudaError_t launch_walker_init(double *scal, int *status, int W, cudaStream_t st, const double *r, int N) {
  if (W <= 0) return cudaSuccess;
  k_walker_init<<<(W + 255) / 256, 256, 0, st>>>(scal, status, W, r, N);
  return cudaGetLastError();
}

__global__ void k_logpsi_out(const double *scal, int W, double *logabs, double *sign) {
  const int w = blockIdx.x * blockDim.x + threadIdx.x;
  if (w >= W) return;
  const double *sw = scal + (size_t)w * S_STRIDE;
  if (logabs) logabs[w] = sw[S_LOGDET] + sw[S_J];
  if (sign) sign[w] = sw[S_SIGN];
}

cudaError_t launch_logpsi_out(const double *scal, int W, double *logabs, double *sign, cudaStream_t st) {
  if (W <= 0 || (!logabs && !sign)) return cudaSuccess;
  k_logpsi_out<<<(W + 255) / 256, 256, 0, st>>>(scal, W, logabs, sign);
  return cudaGetLastError();
}

__global__ void k_walker_info(const double *scal, const int *status, int W, double *logabs, double *sign,
                              double *nacc, double *drift, int *st_out) {
  const int w = blockIdx.x * blockDim.x + threadIdx.x;
  if (w >= W) return;
  const double *sw = scal + (size_t)w * S_STRIDE;
  if (logabs) logabs[w] = sw[S_LOGDET] + sw[S_J];
  if (sign) sign[w] = sw[S_SIGN];
  if (nacc) nacc[w] = sw[S_NACC];
  if (drift) drift[w] = sw[S_DRIFT];
  if (st_out) st_out[w] = status[w];
}

cudaError_t launch_walker_info(const double *scal, const int *status, int W, double *logabs, double *sign,
                               double *nacc, double *drift, int *st_out, cudaStream_t st) {
  if (W <= 0) return cudaSuccess;
  k_walker_info<<<(W + 255) / 256, 256, 0, st>>>(scal, status, W, logabs, sign, nacc, drift, st_out);
  return cudaGetLastError();
}

// Per-sweep accumulators in a fixed reduction order (bitwise reproducible):
// acc = (sum e_L, sum e_L^2, accepted moves of this sweep, max drift).
struct ReduceAcc {
  static __device__ __forceinline__ void run(const double *eL, const double *scal, const int *count, int W,
                                             double *acc, int accumulate, const uint3 bid, const uint3 gdim) {
    __shared__ double s1[1024], s2[1024], s3[1024];
    double a = 0.0, b = 0.0, d = 0.0;
    for (int w = threadIdx.x; w < W; w += blockDim.x) {
      if (eL) {
        const double e = eL[w];
        a += e;
        b += e * e;
      }
      d = fmax(d, scal[(size_t)w * S_STRIDE + S_DRIFT]);
    }
    s1[threadIdx.x] = a;
    s2[threadIdx.x] = b;
    s3[threadIdx.x] = d;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
      if ((int)threadIdx.x < o) {
        s1[threadIdx.x] += s1[threadIdx.x + o];
        s2[threadIdx.x] += s2[threadIdx.x + o];
        s3[threadIdx.x] = fmax(s3[threadIdx.x], s3[threadIdx.x + o]);
      }
      __syncthreads();
    }
    if (threadIdx.x == 0) {
      const double c = (double)count[0] + (double)count[1];
      if (accumulate) {
        acc[0] += s1[0];
        acc[1] += s2[0];
        acc[2] += c;
        acc[3] = fmax(acc[3], s3[0]);
      } else {
        acc[0] = s1[0];
        acc[1] = s2[0];
        acc[2] = c;
        acc[3] = s3[0];
      }
    }
}
};
__global__ void __launch_bounds__(1024) k_reduce_acc(const double *eL, const double *scal, const int *count, int W,
                                                     double *acc, int accumulate) {
  ReduceAcc::run(eL, scal, count, W, acc, accumulate, blockIdx, gridDim);
}

cudaError_t launch_reduce_acc(const double *eL, const double *scal, const int *count, int W, double *acc,
                              cudaStream_t st, int accumulate) {
  return launch_or_record<ReduceAcc, 1024>(k_reduce_acc, dim3(1), dim3(1024), 0, st, eL, scal, count, W, acc, accumulate);
}

// zero n ints (a memset that the grouped launches can take)
struct ZeroInts {
  static __device__ __forceinline__ void run(int *p, int n, const uint3 bid, const uint3 gdim) {
    for (int i = (int)(bid.x * blockDim.x + threadIdx.x); i < n; i += (int)(gdim.x * blockDim.x)) p[i] = 0;
  }
};
__global__ void __launch_bounds__(32) k_zero_ints(int *p, int n) { ZeroInts::run(p, n, blockIdx, gridDim); }

cudaError_t zero_ints(int *p, int n, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  if (group_recorder()) return launch_or_record<ZeroInts, 32>(k_zero_ints, dim3(1), dim3(32), 0, st, p, n);
  return cudaMemsetAsync(p, 0, (size_t)n * sizeof(int), st);
}

__global__ void k_increment(uint32_t *c, uint32_t by) {
  if (threadIdx.x == 0) *c += by;
}

cudaError_t launch_increment(uint32_t *c, uint32_t by, cudaStream_t st) {
  k_increment<<<1, 32, 0, st>>>(c, by);
  return cudaGetLastError();
}

}  // namespace jagp

namespace jagp {
cudaError_t setup_walker_attributes() {
  // (the kernels launched through launch_or_record raise their own limit)
  cudaError_t e = cudaFuncSetAttribute(k_metropolis_guided<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       200 * 1024);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_metropolis_guided<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  return e;
}
}  // namespace jagp
