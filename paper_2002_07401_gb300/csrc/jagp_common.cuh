// jagp_common.cuh -- device-side definitions shared by the libjagp kernels.
//
// Everything here is the GPU path's own code; the CPU oracle shares none of it.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/jagp.h"

namespace jagp {

constexpr int kMaxUp = 64;          // N_up handled with G~^{-1} resident in shared memory
constexpr int kWarp = 32;
constexpr int kPropStride = 8;     // doubles per proposal record

// Shell record packed for one 32-byte load: centre (x, y, z) and exponent.
// info = l | radial << 2 | first-function-offset << 8.
struct DevSystem {
  int n_atoms, n_shells, L, n_up, n_dn, N;
  const double *R;          // [n_atoms][3]
  const double *Z;          // [n_atoms]
  const double *c1;         // (2 Z_a)^{1/4}
  const double4 *shell_geo; // [n_shells]
  const int *shell_info;    // [n_shells]
  const double *lam;        // [L][L]
  const double *lamT;       // [L][L] = lambda^T
  const double *unpaired;   // [n_up - n_dn][L]
  double b_ea, b_para, b_anti;
  int use_j1, use_j2, j2_si;
  double v_ii;              // ion-ion repulsion (a constant of the system)
  double delta;
  uint32_t key0, key1;      // Philox key
};

// Byte offsets of the per-walker arrays inside the caller's state buffer.
struct Layout {
  size_t phi_up;   // double [W][n_up][L]   orbitals at the current up positions
  size_t a_up;     // double [W][n_up][L]   rows phi(r_i^up)^T lambda
  size_t bt;       // double [W][n_up][L]   rows lambda phi(r_j^dn) (j < n_dn), then c^{(l)}
  size_t ginv;     // double [W][n_up][n_up] G~^{-1}
  size_t pprop;    // double [W][n_up][L]   orbitals at the proposals (scratch)
  size_t gprop;    // double [W][n_up][n_up] proposed rows / columns, or G~ at a refresh
  size_t rprop;    // double [W][n_up][8]   proposal (x, y, z), acceptance draw, one-body Jastrow change
  size_t mbuf;     // double [W][N][L]      kinetic contraction vectors
  size_t kin;      // double [W][N][4]      grad_i D/D (3) and lap_i D/D
  size_t scal;     // double [W][8]         log|det|, sign, J, accepted, drift
  size_t status;   // int    [W]
  size_t list;     // int    [W][n_up]      accepted moves of a half-sweep
  size_t count;    // int    [4]
  size_t total;
};

enum { S_LOGDET = 0, S_SIGN = 1, S_J = 2, S_NACC = 3, S_DRIFT = 4, S_STRIDE = 8 };

inline size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

inline Layout make_layout(size_t W, size_t nu, size_t N, size_t L) {
  Layout l;
  size_t o = 0;
  auto take = [&](size_t bytes) { size_t r = o; o = align256(o + bytes); return r; };
  l.phi_up = take(W * nu * L * 8);
  l.a_up = take(W * nu * L * 8);
  l.bt = take(W * nu * L * 8);
  l.ginv = take(W * nu * nu * 8);
  l.pprop = take(W * nu * L * 8);
  l.gprop = take(W * nu * nu * 8);
  l.rprop = take(W * nu * kPropStride * 8);
  l.mbuf = take(W * N * L * 8);
  l.kin = take(W * N * 4 * 8);
  l.scal = take(W * S_STRIDE * 8);
  l.status = take(W * 4);
  l.list = take(W * nu * 4);
  l.count = take(16);
  l.total = o;
  return l;
}

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon et al., SC'11): 10 rounds of the 4x32 S-box with the
// Weyl key schedule; written from the published definition.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void philox4x32_10(uint32_t c[4], uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r) {
      k0 += 0x9E3779B9u;
      k1 += 0xBB67AE85u;
    }
    const uint32_t hi0 = __umulhi(0xD2511F53u, c[0]), lo0 = 0xD2511F53u * c[0];
    const uint32_t hi1 = __umulhi(0xCD9E8D57u, c[2]), lo1 = 0xCD9E8D57u * c[2];
    const uint32_t n0 = hi1 ^ c[1] ^ k0, n2 = hi0 ^ c[3] ^ k1;
    c[0] = n0;
    c[1] = lo1;
    c[2] = n2;
    c[3] = lo0;
  }
}

// The move of `electron` in `sweep` of `walker`: proposal r' and acceptance draw.
__device__ __forceinline__ void move_draw(const DevSystem &s, uint32_t walker, uint32_t sweep,
                                          uint32_t electron, const double r[3], double rp[3],
                                          double *u) {
  uint32_t c[4] = {walker, sweep, electron, 1u};
  philox4x32_10(c, s.key0, s.key1);
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const double t = __dsub_rn(__dmul_rn(__dadd_rn((double)c[k], 0.5), 0x1p-31), 1.0);
    rp[k] = fma(s.delta, t, r[k]);
  }
  *u = (double)c[3] * 0x1p-32;
}

// ---------------------------------------------------------------------------
// Atomic orbitals of one shell at displacement d = r - R_a (Eqs. gaussian,
// slater): components P_c(d) * g(|d|) with P = 1; x, y, z; xy, yz, zx,
// x^2 - y^2, 3z^2 - r^2.  No normalisation (lambda absorbs it).
// ---------------------------------------------------------------------------
__device__ __forceinline__ int shell_l(int info) { return info & 3; }
__device__ __forceinline__ int shell_rad(int info) { return (info >> 2) & 1; }
__device__ __forceinline__ int shell_off(int info) { return info >> 8; }

template <typename T>
__device__ __forceinline__ T texp(T x);
template <>
__device__ __forceinline__ double texp<double>(double x) { return exp(x); }
template <>
__device__ __forceinline__ float texp<float>(float x) { return expf(x); }

// values only; returns the number of components written to v
template <typename T>
__device__ __forceinline__ int shell_values(int info, T zeta, T dx, T dy, T dz, T v[5]) {
  const int l = shell_l(info);
  const T r2 = dx * dx + dy * dy + dz * dz;
  const T g = shell_rad(info) ? texp<T>(-zeta * sqrt(r2)) : texp<T>(-zeta * r2);
  if (l == 0) {
    v[0] = g;
    return 1;
  }
  if (l == 1) {
    v[0] = dx * g;
    v[1] = dy * g;
    v[2] = dz * g;
    return 3;
  }
  v[0] = dx * dy * g;
  v[1] = dy * dz * g;
  v[2] = dz * dx * g;
  v[3] = (dx * dx - dy * dy) * g;
  v[4] = (T(3) * dz * dz - r2) * g;
  return 5;
}

// values, gradients and Laplacians: out[c] = {v, gx, gy, gz, lap}
__device__ __forceinline__ int shell_derivs(int info, double zeta, double dx, double dy, double dz,
                                            double out[5][5]) {
  const int l = shell_l(info);
  const double r2 = dx * dx + dy * dy + dz * dz;
  double g, gg[3], lapg;
  if (shell_rad(info)) {
    const double r = sqrt(r2);
    g = exp(-zeta * r);
    const double f = -zeta / r * g;
    gg[0] = f * dx;
    gg[1] = f * dy;
    gg[2] = f * dz;
    lapg = (zeta * zeta - 2.0 * zeta / r) * g;
  } else {
    g = exp(-zeta * r2);
    const double f = -2.0 * zeta * g;
    gg[0] = f * dx;
    gg[1] = f * dy;
    gg[2] = f * dz;
    lapg = (4.0 * zeta * zeta * r2 - 6.0 * zeta) * g;
  }
  const double d[3] = {dx, dy, dz};
  const int nc = 2 * l + 1;
#pragma unroll
  for (int c = 0; c < 5; ++c) {
    if (c >= nc) break;
    double P, gP[3] = {0.0, 0.0, 0.0};
    if (l == 0) {
      P = 1.0;
    } else if (l == 1) {
      P = d[c];
      gP[c] = 1.0;
    } else if (c == 0) {
      P = dx * dy; gP[0] = dy; gP[1] = dx;
    } else if (c == 1) {
      P = dy * dz; gP[1] = dz; gP[2] = dy;
    } else if (c == 2) {
      P = dz * dx; gP[0] = dz; gP[2] = dx;
    } else if (c == 3) {
      P = dx * dx - dy * dy; gP[0] = 2.0 * dx; gP[1] = -2.0 * dy;
    } else {
      P = 3.0 * dz * dz - r2; gP[0] = -2.0 * dx; gP[1] = -2.0 * dy; gP[2] = 4.0 * dz;
    }
    out[c][0] = P * g;
    out[c][1] = gP[0] * g + P * gg[0];
    out[c][2] = gP[1] * g + P * gg[1];
    out[c][3] = gP[2] * g + P * gg[2];
    out[c][4] = 2.0 * (gP[0] * gg[0] + gP[1] * gg[1] + gP[2] * gg[2]) + P * lapg;
  }
  return nc;
}

// ---------------------------------------------------------------------------
// Jastrow pieces (Eqs. onebody_J_hom, onebody_u, twobody_v).
// ---------------------------------------------------------------------------
// one-body term of one atom at distance r: f = -c^3 u(c r), c = (2Z)^{1/4}
__device__ __forceinline__ double j1_val(double c, double b, double r) {
  const double s = c * r;
  const double u = (b == 0.0) ? 0.5 * s : (1.0 - exp(-b * s)) / (2.0 * b);
  return -c * c * c * u;
}
// f' and f'' in r
__device__ __forceinline__ void j1_d(double c, double b, double r, double *fp, double *fpp) {
  const double c4 = c * c * c * c;
  if (b == 0.0) {
    *fp = -0.5 * c4;
    *fpp = 0.0;
  } else {
    const double e = exp(-b * c * r);
    *fp = -0.5 * c4 * e;
    *fpp = 0.5 * c4 * c * b * e;
  }
}
// pair term v(r) = r / (k (1 + b r)); parameters chosen by spins
__device__ __forceinline__ void j2_params(const DevSystem &s, bool same, double *k, double *b) {
  if (same && !s.j2_si) {
    *k = 4.0;
    *b = s.b_para;
  } else {
    *k = 2.0;
    *b = s.b_anti;
  }
}
__device__ __forceinline__ double j2_val(double k, double b, double r) { return r / (k * (1.0 + b * r)); }

// ---------------------------------------------------------------------------
// reductions
// ---------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

}  // namespace jagp
