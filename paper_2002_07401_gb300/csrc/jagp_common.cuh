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
  const int *shell_atom;    // [n_shells] owning atom, in the same (evaluation) order
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
// Orbital tables, G~ and its inverse are stored in the precision of the path
// (FP64, or FP32 in the mixed path, "T" below); positions, proposals,
// per-walker scalars and the kinetic partial sums are always FP64.
struct Layout {
  size_t phi_up;   // T      [W][n_up][L]    orbitals at the current up positions
  size_t a_up;     // T      [W][n_up][L]    rows phi(r_i^up)^T lambda
  size_t bt;       // T      [W][n_up][L]    rows lambda phi(r_j^dn) (j < n_dn), then c^{(l)}
  size_t ginv;     // T      [W][n_up][n_up] G~^{-1}
  size_t pprop;    // T      [W][n_up][L]    orbitals at the proposals (scratch)
  size_t gprop;    // T      [W][n_up][n_up] proposed rows / columns, or G~ at a refresh
  size_t rprop;    // double [W][n_up][8]    proposal (x, y, z), acceptance draw, one-body Jastrow change
  size_t mbuf;     // T      [W][N][L]       kinetic contraction vectors
  size_t kin;      // double [W][N][4]       grad_i D/D (3) and lap_i D/D
  size_t scal;     // double [W][8]          log|det|, sign, J, accepted, drift
  size_t status;   // int    [W]
  size_t list;     // int    [W][n_up]       accepted moves of a half-sweep
  size_t count;    // int    [4]
  size_t pack;     // BF16   [W n_up][4 kp]  mixed path: fixed-point slices of the lambda-product rows
  size_t rows;     // int    [W n_up]        mixed path: destination rows of the packed operand
  size_t exps;     // int    [W n_up]        mixed path: row exponents of the packed operand
  size_t g64;      // double [W][n_up][n_up] mixed path: G~ at a refresh (FP64 result of the compensated sum)
  size_t bt_lo;    // float  [W][n_up][L]    mixed path: low parts of Bt (Bt + bt_lo is a two-float table)
  size_t total;
};

enum { S_LOGDET = 0, S_SIGN = 1, S_J = 2, S_NACC = 3, S_DRIFT = 4, S_STRIDE = 8 };

inline size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

// esz: bytes per table element (8 or 4); kp: padded K of the packed operand (0 = none)
inline Layout make_layout(size_t W, size_t nu, size_t N, size_t L, size_t esz = 8, size_t kp = 0) {
  Layout l;
  size_t o = 0;
  auto take = [&](size_t bytes) { size_t r = o; o = align256(o + bytes); return r; };
  l.phi_up = take(W * nu * L * esz);
  l.a_up = take(W * nu * L * esz);
  l.bt = take(W * nu * L * esz);
  l.ginv = take(W * nu * nu * esz);
  l.pprop = take(W * nu * L * esz);
  l.gprop = take(W * nu * nu * esz);
  l.rprop = take(W * nu * kPropStride * 8);
  l.mbuf = take(W * N * L * esz);
  l.kin = take(W * N * 4 * 8);
  l.scal = take(W * S_STRIDE * 8);
  l.status = take(W * 4);
  l.list = take(W * nu * 4);
  l.count = take(16);
  l.pack = take(W * nu * 4 * kp * 2);
  l.rows = take(kp ? W * nu * 4 : 0);
  l.exps = take(kp ? W * nu * 4 : 0);
  l.g64 = take(esz == 4 ? W * nu * nu * 8 : 0);
  l.bt_lo = take(esz == 4 ? W * nu * L * 4 : 0);
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

// Radial factor g = e^{-zeta r^2} (Gaussian) or e^{-zeta r} (Slater) from the
// FP64 squared distance.  FP64: the library exp.  FP32 (mixed path): the
// exponent x is formed in FP64 and split x = x_hi + x_lo (x_hi its FP32
// rounding), and g = exp_f32(x_hi) (1 + x_lo): FP32 relative accuracy even for
// large |x|, where rounding the argument itself to FP32 would not be.
template <typename T>
__device__ __forceinline__ T radial_factor(int rad, double zeta, double r2);
template <>
__device__ __forceinline__ double radial_factor<double>(int rad, double zeta, double r2) {
  return rad ? exp(-zeta * sqrt(r2)) : exp(-zeta * r2);
}
template <>
__device__ __forceinline__ float radial_factor<float>(int rad, double zeta, double r2) {
  const double x = rad ? -zeta * sqrt(r2) : -zeta * r2;
  const float xh = static_cast<float>(x);
  const float xl = static_cast<float>(x - static_cast<double>(xh));
  return expf(xh) * (1.0f + xl);
}

// values only, at the FP64 displacement (dx, dy, dz) from the shell's atom;
// returns the number of components written to v.  FP32 values: the radial
// factor exp(x_hi)(1 + x_lo) and the angular polynomial are multiplied in FP64
// and rounded once, so each value carries the FP32 exponential's error and a
// single rounding.
template <typename T>
__device__ __forceinline__ int shell_values(int info, double zeta, double dx, double dy, double dz, T v[5]);

template <>
__device__ __forceinline__ int shell_values<double>(int info, double zeta, double dx, double dy, double dz,
                                                    double v[5]) {
  const int l = shell_l(info);
  const double r2 = dx * dx + dy * dy + dz * dz;
  const double g = radial_factor<double>(shell_rad(info), zeta, r2);
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
  v[4] = (3.0 * dz * dz - r2) * g;
  return 5;
}

template <>
__device__ __forceinline__ int shell_values<float>(int info, double zeta, double dx, double dy, double dz,
                                                   float v[5]) {
  const int l = shell_l(info);
  const double r2 = dx * dx + dy * dy + dz * dz;
  const double x = shell_rad(info) ? -zeta * sqrt(r2) : -zeta * r2;
  const float xh = static_cast<float>(x);
  const float xl = static_cast<float>(x - static_cast<double>(xh));
  const double g = static_cast<double>(expf(xh)) * (1.0 + static_cast<double>(xl));
  if (l == 0) {
    v[0] = static_cast<float>(g);
    return 1;
  }
  if (l == 1) {
    v[0] = static_cast<float>(dx * g);
    v[1] = static_cast<float>(dy * g);
    v[2] = static_cast<float>(dz * g);
    return 3;
  }
  v[0] = static_cast<float>(dx * dy * g);
  v[1] = static_cast<float>(dy * dz * g);
  v[2] = static_cast<float>(dz * dx * g);
  v[3] = static_cast<float>((dx * dx - dy * dy) * g);
  v[4] = static_cast<float>((3.0 * dz * dz - r2) * g);
  return 5;
}

// values, gradients and Laplacians: out[c] = {v, gx, gy, gz, lap}
template <typename T>
__device__ __forceinline__ int shell_derivs(int info, double zeta_d, double dxd, double dyd, double dzd,
                                            T out[5][5]) {
  const int l = shell_l(info);
  const double r2d = dxd * dxd + dyd * dyd + dzd * dzd;
  const T zeta = static_cast<T>(zeta_d), dx = static_cast<T>(dxd), dy = static_cast<T>(dyd), dz = static_cast<T>(dzd);
  const T r2 = static_cast<T>(r2d);
  const T g = radial_factor<T>(shell_rad(info), zeta_d, r2d);
  T gg[3], lapg;
  if (shell_rad(info)) {
    const T r = static_cast<T>(sqrt(r2d));
    const T f = -zeta / r * g;
    gg[0] = f * dx;
    gg[1] = f * dy;
    gg[2] = f * dz;
    lapg = (zeta * zeta - T(2) * zeta / r) * g;
  } else {
    const T f = T(-2) * zeta * g;
    gg[0] = f * dx;
    gg[1] = f * dy;
    gg[2] = f * dz;
    lapg = (T(4) * zeta * zeta * r2 - T(6) * zeta) * g;
  }
  const T d[3] = {dx, dy, dz};
  const int nc = 2 * l + 1;
#pragma unroll
  for (int c = 0; c < 5; ++c) {
    if (c >= nc) break;
    T P, gP[3] = {T(0), T(0), T(0)};
    if (l == 0) {
      P = T(1);
    } else if (l == 1) {
      P = d[c];
      gP[c] = T(1);
    } else if (c == 0) {
      P = dx * dy; gP[0] = dy; gP[1] = dx;
    } else if (c == 1) {
      P = dy * dz; gP[1] = dz; gP[2] = dy;
    } else if (c == 2) {
      P = dz * dx; gP[0] = dz; gP[2] = dx;
    } else if (c == 3) {
      P = dx * dx - dy * dy; gP[0] = T(2) * dx; gP[1] = T(-2) * dy;
    } else {
      P = T(3) * dz * dz - r2; gP[0] = T(-2) * dx; gP[1] = T(-2) * dy; gP[2] = T(4) * dz;
    }
    out[c][0] = P * g;
    out[c][1] = gP[0] * g + P * gg[0];
    out[c][2] = gP[1] * g + P * gg[1];
    out[c][3] = gP[2] * g + P * gg[2];
    out[c][4] = T(2) * (gP[0] * gg[0] + gP[1] * gg[1] + gP[2] * gg[2]) + P * lapg;
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
