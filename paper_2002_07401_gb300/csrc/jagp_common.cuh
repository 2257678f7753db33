// jagp_common.cuh -- device-side definitions shared by the libjagp kernels.
//
// Everything here is the GPU path's own code; the CPU oracle shares none of it.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/jagp.h"
#include "dword.cuh"

namespace jagp {

constexpr int kMaxUp = 1024;        // largest N_up accepted (G~^{-1} leaves shared memory above ~160)
constexpr int kMaxUpGrad = 64;     // above this N_up the adjoint's G~-sized steps run as per-walker GEMMs
constexpr int kWarp = 32;
constexpr int kPropStride = 8;     // doubles per proposal record
constexpr int kFixedSlices = 6;    // 8-bit slices per element of the fixed-point lambda products (mixed path)
constexpr int kFixedPairs = 21;    // slice pairs (a, b) with a + b < kFixedSlices
constexpr int kMaxPairs = 36;      // slice pairs of the FP64-equivalent products (eight slices)
constexpr int kTcRefreshMinUp = 32;  // mixed path: G~ of a refresh on the tensor cores from this N_up on
constexpr int kGuidedMaxUp = 64;     // guided sampling: G~ and G~^{-1} in shared memory up to this N_up
constexpr int kMmatDwMaxUp = 32;     // mixed path: exact M vectors on the CUDA cores up to this N_up (tensor cores above)

// Shell record packed for one 32-byte load: centre (x, y, z) and exponent.
// info = l | radial << 2 | first-function-offset << 8.
// Tell the compiler that these (non-null) pointers address global memory, so
// that it may use global loads and stores through them where it cannot infer
// that from where they came from (kernel arguments read from memory).
template <class... P>
__device__ __forceinline__ void assume_global(const P *...p) {
  (__builtin_assume(__isGlobal(p)), ...);
}

struct DevSystem {
  int n_atoms, n_shells, L, n_up, n_dn, N;
  const double *R;          // [n_atoms][3]
  const double *Z;          // [n_atoms]
  const double *c1;         // (2 Z_a)^{1/4}
  const double4 *shell_geo; // [n_shells]
  const float4 *shell_dw;   // [n_shells][2]: (x, y, z, zeta) rounded to FP32, then the remainders
  const int *shell_info;    // [n_shells]
  const int *shell_atom;    // [n_shells] owning atom, in the same (evaluation) order
  const double *lam;        // [L][L]
  const double *lamT;       // [L][L] = lambda^T
  const double *unpaired;   // [n_up - n_dn][L]
  double b_ea, b_para, b_anti;
  // FP32 copies for the mixed path's acceptance test (Jastrow changes only)
  const float4 *atom_f;     // [n_atoms]: (x, y, z, c1) rounded to FP32
  float b_ea_f, b_para_f, b_anti_f;
  int use_j1, use_j2, j2_si;
  double v_ii;              // ion-ion repulsion (a constant of the system)
  double delta;
  uint32_t key0, key1;      // Philox key
  // three/four-body Jastrow (FP64 path): its shells, LJ functions, couplings [LJ][LJ]
  int use_j3, n_jshells, LJ;
  const double4 *jshell_geo;
  const int *jshell_info;
  const double *j3p, *j3a;
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
  size_t pack;     // BF16   [W n_up][nsl kp] fixed-point slices of the lambda-product rows (tensor-core paths)
  size_t rows;     // int    [W n_up]        mixed path: destination rows of the packed operand
  size_t exps;     // int    [W n_up]        mixed path: row exponents of the packed operand
  size_t g64;      // double [W][n_up][n_up] G~ at a refresh (overwritten by the in-place inverse when large)
  size_t bt_lo;    // float  [W][n_up][L]    mixed path: low parts of Bt (Bt + bt_lo is a two-float table)
  size_t phi_lo;   // float  [W][n_up][L]    mixed path: low parts of phi_up
  size_t pprop_lo; // float  [W][n_up][L]    mixed path: low parts of pprop
  size_t gpack_a;  // BF16   [W n_up][5 kp]  mixed path, large N_up: slices of Phi_up + lo for G~ on the tensor cores
  size_t gpack_b;  // BF16   [W n_up][5 kp]  ... and of Bt + lo
  size_t gexp_a;   // int    [W n_up]        their row exponents
  size_t gexp_b;   // int    [W n_up]
  size_t grows;    // int    [W n_up]        scratch row map of the packing
  // mixed path, local energy: the M vectors as exact fixed-point tensor-core
  // products of the FP64 inverse with the two-float tables (kpn = N_up padded to 64)
  size_t ginv64;   // double [W][n_up][n_up] G~^{-1} of the last refresh in FP64
  size_t a_up_lo;  // float  [W][n_up][L]    low parts of A_up (A_up + a_up_lo is a two-float table)
  size_t mbuf_lo;  // float  [W][N][L]       low parts of the M vectors
  size_t mpack_a;  // BF16   [W n_up][5 kpn] slices of G~^{-1} columns (up) or rows (down)
  size_t mpack_b;  // BF16   [W L][5 kpn]    slices of Bt columns (up) or A_up columns (down)
  size_t mexp_a;   // int    [W n_up]        their exponents
  size_t mexp_b;   // int    [W L]
  size_t mrows;    // int    [W n_up]        destination rows of the M product
  size_t j3buf;    // double [W][6][LJ]      three-body Jastrow: U_up, U_dn (spin sums of chi), M_p U_up,
                   //                        M_p U_dn, M_a U_up, M_a U_dn
  size_t total;
};

enum { S_LOGDET = 0, S_SIGN = 1, S_J = 2, S_NACC = 3, S_DRIFT = 4, S_STRIDE = 8 };

inline size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

// esz: bytes per table element (8 or 4); kp: padded K of the packed operand (0 = none)
inline Layout make_layout(size_t W, size_t nu, size_t N, size_t L, size_t esz = 8, size_t kp = 0,
                          size_t nsl = kFixedSlices, bool tc_refresh = false, size_t lj = 0) {
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
  l.pack = take(W * nu * nsl * kp * 2);
  l.rows = take(kp ? W * nu * 4 : 0);
  l.exps = take(kp ? W * nu * 4 : 0);
  l.g64 = take(W * nu * nu * 8);
  l.bt_lo = take(esz == 4 ? W * nu * L * 4 : 0);
  l.phi_lo = take(esz == 4 ? W * nu * L * 4 : 0);
  l.pprop_lo = take(esz == 4 ? W * nu * L * 4 : 0);
  const size_t gp = tc_refresh ? W * nu * kFixedSlices * kp * 2 : 0, gi = tc_refresh ? W * nu * 4 : 0;
  l.gpack_a = take(gp);
  l.gpack_b = take(gp);
  l.gexp_a = take(gi);
  l.gexp_b = take(gi);
  l.grows = take(gi);
  const bool mx = esz == 4;
  const size_t kpn = (nu + 63) / 64 * 64;
  l.ginv64 = take(mx ? W * nu * nu * 8 : 0);
  l.a_up_lo = take(mx ? W * nu * L * 4 : 0);
  l.mbuf_lo = take(mx ? W * N * L * 4 : 0);
  l.mpack_a = take(mx ? W * nu * kFixedSlices * kpn * 2 : 0);
  l.mpack_b = take(mx ? W * L * kFixedSlices * kpn * 2 : 0);
  l.mexp_a = take(mx ? W * nu * 4 : 0);
  l.mexp_b = take(mx ? W * L * 4 : 0);
  l.mrows = take(mx ? W * nu * 4 : 0);
  l.j3buf = take(W * 6 * lj * 8);
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

// The move of `electron` in `sweep` of `walker`: coordinate k (0, 1, 2) of the
// proposal r' = r + delta (2 t - 1) from Philox output word k, and the
// acceptance draw u from word 3.  A warp's lanes each take one coordinate, so
// the FP64 arithmetic of a proposal is issued once rather than three times.
__device__ __forceinline__ void move_draw_coord(const DevSystem &s, uint32_t walker, uint32_t sweep,
                                                uint32_t electron, double rk, int k, double *rpk, double *u) {
  uint32_t c[4] = {walker, sweep, electron, 1u};
  philox4x32_10(c, s.key0, s.key1);
  const uint32_t ck = k == 0 ? c[0] : (k == 1 ? c[1] : c[2]);
  const double t = __dsub_rn(__dmul_rn(__dadd_rn((double)ck, 0.5), 0x1p-31), 1.0);
  *rpk = fma(s.delta, t, rk);
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
// FP64 squared distance (FP64 path).
__device__ __forceinline__ double radial_factor(int rad, double zeta, double r2) {
  return rad ? exp(-zeta * sqrt(r2)) : exp(-zeta * r2);
}

// FP64 path: values only, at the displacement (dx, dy, dz) from the shell's
// atom; returns the number of components written to v.
__device__ __forceinline__ int shell_values(int info, double zeta, double dx, double dy, double dz, double v[5]) {
  const int l = shell_l(info);
  const double r2 = dx * dx + dy * dy + dz * dz;
  const double g = radial_factor(shell_rad(info), zeta, r2);
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

// FP32 path: the displacement d = r - R_a of a point from the shell's atom in
// double-word, from the point's and the atom's double-word coordinates (the
// atom's split once on the host: geo_hi = (x, y, z, zeta) rounded to FP32,
// geo_lo = the remainders).
struct DwDisp {
  fdw x, y, z, r2;
};
__device__ __forceinline__ DwDisp dw_displacement(const fdw p[3], float4 geo_hi, float4 geo_lo) {
  DwDisp d;
  d.x = dw_add(p[0], fdw{-geo_hi.x, -geo_lo.x});
  d.y = dw_add(p[1], fdw{-geo_hi.y, -geo_lo.y});
  d.z = dw_add(p[2], fdw{-geo_hi.z, -geo_lo.z});
  d.r2 = dw_add(dw_add(dw_mul(d.x, d.x), dw_mul(d.y, d.y)), dw_mul(d.z, d.z));
  return d;
}

// the radial factor as a double-word (relative error a few units of 2^-46)
__device__ __forceinline__ fdw radial_dw(int rad, fdw zeta, fdw r2) {
  return dw_exp_neg(dw_neg(dw_mul(zeta, rad ? dw_sqrt(r2) : r2)));
}

// FP32 path: the shell's values as double-words; v[c] (hi) is the value
// rounded to FP32 (within half an ulp plus a few units of 2^-46), vlo[c] the rest.
__device__ __forceinline__ int shell_values_dw(int info, fdw zeta, const DwDisp &d, float v[5], float vlo[5]) {
  const int l = shell_l(info);
  const fdw g = radial_dw(shell_rad(info), zeta, d.r2);
  if (l == 0) {
    v[0] = g.hi;
    vlo[0] = g.lo;
    return 1;
  }
  fdw p[5];
  int nc;
  if (l == 1) {
    p[0] = d.x;
    p[1] = d.y;
    p[2] = d.z;
    nc = 3;
  } else {
    const fdw xx = dw_mul(d.x, d.x), yy = dw_mul(d.y, d.y), zz = dw_mul(d.z, d.z);
    p[0] = dw_mul(d.x, d.y);
    p[1] = dw_mul(d.y, d.z);
    p[2] = dw_mul(d.z, d.x);
    p[3] = dw_add(xx, dw_neg(yy));
    p[4] = dw_add(dw_mul_f(zz, 3.0f), dw_neg(d.r2));
    nc = 5;
  }
#pragma unroll
  for (int c = 0; c < 5; ++c) {
    if (c >= nc) break;
    const fdw t = dw_mul(p[c], g);
    v[c] = t.hi;
    vlo[c] = t.lo;
  }
  return nc;
}

// FP64 path: values, gradients and Laplacians: out[c] = {v, gx, gy, gz, lap}
__device__ __forceinline__ int shell_derivs(int info, double zeta, double dx, double dy, double dz,
                                            double out[5][5]) {
  const int l = shell_l(info);
  const double r2 = dx * dx + dy * dy + dz * dz;
  const double g = radial_factor(shell_rad(info), zeta, r2);
  double gg[3], lapg;
  if (shell_rad(info)) {
    const double r = sqrt(r2);
    const double f = -zeta / r * g;
    gg[0] = f * dx;
    gg[1] = f * dy;
    gg[2] = f * dz;
    lapg = (zeta * zeta - 2.0 * zeta / r) * g;
  } else {
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
// d/d b of an atom's J1 term F = -c^3 u(c r), u = (1 - e^{-b s}) / (2b) (the
// b -> 0 limit at b = 0)
__device__ __forceinline__ double j1_db(double c, double b, double r) {
  const double s = c * r;
  if (b == 0.0) return -c * c * c * (-s * s / 4.0);
  const double e = exp(-b * s);
  return -c * c * c * (s * e / (2.0 * b) - (1.0 - e) / (2.0 * b * b));
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

// Two-body Jastrow change when electron e (spin UP) moves from (ox, oy, oz) to
// (px, py, pz), summed over the other electrons k = k0, k0 + dk, ... < N at
// positions xs.  FP64 path in FP64; FP32 path with FP32 distances (the value
// only enters the acceptance test; J itself is recomputed in FP64).
template <typename T, bool UP>
__device__ __forceinline__ double j2_move_change(const DevSystem &s, const double *xs, int e, double px, double py,
                                                 double pz, double ox, double oy, double oz, int k0, int dk) {
  double pj = 0.0;
  for (int k = k0; k < s.N; k += dk) {
    if (k == e) continue;
    double kk, bb;
    j2_params(s, (k < s.n_up) == UP, &kk, &bb);
    const double qx = xs[3 * k], qy = xs[3 * k + 1], qz = xs[3 * k + 2];
    if constexpr (sizeof(T) == 8) {
      const double dn = sqrt((px - qx) * (px - qx) + (py - qy) * (py - qy) + (pz - qz) * (pz - qz));
      const double d0 = sqrt((ox - qx) * (ox - qx) + (oy - qy) * (oy - qy) + (oz - qz) * (oz - qz));
      pj += j2_val(kk, bb, dn) - j2_val(kk, bb, d0);
    } else {
      const float ax = static_cast<float>(px - qx), ay = static_cast<float>(py - qy), az = static_cast<float>(pz - qz);
      const float bx = static_cast<float>(ox - qx), by = static_cast<float>(oy - qy), bz = static_cast<float>(oz - qz);
      const float dn = sqrtf(ax * ax + ay * ay + az * az), d0 = sqrtf(bx * bx + by * by + bz * bz);
      const float ik = static_cast<float>(1.0 / kk), b = static_cast<float>(bb);
      pj += static_cast<double>(ik * (__fdividef(dn, 1.0f + b * dn) - __fdividef(d0, 1.0f + b * d0)));
    }
  }
  return pj;
}

// The mixed path's two-body change with FP32 instructions only: positions from
// an FP32 mirror xf of the walker's coordinates, proposal p and old position o
// rounded to FP32 (the value only enters the acceptance test).
template <bool UP>
__device__ __forceinline__ float j2_move_change_f(const DevSystem &s, const float *xf, int e, const float p[3],
                                                  const float o[3], int k0, int dk) {
  float pj = 0.0f;
  for (int k = k0; k < s.N; k += dk) {
    if (k == e) continue;
    const bool same = (k < s.n_up) == UP;
    const bool para = same && !s.j2_si;  // k = 4, b_para; else k = 2, b_anti
    const float ik = para ? 0.25f : 0.5f, b = para ? s.b_para_f : s.b_anti_f;
    const float qx = xf[3 * k], qy = xf[3 * k + 1], qz = xf[3 * k + 2];
    const float ax = p[0] - qx, ay = p[1] - qy, az = p[2] - qz;
    const float bx = o[0] - qx, by = o[1] - qy, bz = o[2] - qz;
    const float dn = sqrtf(ax * ax + ay * ay + az * az), d0 = sqrtf(bx * bx + by * by + bz * bz);
    pj += ik * (__fdividef(dn, 1.0f + b * dn) - __fdividef(d0, 1.0f + b * d0));
  }
  return pj;
}

// ---------------------------------------------------------------------------
// reductions
// ---------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// One-body Jastrow change when an electron moves from rr to rp, FP64
// distances, summed over a warp (every lane gets the sum).
__device__ __forceinline__ double j1_move_change(const DevSystem &s, const double *rp, const double *rr, int lane) {
  double dj1 = 0.0;
  // lane pairs: even lanes take the new position, odd lanes the old one
  for (int q = lane; q < 2 * s.n_atoms; q += 32) {
    const int a = q >> 1;
    const double *pos = (q & 1) ? rr : rp;
    const double ax = pos[0] - s.R[3 * a], ay = pos[1] - s.R[3 * a + 1], az = pos[2] - s.R[3 * a + 2];
    const double v = j1_val(s.c1[a], s.b_ea, sqrt(ax * ax + ay * ay + az * az));
    dj1 += (q & 1) ? -v : v;
  }
  return warp_sum(dj1);
}

}  // namespace jagp
