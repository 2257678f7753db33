// jagp_api.cu -- the C ABI of libjagp (declared in include/jagp.h): argument
// checking, device copies of the system, and the launch sequence of each
// entry point.  All per-walker memory is the caller's state buffer.
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <cmath>
#include <mutex>
#include <type_traits>
#include <vector>

#include "jagp_group.cuh"
#include "jagp_launch.h"

using namespace jagp;

#include "jagp_ctx.h"

#include <stdarg.h>
#include <stdio.h>

namespace jagp {
static thread_local GroupRecorder *g_group_recorder = nullptr;
GroupRecorder *group_recorder() { return g_group_recorder; }
void set_group_recorder(GroupRecorder *r) { g_group_recorder = r; }
cudaError_t group_raise_smem(const void *fn, std::atomic<unsigned char> *done) {
  int dev = 0, optin = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev >= 0 && dev < 64 && done[dev].load(std::memory_order_acquire)) return cudaSuccess;
  if ((e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev)) != cudaSuccess) return e;
  cudaFuncAttributes fa;
  if ((e = cudaFuncGetAttributes(&fa, fn)) != cudaSuccess) return e;
  e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, optin - (int)fa.sharedSizeBytes);
  if (e == cudaSuccess && dev >= 0 && dev < 64) done[dev].store(1, std::memory_order_release);
  return e;
}
}  // namespace jagp

namespace {

std::once_flag g_attr_once;
cudaError_t g_attr_err = cudaSuccess;

thread_local const char *g_last_cuda_error = "no error";
thread_local char g_detail[256] = "";

#define JAGP_CU(call)                                  \
  do {                                                 \
    cudaError_t e_ = (call);                           \
    if (e_ != cudaSuccess) {                           \
      g_last_cuda_error = cudaGetErrorString(e_);      \
      return JAGP_ERR_CUDA;                            \
    }                                                  \
  } while (0)

// Launch bookkeeping: count the kernels a launcher issues and, when profiling
// is on for that kernel class, bracket it with an event pair on its stream.
struct LaunchScope {
  jagp_ctx *h;
  cudaStream_t st;
  bool timed;
  cudaEvent_t a = nullptr, b = nullptr;
  LaunchScope(jagp_ctx *h_, int kernel, cudaStream_t st_, int nkernels = 1)
      : h(h_), st(st_), timed(kernel != 0 && h_->prof_kernel == kernel) {
    h->launches += nkernels;
    if (timed && cudaEventCreate(&a) == cudaSuccess && cudaEventCreate(&b) == cudaSuccess)
      cudaEventRecord(a, st);
    else
      timed = false;
  }
  ~LaunchScope() {
    if (timed) {
      cudaEventRecord(b, st);
      h->prof_events.emplace_back(a, b);
    }
  }
};

#define LAUNCH(kernel_id, nk, call)             \
  do {                                          \
    LaunchScope ls_(h, (kernel_id), st, (nk));  \
    JAGP_CU(call);                              \
  } while (0)

bool tc_refresh(const jagp_ctx *h) { return h->precision == JAGP_PREC_MIXED && h->ds.n_up >= kTcRefreshMinUp; }

Layout layout_of(const jagp_ctx *h, int W) {
  const bool mixed = h->precision == JAGP_PREC_MIXED;
  return make_layout((size_t)W, (size_t)h->ds.n_up, (size_t)h->ds.N, (size_t)h->ds.L, mixed ? 4 : 8,
                     h->tc_lambda ? (size_t)h->kp : 0, (size_t)h->tc_slices, tc_refresh(h),
                     h->ds.use_j3 ? (size_t)h->ds.LJ : 0);
}

// the twenty-one slice pairs (a, b) with a + b <= 5 of the six-slice
// fixed-point operands (each row kept to 2^-47 of its largest magnitude, about
// the precision of its two-float values).  Both lambda products take all of
// them: the rows lambda phi (Bt) enter G~ and the up electrons' M vectors, the
// rows phi^T lambda (A_up) the down electrons' M vectors, all as two-float
// numbers; the kinetic term amplifies their relative error by about cond(G~).
const int kPairA[kFixedPairs] = {0, 0, 1, 0, 1, 2, 0, 1, 2, 3, 0, 1, 2, 3, 4, 0, 1, 2, 3, 4, 5};
const int kPairB[kFixedPairs] = {0, 1, 0, 2, 1, 0, 3, 2, 1, 0, 4, 3, 2, 1, 0, 5, 4, 3, 2, 1, 0};

// all slice pairs (a, b) with a + b < nsl, ordered by a + b, then a
int slice_pairs(int nsl, int *pa, int *pb) {
  int np = 0;
  for (int d = 0; d < nsl; ++d)
    for (int a = 0; a <= d; ++a) {
      pa[np] = a;
      pb[np] = d - a;
      ++np;
    }
  return np;
}

template <typename T>
T *at(void *base, size_t off) {
  return reinterpret_cast<T *>(static_cast<char *>(base) + off);
}

// host: one row of FP64 values -> kFixedSlices exact 8-bit fixed-point slices
// (BF16 bits) relative to 2^e, e = 1 + the binary exponent of the row's largest
// magnitude: v = 2^(e - 7) (t0 + t1 / 256 + t2 / 256^2 + ...), |t| <= 128.
uint16_t bf16_of_small_int(double q) {
  const float f = static_cast<float>(q);  // |q| <= 128: exact in BF16
  uint32_t u;
  memcpy(&u, &f, 4);
  return static_cast<uint16_t>(u >> 16);
}
int slice_row_fixed(const double *v, size_t vstride, int L, uint16_t *dst, size_t kp, int nsl, int bits) {
  double mx = 0.0;
  for (int k = 0; k < L; ++k) mx = std::max(mx, std::fabs(v[k * vstride]));
  int e = 0;
  if (mx > 0.0) std::frexp(mx, &e);  // mx = f 2^e, f in [0.5, 1)
  for (int k = 0; k < L; ++k) {
    double x = std::ldexp(v[k * vstride], bits - 1 - e);
    for (int t = 0; t < nsl; ++t) {
      const double q = std::nearbyint(x);
      dst[t * kp + k] = bf16_of_small_int(q);
      x = (x - q) * std::ldexp(1.0, bits);
    }
  }
  return e;
}

jagp_status_t check_walkers(const jagp_ctx *h, int W, const void *state) {
  if (!h) return JAGP_ERR_INVALID_ARG;
  if (W <= 0 || W > h->max_walkers) {
    jagp_set_detail("W = %d outside 1..%d (max_walkers)", W, h->max_walkers);
    return JAGP_ERR_INVALID_ARG;
  }
  if (!state || (reinterpret_cast<uintptr_t>(state) & 255u)) {
    jagp_set_detail("walker state is null or not 256-byte aligned");
    return JAGP_ERR_INVALID_ARG;
  }
  return JAGP_OK;
}

// lambda products of orbital rows: out[row] = P[row]^T lambda (left) or lambda P[row] (!left)
// for the listed rows (list/count) or the (nsub, stride) rows r < nrows.
jagp_status_t lambda_products(jagp_ctx *h, const double *P, const float *, double *out, bool left, const int *list,
                              const int *count, int nrows, int nsub, int stride, int max_rows, void *state, int W,
                              cudaStream_t st) {
  if (h->tc_lambda) {
    // FP64-equivalent products on the tensor cores: FP64 rows cut into exact
    // slices, every pair of weight >= 2^-(slices x bits) summed exactly, FP64 epilogue
    const Layout L = layout_of(h, W);
    uint16_t *pack = at<uint16_t>(state, L.pack);
    int *rows = at<int>(state, L.rows), *exps = at<int>(state, L.exps);
    int pa[kMaxPairs], pb[kMaxPairs];
    const int np = slice_pairs(h->tc_slices, pa, pb);
    LAUNCH(0, 1,
           launch_pack_fixed64(P, list, count, nrows, nsub, stride, h->ds.L, h->kp, h->tc_slices, h->tc_bits, pack,
                               rows, exps, max_rows, st));
    LAUNCH(JAGP_KERNEL_LAMBDA_ROWS, 1,
           launch_umma_gemm(pack, max_rows, count, h->tc_slices, left ? h->split_lamT : h->split_lam, h->ds.L,
                            h->tc_slices, h->kp, np, pa, pb, nullptr, h->ds.L, rows, h->d_err, st, exps,
                            left ? h->exp_lamT : h->exp_lam, nullptr, left ? h->tune_bn_left : h->tune_bn_right, out,
                            h->tc_bits, 0, 0, left ? h->tune_st_left : h->tune_st_right));
    return JAGP_OK;
  }
  LAUNCH(JAGP_KERNEL_LAMBDA_ROWS, 1,
         launch_lambda_rows(P, left ? h->ds.lam : h->ds.lamT, out, list, count, nrows, nsub, stride, h->ds.L, max_rows,
                            st));
  return JAGP_OK;
}
jagp_status_t lambda_products(jagp_ctx *h, const float *P, const float *P_lo, float *out, bool left, const int *list,
                              const int *count, int nrows, int nsub, int stride, int max_rows, void *state, int W,
                              cudaStream_t st) {
  // mixed path: cut the two-float rows P + P_lo into fixed-point slices, then
  // the exact tensor-core contraction against the sliced lambda
  const Layout L = layout_of(h, W);
  uint16_t *pack = at<uint16_t>(state, L.pack);
  int *rows = at<int>(state, L.rows), *exps = at<int>(state, L.exps);
  LAUNCH(0, 1,
         launch_pack_fixed(P, P_lo, list, count, nrows, nsub, stride, h->ds.L, h->kp, pack, rows, exps, max_rows,
                            st));
  // the rows keep their low parts (two-float Bt and A_up tables)
  float *out_lo = at<float>(state, left ? L.a_up_lo : L.bt_lo);
  LAUNCH(JAGP_KERNEL_LAMBDA_ROWS, 1,
         launch_umma_gemm(pack, max_rows, count, kFixedSlices, left ? h->split_lamT : h->split_lam, h->ds.L,
                          kFixedSlices, h->kp, kFixedPairs, kPairA, kPairB, out, h->ds.L,
                          rows, h->d_err, st, exps, left ? h->exp_lamT : h->exp_lam, out_lo,
                          left ? h->tune_bn_left : h->tune_bn_right, nullptr, 8, 0, 0,
                          left ? h->tune_st_left : h->tune_st_right));
  return JAGP_OK;
}

// G~ = Phi_up Bt^T at a refresh: plain FP64 products, or the compensated FP32 sum
cudaError_t refresh_geminal(const double *phi, const float *, size_t pw, const double *bt, const float *, size_t bw,
                            int n, int Lb, double *g, int W, cudaStream_t st, int tile) {
  return launch_gemm_rows<double>(phi, pw, bt, bw, n, n, Lb, g, (size_t)n * n, n, W, st, tile);
}
cudaError_t refresh_geminal(const float *phi, const float *phi_lo, size_t pw, const float *bt, const float *bt_lo,
                            size_t bw, int n, int Lb, double *g, int W, cudaStream_t st, int tile) {
  return launch_gemm_rows_dot2(phi, phi_lo, pw, bt, bt_lo, bw, n, n, Lb, g, (size_t)n * n, n, W, st, tile);
}
// low parts of the two-float tables of the mixed path (none in the FP64 path)
float *lo_table(const jagp_ctx *h, void *state, size_t off) {
  return h->precision == JAGP_PREC_MIXED ? at<float>(state, off) : nullptr;
}
// where the refresh keeps G~ (its own array: the proposed rows in gprop stay
// valid across refreshes within a half-sweep)
double *refresh_g(const Layout &L, void *state) { return at<double>(state, L.g64); }
// the three-body Jastrow's per-walker vectors (null without it)
double *j3_vectors(const jagp_ctx *h, const Layout &L, void *state) {
  return h->ds.use_j3 ? at<double>(state, L.j3buf) : nullptr;
}

// the local-energy sequence on a current state
// Mixed path: the M vectors of the kinetic energy as exact fixed-point
// tensor-core products of the FP64 inverse of the last refresh with the
// two-float tables (six 8-bit slices per element, twenty-one slice pairs, a
// two-float result M + M_lo; every accumulator sum exact for N_up <= 256 but
// the last, whose rounding lies below 2^-55 of the leading term):
//   up:   M[i][mu]        = sum_j Bt[j][mu] Ginv[j][i]    (columns of Bt against columns of G~^{-1})
//   down: M[n_up + j][mu] = sum_i A_up[i][mu] Ginv[j][i]  (columns of A_up against rows of G~^{-1})
// as transposed products (the L basis functions of a walker are the rows of a
// tile, its electrons the columns), written back transposed; for N_up up to
// kMmatDwMaxUp the same sums as compensated dot products on the CUDA cores.
// Then the per-shell contraction in double-word arithmetic.
jagp_status_t run_kinetic_mixed(jagp_ctx *h, const double *r, void *state, int W, cudaStream_t st) {
  const Layout L = layout_of(h, W);
  const DevSystem &d = h->ds;
  const int n = d.n_up, nd = d.n_dn, Lb = d.L, kpn = (n + 63) / 64 * 64;
  const long long NL = (long long)d.N * Lb;
  const double *gi64 = at<double>(state, L.ginv64);
  uint16_t *pa = at<uint16_t>(state, L.mpack_a), *pb = at<uint16_t>(state, L.mpack_b);
  int *ea = at<int>(state, L.mexp_a), *eb = at<int>(state, L.mexp_b), *mr = at<int>(state, L.mrows);
  float *mb = at<float>(state, L.mbuf), *ml = at<float>(state, L.mbuf_lo);
  if (n <= kMmatDwMaxUp) {
    // small N_up: compensated sums on the CUDA cores (a tensor-core tile would be mostly padding)
    LAUNCH(JAGP_KERNEL_ENERGY, 1,
           launch_mmat_dw(d, gi64, at<float>(state, L.bt), at<float>(state, L.bt_lo), at<float>(state, L.a_up),
                          at<float>(state, L.a_up_lo), mb, ml, W, st));
    LAUNCH(JAGP_KERNEL_ENERGY, 1, launch_kinetic_m2(d, r, mb, ml, at<double>(state, L.kin), W, st));
    return JAGP_OK;
  }
  // up electrons: A = columns of Bt (L rows per walker), B = columns of G~^{-1} (N_up rows)
  LAUNCH(0, 1, launch_pack_cols(gi64, nullptr, nullptr, (size_t)n * n, n, n, kpn, W, pa, ea, nullptr, 0, 0, st));
  LAUNCH(0, 1,
         launch_pack_cols(nullptr, at<float>(state, L.bt), at<float>(state, L.bt_lo), (size_t)n * Lb, n, Lb, kpn, W,
                          pb, eb, nullptr, 0, 0, st));
  LAUNCH(JAGP_KERNEL_ENERGY, 1,
         launch_umma_gemm(pb, W * Lb, nullptr, kFixedSlices, pa, n, kFixedSlices, kpn, kFixedPairs, kPairA, kPairB, mb,
                          0, nullptr, h->d_err, st, eb, ea, ml, 0, nullptr, 8, Lb, W, 0, n, NL, 1, Lb));
  if (nd > 0) {
    // down electrons: A = columns of A_up, B = rows j < N_dn of G~^{-1}
    LAUNCH(0, 1,
           launch_pack_fixed64(gi64, nullptr, nullptr, W * nd, nd, n, n, kpn, kFixedSlices, 8, pa, mr, ea, W * nd, st));
    LAUNCH(0, 1,
           launch_pack_cols(nullptr, at<float>(state, L.a_up), at<float>(state, L.a_up_lo), (size_t)n * Lb, n, Lb,
                            kpn, W, pb, eb, nullptr, 0, 0, st));
    LAUNCH(JAGP_KERNEL_ENERGY, 1,
           launch_umma_gemm(pb, W * Lb, nullptr, kFixedSlices, pa, nd, kFixedSlices, kpn, kFixedPairs, kPairA, kPairB,
                            mb + (size_t)n * Lb, 0, nullptr, h->d_err, st, eb, ea, ml + (size_t)n * Lb, 0, nullptr, 8,
                            Lb, W, 0, nd, NL, 1, Lb));
  }
  LAUNCH(JAGP_KERNEL_ENERGY, 1, launch_kinetic_m2(d, r, mb, ml, at<double>(state, L.kin), W, st));
  return JAGP_OK;
}

template <typename T>
jagp_status_t run_local_energy(jagp_ctx *h, const double *r, void *state, int W, double *eL, double *parts,
                               cudaStream_t st, bool write_jastrow = false) {
  const Layout L = layout_of(h, W);
  if (std::is_same<T, float>::value) {
    if (h->ds.use_j3) LAUNCH(0, 1, launch_j3_prep(h->ds, r, j3_vectors(h, L, state), W, st));
    const jagp_status_t s = run_kinetic_mixed(h, r, state, W, st);
    if (s != JAGP_OK) return s;
  } else {
    if (h->ds.use_j3) LAUNCH(0, 1, launch_j3_prep(h->ds, r, j3_vectors(h, L, state), W, st));
    LAUNCH(JAGP_KERNEL_ENERGY, 1,
           launch_mmat<T>(h->ds, at<T>(state, L.ginv), at<T>(state, L.bt), at<T>(state, L.a_up), at<T>(state, L.mbuf),
                          W, st));
    LAUNCH(JAGP_KERNEL_ENERGY, 1,
           launch_kinetic<T>(h->ds, r, at<T>(state, L.mbuf), at<double>(state, L.kin), W, st));
  }
  double *sc = write_jastrow ? at<double>(state, L.scal) : nullptr;
  if (std::is_same<T, float>::value)
    LAUNCH(JAGP_KERNEL_ENERGY, 1,
           launch_elocal_dw(h->ds, r, at<double>(state, L.kin), eL, parts, W, st, sc, j3_vectors(h, L, state)));
  else
    LAUNCH(JAGP_KERNEL_ENERGY, 1,
           launch_elocal(h->ds, r, at<double>(state, L.kin), eL, parts, W, st, sc, j3_vectors(h, L, state)));
  return JAGP_OK;
}

// G~ = Phi_up Bt^T, its inverse (FP64 elimination), log|det| and (optionally) J
template <typename T>
jagp_status_t run_refresh(jagp_ctx *h, const double *r, void *state, int W, int check_drift, bool jastrow,
                          cudaStream_t st) {
  const Layout L = layout_of(h, W);
  const int n = h->ds.n_up, Lb = h->ds.L;
  double *gm = refresh_g(L, state);
  group_subkey(0);  // grouped sweeps: packing, then the G~ product, then the elimination
  if (tc_refresh(h)) {
    // G~ = (Phi_up + lo)(Bt + lo)^T per walker on the tensor cores: both tables
    // cut into six fixed-point slices, twenty-one pairs, FP64 epilogue
    int *rows = at<int>(state, L.grows);
    uint16_t *pa = at<uint16_t>(state, L.gpack_a), *pb = at<uint16_t>(state, L.gpack_b);
    int *ea = at<int>(state, L.gexp_a), *eb = at<int>(state, L.gexp_b);
    LAUNCH(0, 1,
           launch_pack_fixed(at<float>(state, L.phi_up), lo_table(h, state, L.phi_lo), nullptr, nullptr, W * n, 1, 1,
                             Lb, h->kp, pa, rows, ea, W * n, st));
    LAUNCH(0, 1,
           launch_pack_fixed(at<float>(state, L.bt), lo_table(h, state, L.bt_lo), nullptr, nullptr, W * n, 1, 1, Lb,
                             h->kp, pb, rows, eb, W * n, st));
    group_subkey(1);
    LAUNCH(JAGP_KERNEL_GEMM_ROWS, 1,
           launch_umma_gemm(pa, W * n, nullptr, kFixedSlices, pb, n, kFixedSlices, h->kp, kFixedPairs, kPairA, kPairB,
                            nullptr, n, nullptr, h->d_err, st, ea, eb, nullptr, 0, gm, 8, n, W));
  } else {
    group_subkey(1);
    LAUNCH(JAGP_KERNEL_GEMM_ROWS, 1,
           refresh_geminal(at<T>(state, L.phi_up), lo_table(h, state, L.phi_lo), (size_t)n * Lb, at<T>(state, L.bt),
                           lo_table(h, state, L.bt_lo), (size_t)n * Lb, n, Lb, gm, W, st, h->tune_tile_refresh));
  }
  // the mixed path keeps an FP64 copy of the inverse for the local energy
  double *gi64 = h->precision == JAGP_PREC_MIXED ? at<double>(state, L.ginv64) : nullptr;
  group_subkey(2);
  LAUNCH(0, 1,
         launch_refresh_inverse<T>(gm, at<T>(state, L.ginv), at<double>(state, L.scal), at<int>(state, L.status), n,
                                   W, check_drift, h->drift_tol, st, gi64));
  if (jastrow) {
    if (h->ds.use_j3) LAUNCH(0, 1, launch_j3_prep(h->ds, r, j3_vectors(h, L, state), W, st));
    LAUNCH(0, 1, launch_jastrow_full(h->ds, r, at<double>(state, L.scal), W, st, j3_vectors(h, L, state)));
  }
  return JAGP_OK;
}

template <typename T>
jagp_status_t run_eval(jagp_ctx *h, const double *d_r, int W, void *d_state, double *d_logabs, double *d_sign,
                       cudaStream_t st) {
  const Layout L = layout_of(h, W);
  const DevSystem &d = h->ds;
  const int n = d.n_up;
  T *phi_up = at<T>(d_state, L.phi_up), *pprop = at<T>(d_state, L.pprop);
  float *phi_lo = lo_table(h, d_state, L.phi_lo), *pprop_lo = lo_table(h, d_state, L.pprop_lo);
  LAUNCH(0, 1, launch_walker_init(at<double>(d_state, L.scal), at<int>(d_state, L.status), W, st, d_r, d.N));
  LAUNCH(JAGP_KERNEL_BASIS, 1, launch_basis_points<T>(d, false, d_r, W, 0, n, phi_up, phi_lo, nullptr, 0, 0, st));
  LAUNCH(JAGP_KERNEL_BASIS, d.n_dn > 0,
         launch_basis_points<T>(d, false, d_r, W, n, d.n_dn, pprop, pprop_lo, nullptr, 0, 0, st));
  // A_up = Phi_up lambda (every row); Bt rows j < n_dn = lambda phi(r_j^dn)
  jagp_status_t s = lambda_products(h, phi_up, phi_lo, at<T>(d_state, L.a_up), true, nullptr, nullptr, W * n, n, n,
                                    W * n, d_state, W, st);
  if (s != JAGP_OK) return s;
  if (d.n_dn > 0) {
    s = lambda_products(h, pprop, pprop_lo, at<T>(d_state, L.bt), false, nullptr, nullptr, W * d.n_dn, d.n_dn, n,
                        W * d.n_dn, d_state, W, st);
    if (s != JAGP_OK) return s;
  }
  LAUNCH(0, d.n_up > d.n_dn, launch_fill_unpaired<T>(d, at<T>(d_state, L.bt), W, st));
  if (h->precision == JAGP_PREC_MIXED)
    LAUNCH(0, d.n_up > d.n_dn, launch_fill_unpaired_lo(d, at<float>(d_state, L.bt_lo), W, st));
  s = run_refresh<T>(h, d_r, d_state, W, 0, true, st);
  if (s != JAGP_OK) return s;
  LAUNCH(0, (d_logabs || d_sign), launch_logpsi_out(at<double>(d_state, L.scal), W, d_logabs, d_sign, st));
  return JAGP_OK;
}

template <typename T>
jagp_status_t run_sweeps(jagp_ctx *h, double *d_r, void *d_state, int W, int nsweeps, uint64_t walker0,
                         uint64_t sweep0, double *d_eL, double *d_acc, cudaStream_t st,
                         const uint32_t *sweep_dev = nullptr, int accumulate = 0) {
  const Layout L = layout_of(h, W);
  const DevSystem &d = h->ds;
  const int n = d.n_up, Lb = d.L;
  // the mixed path refreshes G~^{-1} in FP64 after every half-sweep (every N_up
  // moves), the FP64 path once per sweep
  const bool half_refresh = h->precision == JAGP_PREC_MIXED;
  T *phi_up = at<T>(d_state, L.phi_up), *a_up = at<T>(d_state, L.a_up);
  T *bt = at<T>(d_state, L.bt), *ginv = at<T>(d_state, L.ginv);
  T *pprop = at<T>(d_state, L.pprop), *gprop = at<T>(d_state, L.gprop);
  double *rprop = at<double>(d_state, L.rprop), *scal = at<double>(d_state, L.scal);
  int *status = at<int>(d_state, L.status), *list = at<int>(d_state, L.list), *count = at<int>(d_state, L.count);
  float *phi_lo = lo_table(h, d_state, L.phi_lo), *pprop_lo = lo_table(h, d_state, L.pprop_lo);
  jagp_status_t s;
  // one spin half-sweep: all proposals and their rows (up) or columns (down) of
  // G~ at once, then the acceptance in chunks of refresh_moves moves, each
  // followed by the lambda products of its accepted rows and, but for the
  // last chunk, a refresh of G~^{-1} from the tables
  auto half_sweep = [&](bool up, uint32_t sw, int t) -> jagp_status_t {
    const int moves = up ? n : d.n_dn;
    if (moves == 0) return JAGP_OK;
    const int hk = up ? 1 : 3;  // grouped sweeps: (sweep, part, chunk, phase) of the launches below
    group_key(t, hk, 0, 0);
    int *total = count + (up ? 0 : 1), *chunk = count + 2;
    LAUNCH(JAGP_KERNEL_BASIS, 1,
           launch_basis_points<T>(d, true, d_r, W, up ? 0 : n, moves, pprop, pprop_lo, rprop, (uint32_t)walker0, sw,
                                  st, sweep_dev));
    if (up)
      LAUNCH(JAGP_KERNEL_GEMM_ROWS, 1,
             launch_gemm_rows<T>(pprop, (size_t)n * Lb, bt, (size_t)n * Lb, n, n, Lb, gprop, (size_t)n * n, n, W, st,
                                 h->tune_tile_prop));
    else
      LAUNCH(JAGP_KERNEL_GEMM_ROWS, 1,
             launch_gemm_rows<T>(pprop, (size_t)n * Lb, a_up, (size_t)n * Lb, d.n_dn, n, Lb, gprop, (size_t)n * n, n,
                                 W, st, h->tune_tile_prop));
    const int step = h->refresh_moves > 0 ? h->refresh_moves : moves;
    for (int m0 = 0; m0 < moves; m0 += step) {
      const int m1 = m0 + step < moves ? m0 + step : moves;
      group_key(t, hk, m0 / step, 1);
      JAGP_CU(zero_ints(chunk, 1, st));
      bool guided = false;
      if constexpr (std::is_same<T, double>::value) {
        if (h->guide_eps > 0.0) {
          guided = true;
          LAUNCH(JAGP_KERNEL_METROPOLIS, 1,
                 launch_metropolis_guided(d, up, d_r, rprop, gprop, ginv, scal, status, pprop, phi_up, list, chunk,
                                          refresh_g(L, d_state), h->guide_theta, h->guide_eps, W, st, m0, m1,
                                          total));
        }
      }
      if (!guided)
        LAUNCH(JAGP_KERNEL_METROPOLIS, 1,
               launch_metropolis<T>(d, up, d_r, rprop, gprop, ginv, scal, status, pprop, phi_up, list, chunk, W, st,
                                    pprop_lo, phi_lo, m0, m1, total, j3_vectors(h, L, d_state)));
      jagp_status_t q =
          lambda_products(h, pprop, pprop_lo, up ? a_up : bt, up, list, chunk, 0, 1, 0, W * n, d_state, W, st);
      if (q != JAGP_OK) return q;
      if (m1 < moves) {
        group_key(t, hk, m0 / step, 2);
        q = run_refresh<T>(h, d_r, d_state, W, 1, false, st);
        if (q != JAGP_OK) return q;
      }
    }
    return JAGP_OK;
  };
  // the three-body Jastrow's vectors from the positions (the acceptance kernels keep them current)
  group_key(-1, 0, 0, 0);
  if (d.use_j3 && nsweeps > 0) LAUNCH(0, 1, launch_j3_prep(d, d_r, j3_vectors(h, L, d_state), W, st));
  for (int t = 0; t < nsweeps; ++t) {
    const uint32_t sw = (uint32_t)(sweep0 + (uint64_t)t);
    group_key(t, 0, 0, 0);
    JAGP_CU(zero_ints(count, 2, st));
    // up electrons: rows of G~ against the frozen down-spin table Bt
    s = half_sweep(true, sw, t);
    if (s != JAGP_OK) return s;
    if (half_refresh && d.n_dn > 0) {
      group_key(t, 2, 0, 0);
      s = run_refresh<T>(h, d_r, d_state, W, 1, false, st);
      if (s != JAGP_OK) return s;
    }
    // down electrons: columns of G~ against the updated up-spin table A_up
    s = half_sweep(false, sw, t);
    if (s != JAGP_OK) return s;
    double *eL = d_eL ? d_eL + (accumulate ? 0 : (size_t)t * W) : nullptr;
    // the local-energy pass also forms J, so the refresh skips its Jastrow pass then
    group_key(t, 4, 0, 0);
    s = run_refresh<T>(h, d_r, d_state, W, 1, eL == nullptr, st);
    if (s != JAGP_OK) return s;
    if (eL) {
      group_key(t, 4, 0, 1);
      s = run_local_energy<T>(h, d_r, d_state, W, eL, nullptr, st, true);
      if (s != JAGP_OK) return s;
    }
    group_key(t, 4, 0, 2);
    if (d_acc)
      LAUNCH(0, 1, launch_reduce_acc(eL, scal, count, W, d_acc + (accumulate ? 0 : (size_t)t * 4), st, accumulate));
  }
  return JAGP_OK;
}

// workspace of jagp_grad (byte offsets)
struct GradLayout {
  size_t jg, kbar, dnphi, h1, h2, gbar, btbar, abar, phibar_a, phibar_b, phibar_dn, part, rbar, rbar_at, jpar, eL,
      lam_part, total;
  int nparts, nz;
  // lambda-bar on the tensor cores (FP64-equivalent handles, N_dn = N_up):
  // segments of seg_w walkers (seg_w N_up <= 2048 rows of K each), the packed
  // columns of both operands, their exponents and the per-segment products
  int tc_lam, seg_w, nseg, kpseg;
  size_t tc_u, tc_v, tc_eu, tc_ev, tc_part;
};
constexpr int kLamBarSlices = 8, kLamBarBits = 7;  // 7-bit slices: K <= 2048 sums stay below 2^24
GradLayout grad_layout(const jagp_ctx *h, int W) {
  const size_t w = (size_t)W, n = h->ds.n_up, N = h->ds.N, L = h->ds.L, na = h->ds.n_atoms;
  GradLayout g;
  g.nparts = adj_position_parts(h->ds);
  const size_t rows = w * (n + h->ds.n_dn);
  g.nz = (int)std::max<size_t>(1, std::min<size_t>(64, rows / 1024));
  size_t o = 0;
  auto take = [&](size_t bytes) { size_t r = o; o = align256(o + bytes); return r; };
  g.jg = take(w * N * 3 * 8);
  g.kbar = take(w * N * L * 8);
  g.dnphi = take(w * n * L * 8);
  g.h1 = take(w * n * n * 8);
  g.h2 = take(w * n * n * 8);
  g.gbar = take(w * n * n * 8);
  g.btbar = take(w * n * L * 8);
  g.abar = take(w * n * L * 8);
  g.phibar_a = take(w * n * L * 8);
  g.phibar_b = take(w * n * L * 8);
  g.phibar_dn = take(w * n * L * 8);
  g.part = take(w * g.nparts * na * 3 * 8);
  g.rbar = take(w * N * 3 * 8);
  g.rbar_at = take(w * na * 3 * 8);
  g.jpar = take(w * 3 * 8);
  g.eL = take(w * 8);
  g.lam_part = take((size_t)g.nz * L * L * 8);
  g.tc_lam = h->tc_lambda && h->ds.n_dn == h->ds.n_up && n > 0;
  g.seg_w = g.tc_lam ? (int)std::max<size_t>(1, 2048 / n) : 0;
  g.nseg = g.tc_lam ? 2 * ((W + g.seg_w - 1) / g.seg_w) : 0;
  g.kpseg = g.tc_lam ? (int)((g.seg_w * n + 63) / 64 * 64) : 0;
  const size_t pk = g.tc_lam ? (size_t)g.nseg * L * kLamBarSlices * g.kpseg * 2 : 0;
  g.tc_u = take(pk);
  g.tc_v = take(pk);
  g.tc_eu = take(g.tc_lam ? (size_t)g.nseg * L * 4 : 0);
  g.tc_ev = take(g.tc_lam ? (size_t)g.nseg * L * 4 : 0);
  g.tc_part = take(g.tc_lam ? (size_t)g.nseg * L * L * 8 : 0);
  g.total = o;
  return g;
}

}  // namespace

void jagp_set_cuda_error(cudaError_t e) { g_last_cuda_error = cudaGetErrorString(e); }

void jagp_set_detail(const char *fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_detail, sizeof(g_detail), fmt, ap);
  va_end(ap);
}

jagp_status_t jagp_note(jagp_ctx *h, const char *fn, jagp_status_t s) {
  if (s != JAGP_OK && h) {
    h->last_status = s;
    snprintf(h->last_error, sizeof(h->last_error), "%s: %s%s%s%s%s", fn, jagp_status_string(s),
             s == JAGP_ERR_CUDA ? ": " : "", s == JAGP_ERR_CUDA ? g_last_cuda_error : "", g_detail[0] ? ": " : "",
             g_detail);
  }
  g_detail[0] = 0;
  return s;
}

extern "C" {

size_t jagp_grad_workspace_bytes(jagp_handle_t h, int W) {
  if (!h || W <= 0 || W > h->max_walkers) return 0;
  return grad_layout(h, W).total;
}

static jagp_status_t jagp_grad_impl(jagp_handle_t h, const double *d_r, void *d_state, int W, const double *d_seed_logpsi,
                        const double *d_seed_eL, void *d_work, double *d_eL, double *d_dlambda, double *d_djas,
                        double *d_dR, double *d_dR_walker, double *d_dr, void *stream) {
  jagp_status_t s = check_walkers(h, W, d_state);
  if (s != JAGP_OK) return s;
  if (!d_r || !d_work || (reinterpret_cast<uintptr_t>(d_work) & 255u)) return JAGP_ERR_INVALID_ARG;
  if (h->precision != JAGP_PREC_FP64) return JAGP_ERR_UNSUPPORTED;
  if (h->ds.use_j3) {
    jagp_set_detail("the adjoint does not carry the three-body Jastrow");
    return JAGP_ERR_UNSUPPORTED;
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const DevSystem &d = h->ds;
  const int n = d.n_up, nd = d.n_dn, N = d.N, Lb = d.L;
  const Layout L = layout_of(h, W);
  const GradLayout G = grad_layout(h, W);
  char *wk = static_cast<char *>(d_work);
  auto wp = [&](size_t off) { return reinterpret_cast<double *>(wk + off); };
  double *eL = d_eL ? d_eL : wp(G.eL);
  // forward: M vectors and grad D / D at the current state
  s = run_local_energy<double>(h, d_r, d_state, W, eL, nullptr, st);
  if (s != JAGP_OK) return s;
  double *kbar = wp(G.kbar), *dnphi = wp(G.dnphi);
  LAUNCH(0, 1, launch_adj_kvec(d, d_r, d_seed_eL, wp(G.jg), kbar, dnphi, W, st));
  LAUNCH(JAGP_KERNEL_GEMM_ROWS, 1,
         launch_gemm_rows<double>(kbar, (size_t)N * Lb, at<double>(d_state, L.bt), (size_t)n * Lb, n, n, Lb,
                                  wp(G.h1), (size_t)n * n, n, W, st));
  if (nd > 0)
    LAUNCH(JAGP_KERNEL_GEMM_ROWS, 1,
           launch_gemm_rows<double>(at<double>(d_state, L.a_up), (size_t)n * Lb, kbar + (size_t)n * Lb,
                                    (size_t)N * Lb, n, nd, Lb, wp(G.h2), (size_t)n * n, n, W, st));
  if (n <= kMaxUpGrad) {
    LAUNCH(0, 1, launch_adj_gbar(at<double>(d_state, L.ginv), wp(G.h1), wp(G.h2), d_seed_logpsi, n, nd, wp(G.gbar),
                                 W, st));
    LAUNCH(0, 1,
           launch_adj_rows(d, at<double>(d_state, L.ginv), wp(G.gbar), at<double>(d_state, L.phi_up),
                           at<double>(d_state, L.bt), kbar, wp(G.btbar), wp(G.abar), wp(G.phibar_a), W, st));
  } else {
    LAUNCH(0, 8,
           launch_adj_rows_gemm(d, at<double>(d_state, L.ginv), wp(G.h1), wp(G.h2), d_seed_logpsi,
                                at<double>(d_state, L.phi_up), at<double>(d_state, L.bt), kbar, wp(G.gbar),
                                wp(G.btbar), wp(G.abar), wp(G.phibar_a), W, st));
  }
  // phibar_dn = Btbar^T lambda rows, phibar_b = lambda Abar rows (on the tensor
  // cores when the handle has FP64-equivalent products)
  if (nd > 0) {
    s = lambda_products(h, wp(G.btbar), nullptr, wp(G.phibar_dn), true, nullptr, nullptr, W * nd, nd, n, W * nd,
                        d_state, W, st);
    if (s != JAGP_OK) return s;
  }
  s = lambda_products(h, wp(G.abar), nullptr, wp(G.phibar_b), false, nullptr, nullptr, W * n, n, n, W * n, d_state,
                      W, st);
  if (s != JAGP_OK) return s;
  LAUNCH(0, 1,
         launch_adj_positions(d, d_r, d_seed_eL, wp(G.jg), at<double>(d_state, L.mbuf), wp(G.phibar_a),
                              wp(G.phibar_b), wp(G.phibar_dn), d.shell_atom, wp(G.rbar), wp(G.part), W, st));
  LAUNCH(0, 1,
         launch_adj_jastrow(d, d_r, d_seed_logpsi, d_seed_eL, wp(G.jg), at<double>(d_state, L.kin), wp(G.rbar),
                            wp(G.rbar_at), wp(G.jpar), W, st));
  LAUNCH(0, 1, launch_adj_reduce(wp(G.part), G.nparts, d.n_atoms, wp(G.rbar_at), wp(G.jpar), W, d_dR, d_djas, st));
  if (d_dlambda && G.tc_lam) {
    // lambda-bar = sum over rows of U^T V with (U, V) = (Btbar, dnphi) and
    // (phi_up, Abar) on the tensor cores: the columns of each segment of
    // seg_w walkers cut into eight exact 7-bit slices (K <= 2048 per segment,
    // so every accumulator sum stays exact), the per-segment FP64 products,
    // then their sum in segment order
    uint16_t *pu = reinterpret_cast<uint16_t *>(wk + G.tc_u), *pv = reinterpret_cast<uint16_t *>(wk + G.tc_v);
    int *eu = reinterpret_cast<int *>(wk + G.tc_eu), *ev = reinterpret_cast<int *>(wk + G.tc_ev);
    const int full = W / G.seg_w, rest = W - full * G.seg_w, per = G.nseg / 2;
    const size_t segk = (size_t)Lb * kLamBarSlices * G.kpseg;  // packed elements per segment
    const double *U[2] = {wp(G.btbar), at<double>(d_state, L.phi_up)}, *V[2] = {dnphi, wp(G.abar)};
    for (int set = 0; set < 2; ++set) {
      const size_t s0 = (size_t)set * per;
      const size_t xw = (size_t)G.seg_w * n * Lb;  // elements per segment of the [W][n][L] tables
      for (int part = 0; part < 2; ++part) {
        const int segs = part == 0 ? full : (rest > 0 ? 1 : 0);
        if (segs == 0) continue;
        const int rows = (part == 0 ? G.seg_w : rest) * n;
        const size_t sg = s0 + (part == 0 ? 0 : full);
        const size_t src = (part == 0 ? 0 : (size_t)full * xw);
        LAUNCH(0, 1,
               launch_pack_cols(U[set] + src, nullptr, nullptr, xw, rows, Lb, G.kpseg, segs, pu + sg * segk,
                                eu + sg * Lb, nullptr, 0, 0, st, kLamBarSlices, kLamBarBits));
        LAUNCH(0, 1,
               launch_pack_cols(V[set] + src, nullptr, nullptr, xw, rows, Lb, G.kpseg, segs, pv + sg * segk,
                                ev + sg * Lb, nullptr, 0, 0, st, kLamBarSlices, kLamBarBits));
      }
    }
    int pa[kMaxPairs], pb[kMaxPairs];
    const int np = slice_pairs(kLamBarSlices, pa, pb);
    LAUNCH(JAGP_KERNEL_LAMBDA_ROWS, 1,
           launch_umma_gemm(pu, G.nseg * Lb, nullptr, kLamBarSlices, pv, Lb, kLamBarSlices, G.kpseg, np, pa, pb,
                            nullptr, 0, nullptr, h->d_err, st, eu, ev, nullptr, 0, wp(G.tc_part), kLamBarBits, Lb,
                            G.nseg, 0, Lb, (long long)Lb * Lb, Lb, 1));
    LAUNCH(0, 1, launch_adj_lambda_sum(wp(G.tc_part), G.nseg, Lb, d_dlambda, st));
  } else if (d_dlambda) {
    LAUNCH(0, 1,
           launch_adj_lambda(wp(G.btbar), dnphi, at<double>(d_state, L.phi_up), wp(G.abar), W, n, nd, Lb,
                             wp(G.lam_part), G.nz, d_dlambda, st));
  }
  if (d_dr) JAGP_CU(cudaMemcpyAsync(d_dr, wp(G.rbar), (size_t)W * N * 3 * 8, cudaMemcpyDeviceToDevice, st));
  if (d_dR_walker)
    JAGP_CU(cudaMemcpyAsync(d_dR_walker, wp(G.rbar_at), (size_t)W * d.n_atoms * 3 * 8, cudaMemcpyDeviceToDevice, st));
  return JAGP_OK;
}


const char *jagp_last_cuda_error(void) { return g_last_cuda_error; }

const char *jagp_status_string(jagp_status_t s) {
  switch (s) {
    case JAGP_OK: return "ok";
    case JAGP_ERR_INVALID_ARG: return "invalid argument";
    case JAGP_ERR_SINGULAR: return "singular geminal matrix";
    case JAGP_ERR_NONFINITE: return "non-finite position or ratio";
    case JAGP_ERR_OOM: return "device allocation failed";
    case JAGP_ERR_TIMEOUT: return "bounded device wait expired";
    case JAGP_ERR_UNSUPPORTED: return "unsupported system or size";
    case JAGP_ERR_CUDA: return "CUDA runtime error";
    default: return "unknown status";
  }
}

jagp_status_t jagp_create(jagp_handle_t *out, const jagp_system_t *sys, const jagp_options_t *opt) {
  if (!out || !sys || !opt) return JAGP_ERR_INVALID_ARG;
  *out = nullptr;
  if (sys->n_atoms <= 0 || !sys->R || !sys->Z) return JAGP_ERR_INVALID_ARG;
  if (sys->n_shells <= 0 || !sys->shell_atom || !sys->shell_l || !sys->shell_radial || !sys->shell_zeta)
    return JAGP_ERR_INVALID_ARG;
  if (!sys->lambda || sys->n_up < 1 || sys->n_dn < 0) return JAGP_ERR_INVALID_ARG;
  if (sys->n_dn > sys->n_up) return JAGP_ERR_UNSUPPORTED;
  if (sys->n_up > kMaxUp) return JAGP_ERR_UNSUPPORTED;
  if (sys->n_up > sys->n_dn && !sys->unpaired) return JAGP_ERR_INVALID_ARG;
  if (opt->precision != JAGP_PREC_FP64 && opt->precision != JAGP_PREC_MIXED) return JAGP_ERR_UNSUPPORTED;
  if (opt->max_walkers <= 0 || !(opt->delta > 0.0) || !isfinite(opt->delta)) return JAGP_ERR_INVALID_ARG;
  if (opt->refresh_moves < 0) return JAGP_ERR_INVALID_ARG;
  // Shell table in evaluation order: grouped by (radial type, l) so that the 32
  // lanes of a warp, which take consecutive shells, run the same branch; each
  // record keeps the offset of its first function in the caller's order.
  int L = 0;
  std::vector<double4> geo;
  std::vector<float4> geo_dw;
  std::vector<int> info, satom;
  std::vector<int> offset(sys->n_shells);
  for (int k = 0; k < sys->n_shells; ++k) {
    const int l = sys->shell_l[k], a = sys->shell_atom[k], rad = sys->shell_radial[k];
    if (l < 0 || l > 2 || rad < 0 || rad > 1) return JAGP_ERR_UNSUPPORTED;
    if (a < 0 || a >= sys->n_atoms || !(sys->shell_zeta[k] >= 0.0)) return JAGP_ERR_INVALID_ARG;
    offset[k] = L;
    L += 2 * l + 1;
  }
  for (int rad = 0; rad <= 1; ++rad)
    for (int l = 0; l <= 2; ++l)
      for (int k = 0; k < sys->n_shells; ++k) {
        if (sys->shell_l[k] != l || sys->shell_radial[k] != rad) continue;
        const int a = sys->shell_atom[k];
        geo.push_back(make_double4(sys->R[3 * a], sys->R[3 * a + 1], sys->R[3 * a + 2], sys->shell_zeta[k]));
        // the same record as double-words for the FP32 path: FP32 roundings, then the remainders
        const double v4[4] = {sys->R[3 * a], sys->R[3 * a + 1], sys->R[3 * a + 2], sys->shell_zeta[k]};
        float hi[4], lo[4];
        for (int c = 0; c < 4; ++c) {
          hi[c] = static_cast<float>(v4[c]);
          lo[c] = static_cast<float>(v4[c] - static_cast<double>(hi[c]));
        }
        geo_dw.push_back(make_float4(hi[0], hi[1], hi[2], hi[3]));
        geo_dw.push_back(make_float4(lo[0], lo[1], lo[2], lo[3]));
        info.push_back(l | (rad << 2) | (offset[k] << 8));
        satom.push_back(a);
      }
  const int na = sys->n_atoms, k_unp = sys->n_up - sys->n_dn;
  std::vector<double> c1(na), lamT((size_t)L * L);
  double vii = 0.0;
  for (int a = 0; a < na; ++a) {
    c1[a] = pow(2.0 * sys->Z[a], 0.25);
    for (int b = a + 1; b < na; ++b) {
      const double dx = sys->R[3 * a] - sys->R[3 * b], dy = sys->R[3 * a + 1] - sys->R[3 * b + 1],
                   dz = sys->R[3 * a + 2] - sys->R[3 * b + 2];
      vii += sys->Z[a] * sys->Z[b] / sqrt(dx * dx + dy * dy + dz * dz);
    }
  }
  for (int i = 0; i < L; ++i)
    for (int j = 0; j < L; ++j) lamT[(size_t)j * L + i] = sys->lambda[(size_t)i * L + j];

  // three/four-body Jastrow: its shell table (caller order) and couplings
  int LJ = 0;
  std::vector<double4> jgeo;
  std::vector<int> jinfo;
  if (sys->use_j3) {
    if (sys->n_jshells <= 0 || !sys->jshell_atom || !sys->jshell_l || !sys->jshell_radial || !sys->jshell_zeta ||
        !sys->j3_para || !sys->j3_anti)
      return JAGP_ERR_INVALID_ARG;
    for (int k = 0; k < sys->n_jshells; ++k) {
      const int l = sys->jshell_l[k], a = sys->jshell_atom[k], rad = sys->jshell_radial[k];
      if (l < 0 || l > 2 || rad < 0 || rad > 1) return JAGP_ERR_UNSUPPORTED;
      if (a < 0 || a >= sys->n_atoms || !(sys->jshell_zeta[k] >= 0.0)) return JAGP_ERR_INVALID_ARG;
      jgeo.push_back(make_double4(sys->R[3 * a], sys->R[3 * a + 1], sys->R[3 * a + 2], sys->jshell_zeta[k]));
      jinfo.push_back(l | (rad << 2) | (LJ << 8));
      LJ += 2 * l + 1;
    }
    for (int i = 0; i < LJ; ++i)
      for (int j = 0; j < LJ; ++j)
        if (sys->j3_para[i * LJ + j] != sys->j3_para[j * LJ + i] || sys->j3_anti[i * LJ + j] != sys->j3_anti[j * LJ + i]) {
          jagp_set_detail("the three-body couplings must be symmetric");
          return JAGP_ERR_INVALID_ARG;
        }
    // the sequential acceptance keeps G~^{-1} and the Jastrow vectors in shared memory
    const size_t n = sys->n_up, N = sys->n_up + sys->n_dn;
    if ((N * 3 + n * n + 3 * n + 9 * (size_t)LJ) * 8 > 200 * 1024) {
      jagp_set_detail("three-body Jastrow with N_up = %d and LJ = %d does not fit the acceptance kernel", sys->n_up,
                      LJ);
      return JAGP_ERR_UNSUPPORTED;
    }
  }
  jagp_ctx *h = new jagp_ctx();
  if (cudaGetDevice(&h->device) != cudaSuccess) {
    delete h;
    return JAGP_ERR_CUDA;
  }
  std::call_once(g_attr_once, [] {
    g_attr_err = setup_kernel_attributes();
    if (g_attr_err == cudaSuccess) g_attr_err = setup_walker_attributes();
    if (g_attr_err == cudaSuccess) g_attr_err = setup_energy_attributes();
    if (g_attr_err == cudaSuccess) g_attr_err = setup_umma_attributes();
    if (g_attr_err == cudaSuccess) g_attr_err = setup_adjoint_attributes();
    if (g_attr_err == cudaSuccess) g_attr_err = setup_forces_attributes();
  });
  if (g_attr_err != cudaSuccess) {
    delete h;
    return JAGP_ERR_CUDA;
  }
  // one allocation: R, Z, c1, shell geo, shell info, lambda, lambda^T, unpaired
  size_t off = 0;
  auto take = [&](size_t bytes) { size_t r = off; off = align256(off + bytes); return r; };
  const size_t oR = take(na * 3 * 8), oZ = take(na * 8), oC = take(na * 8);
  const size_t oG = take(sys->n_shells * sizeof(double4)), oI = take(sys->n_shells * sizeof(int));
  const size_t oGd = take(sys->n_shells * 2 * sizeof(float4));
  const size_t oSa = take(sys->n_shells * sizeof(int));
  const size_t oAf = take(na * sizeof(float4));
  const size_t oL = take((size_t)L * L * 8), oT = take((size_t)L * L * 8);
  const size_t oU = take((size_t)(k_unp > 0 ? k_unp : 1) * L * 8);
  // mixed path: lambda^T and lambda as fixed-point slices, rows padded to kp
  const bool mixed = opt->precision == JAGP_PREC_MIXED;
  const bool tc64 = !mixed && opt->fp64_tensor_cores != 0;
  const bool tc = mixed || tc64;
  const int kp = (L + 63) / 64 * 64;
  // slices per element: mixed 6 x 8 bits; FP64-equivalent 7 x 8 bits, or 8 x 7
  // bits when L > 512 so that the leading accumulators stay exact
  const int nsl = mixed ? kFixedSlices : (tc64 ? (L <= 512 ? 7 : 8) : 0);
  const int nterms = nsl;
  const int bits = tc64 && L > 512 ? 7 : 8;
  const size_t split_bytes = tc ? (size_t)L * nterms * kp * 2 : 0;
  const size_t exp_bytes = tc ? (size_t)L * 4 : 0;
  const size_t oSA = take(split_bytes), oSB = take(split_bytes), oXA = take(exp_bytes), oXB = take(exp_bytes);
  const size_t oE = take(16);
  const size_t oJG = take((size_t)jgeo.size() * sizeof(double4)), oJI = take(jinfo.size() * sizeof(int));
  const size_t oJP = take((size_t)LJ * LJ * 8), oJA = take((size_t)LJ * LJ * 8);
  std::vector<uint16_t> sA(split_bytes / 2, 0), sB(split_bytes / 2, 0);
  std::vector<int> xA(tc ? L : 0), xB(tc ? L : 0);
  if (tc) {
    for (int nn = 0; nn < L; ++nn) {
      // column nn, then row nn
      uint16_t *ra = &sA[(size_t)nn * nterms * kp], *rb = &sB[(size_t)nn * nterms * kp];
      xA[nn] = slice_row_fixed(sys->lambda + nn, (size_t)L, L, ra, (size_t)kp, nsl, bits);
      xB[nn] = slice_row_fixed(sys->lambda + (size_t)nn * L, 1, L, rb, (size_t)kp, nsl, bits);
    }
  }
  std::vector<float4> atom_f(na);
  for (int a = 0; a < na; ++a)
    atom_f[a] = make_float4(static_cast<float>(sys->R[3 * a]), static_cast<float>(sys->R[3 * a + 1]),
                            static_cast<float>(sys->R[3 * a + 2]), static_cast<float>(c1[a]));
  if (cudaMalloc(&h->d_mem, off) != cudaSuccess) {
    delete h;
    return JAGP_ERR_OOM;
  }
  char *b = static_cast<char *>(h->d_mem);
  bool ok = cudaMemcpy(b + oR, sys->R, na * 3 * 8, cudaMemcpyHostToDevice) == cudaSuccess &&
            cudaMemcpy(b + oZ, sys->Z, na * 8, cudaMemcpyHostToDevice) == cudaSuccess &&
            cudaMemcpy(b + oC, c1.data(), na * 8, cudaMemcpyHostToDevice) == cudaSuccess &&
            cudaMemcpy(b + oG, geo.data(), sys->n_shells * sizeof(double4), cudaMemcpyHostToDevice) == cudaSuccess &&
            cudaMemcpy(b + oGd, geo_dw.data(), sys->n_shells * 2 * sizeof(float4), cudaMemcpyHostToDevice) ==
                cudaSuccess &&
            cudaMemcpy(b + oI, info.data(), sys->n_shells * sizeof(int), cudaMemcpyHostToDevice) == cudaSuccess &&
            cudaMemcpy(b + oSa, satom.data(), sys->n_shells * sizeof(int), cudaMemcpyHostToDevice) == cudaSuccess &&
            cudaMemcpy(b + oAf, atom_f.data(), na * sizeof(float4), cudaMemcpyHostToDevice) == cudaSuccess &&
            cudaMemcpy(b + oL, sys->lambda, (size_t)L * L * 8, cudaMemcpyHostToDevice) == cudaSuccess &&
            cudaMemcpy(b + oT, lamT.data(), (size_t)L * L * 8, cudaMemcpyHostToDevice) == cudaSuccess &&
            (k_unp == 0 ||
             cudaMemcpy(b + oU, sys->unpaired, (size_t)k_unp * L * 8, cudaMemcpyHostToDevice) == cudaSuccess) &&
            (!tc || (cudaMemcpy(b + oSA, sA.data(), split_bytes, cudaMemcpyHostToDevice) == cudaSuccess &&
                        cudaMemcpy(b + oSB, sB.data(), split_bytes, cudaMemcpyHostToDevice) == cudaSuccess &&
                        cudaMemcpy(b + oXA, xA.data(), exp_bytes, cudaMemcpyHostToDevice) == cudaSuccess &&
                        cudaMemcpy(b + oXB, xB.data(), exp_bytes, cudaMemcpyHostToDevice) == cudaSuccess)) &&
            cudaMemset(b + oE, 0, 16) == cudaSuccess &&
            (LJ == 0 ||
             (cudaMemcpy(b + oJG, jgeo.data(), jgeo.size() * sizeof(double4), cudaMemcpyHostToDevice) == cudaSuccess &&
              cudaMemcpy(b + oJI, jinfo.data(), jinfo.size() * sizeof(int), cudaMemcpyHostToDevice) == cudaSuccess &&
              cudaMemcpy(b + oJP, sys->j3_para, (size_t)LJ * LJ * 8, cudaMemcpyHostToDevice) == cudaSuccess &&
              cudaMemcpy(b + oJA, sys->j3_anti, (size_t)LJ * LJ * 8, cudaMemcpyHostToDevice) == cudaSuccess));
  if (!ok) {
    cudaFree(h->d_mem);
    delete h;
    return JAGP_ERR_CUDA;
  }
  DevSystem &d = h->ds;
  d.n_atoms = na;
  d.n_shells = sys->n_shells;
  d.L = L;
  d.n_up = sys->n_up;
  d.n_dn = sys->n_dn;
  d.N = sys->n_up + sys->n_dn;
  d.R = reinterpret_cast<const double *>(b + oR);
  d.Z = reinterpret_cast<const double *>(b + oZ);
  d.c1 = reinterpret_cast<const double *>(b + oC);
  d.shell_geo = reinterpret_cast<const double4 *>(b + oG);
  d.shell_dw = reinterpret_cast<const float4 *>(b + oGd);
  d.shell_info = reinterpret_cast<const int *>(b + oI);
  d.shell_atom = reinterpret_cast<const int *>(b + oSa);
  d.lam = reinterpret_cast<const double *>(b + oL);
  d.lamT = reinterpret_cast<const double *>(b + oT);
  d.unpaired = reinterpret_cast<const double *>(b + oU);
  d.b_ea = sys->b_ea;
  d.b_para = sys->b_para;
  d.b_anti = sys->b_anti;
  d.atom_f = reinterpret_cast<const float4 *>(b + oAf);
  d.b_ea_f = static_cast<float>(sys->b_ea);
  d.b_para_f = static_cast<float>(sys->b_para);
  d.b_anti_f = static_cast<float>(sys->b_anti);
  d.use_j1 = sys->use_j1 ? 1 : 0;
  d.use_j2 = sys->use_j2 ? 1 : 0;
  d.j2_si = sys->j2_spin_independent ? 1 : 0;
  d.v_ii = vii;
  d.delta = opt->delta;
  d.key0 = (uint32_t)(opt->seed & 0xffffffffu);
  d.key1 = (uint32_t)(opt->seed >> 32);
  d.use_j3 = LJ > 0 ? 1 : 0;
  d.n_jshells = LJ > 0 ? sys->n_jshells : 0;
  d.LJ = LJ;
  d.jshell_geo = reinterpret_cast<const double4 *>(b + oJG);
  d.jshell_info = reinterpret_cast<const int *>(b + oJI);
  d.j3p = reinterpret_cast<const double *>(b + oJP);
  d.j3a = reinterpret_cast<const double *>(b + oJA);
  h->precision = opt->precision;
  h->kp = kp;
  h->split_lamT = tc ? reinterpret_cast<const uint16_t *>(b + oSA) : nullptr;
  h->split_lam = tc ? reinterpret_cast<const uint16_t *>(b + oSB) : nullptr;
  h->exp_lamT = tc ? reinterpret_cast<const int *>(b + oXA) : nullptr;
  h->exp_lam = tc ? reinterpret_cast<const int *>(b + oXB) : nullptr;
  h->tc_lambda = tc;
  h->tc_slices = nsl;
  h->tc_bits = bits;
  h->d_err = reinterpret_cast<int *>(b + oE);
  h->max_walkers = opt->max_walkers;
  h->drift_tol = opt->drift_tol > 0.0 ? opt->drift_tol : (mixed ? 1e-3 : 1e-8);
  h->refresh_moves = opt->refresh_moves;
  *out = h;
  return JAGP_OK;
}

jagp_status_t jagp_destroy(jagp_handle_t h) {
  if (!h) return JAGP_ERR_INVALID_ARG;
  for (auto &p : h->prof_events) {
    cudaEventDestroy(p.first);
    cudaEventDestroy(p.second);
  }
  cudaError_t e = cudaFree(h->d_mem);
  delete h;
  return e == cudaSuccess ? JAGP_OK : JAGP_ERR_CUDA;
}

size_t jagp_state_bytes(jagp_handle_t h, int W) {
  if (!h || W <= 0 || W > h->max_walkers) return 0;
  return layout_of(h, W).total;
}

static jagp_status_t jagp_eval_impl(jagp_handle_t h, const double *d_r, int W, void *d_state, double *d_logabs,
                        double *d_sign, void *stream) {
  jagp_status_t s = check_walkers(h, W, d_state);
  if (s != JAGP_OK) return s;
  if (!d_r) return JAGP_ERR_INVALID_ARG;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (h->precision == JAGP_PREC_MIXED) return run_eval<float>(h, d_r, W, d_state, d_logabs, d_sign, st);
  return run_eval<double>(h, d_r, W, d_state, d_logabs, d_sign, st);
}

// ---------------------------------------------------------------------------
// Tile autotuner: every candidate is launched on the handle's own operands in
// the walker state (its tables are overwritten: jagp_eval must follow), timed
// with CUDA events on the caller's stream (two untimed and five timed calls),
// and the fastest is kept in the handle.  The candidates change only how the
// outputs are tiled, never the order of any sum, so results do not depend on
// the choice.
// ---------------------------------------------------------------------------
}  // extern "C"

namespace {

template <typename F>
cudaError_t time_calls(F &&f, cudaStream_t st, float *ms) {
  cudaEvent_t a = nullptr, b = nullptr;
  cudaError_t e = cudaEventCreate(&a);
  if (e == cudaSuccess) e = cudaEventCreate(&b);
  for (int i = 0; i < 2 && e == cudaSuccess; ++i) e = f();
  if (e == cudaSuccess) e = cudaEventRecord(a, st);
  for (int i = 0; i < 5 && e == cudaSuccess; ++i) e = f();
  if (e == cudaSuccess) e = cudaEventRecord(b, st);
  if (e == cudaSuccess) e = cudaEventSynchronize(b);
  if (e == cudaSuccess) e = cudaEventElapsedTime(ms, a, b);
  if (e == cudaSuccess) *ms /= 5.0f;
  if (a) cudaEventDestroy(a);
  if (b) cudaEventDestroy(b);
  return e;
}

template <typename T>
jagp_status_t tune_products(jagp_ctx *h, void *state, int W, cudaStream_t st, jagp_tuning_t *out) {
  const Layout L = layout_of(h, W);
  const DevSystem &d = h->ds;
  const int n = d.n_up, Lb = d.L;
  JAGP_CU(cudaMemsetAsync(state, 0, L.total, st));
  T *pprop = at<T>(state, L.pprop), *bt = at<T>(state, L.bt), *gprop = at<T>(state, L.gprop);
  T *phi = at<T>(state, L.phi_up);
  const int tiles[3] = {0, 32, 64};
  float best = 0.0f;
  for (int c = 0; c < 3; ++c) {
    float ms = 0.0f;
    JAGP_CU(time_calls([&] { return launch_gemm_rows<T>(pprop, (size_t)n * Lb, bt, (size_t)n * Lb, n, n, Lb, gprop,
                                                        (size_t)n * n, n, W, st, tiles[c]); },
                       st, &ms));
    if (c == 0 || ms < best) {
      best = ms;
      h->tune_tile_prop = tiles[c];
    }
  }
  out->tile_proposals = h->tune_tile_prop;
  out->ms[0] = best;
  double *gm = refresh_g(L, state);
  const int rtiles[4] = {0, 32, 64, 16};  // 16: the four-walkers-per-CTA compensated kernel (FP32, N_up <= 16)
  const int nref = (std::is_same<T, float>::value && n <= 16) ? 4 : 3;
  for (int c = 0; c < nref; ++c) {
    float ms = 0.0f;
    JAGP_CU(time_calls([&] { return refresh_geminal(phi, lo_table(h, state, L.phi_lo), (size_t)n * Lb, bt,
                                                    lo_table(h, state, L.bt_lo), (size_t)n * Lb, n, Lb, gm, W, st,
                                                    rtiles[c]); },
                       st, &ms));
    if (c == 0 || ms < best) {
      best = ms;
      h->tune_tile_refresh = rtiles[c];
    }
  }
  out->tile_refresh = h->tune_tile_refresh;
  out->ms[1] = best;
  if (!h->tc_lambda) return JAGP_OK;
  // tensor-core lambda products of half the orbital rows (the accepted rows of
  // a half-sweep at ~50% acceptance): mixed A_up and Bt (twenty-one pairs each),
  // or the FP64-equivalent products (all pairs of 7 or 8 slices, FP64 result)
  const bool f64 = !std::is_same<T, float>::value;
  uint16_t *pack = at<uint16_t>(state, L.pack);
  int *exps = at<int>(state, L.exps);
  const int rows = (W * n + 1) / 2;
  int pa64[kMaxPairs], pb64[kMaxPairs];
  const int np64 = slice_pairs(h->tc_slices, pa64, pb64);
  for (int side = 0; side < 2; ++side) {
    const bool left = side == 0;
    // tile widths; 16 lets several CTAs share an SM's tensor memory (6 x 16 columns each)
    const int cands[7] = {16, 32, 48, 64, 80, 96, 128};
    // stages: as many as fit (one CTA per SM), three or two (several CTAs per SM),
    // or chunk-major (every slice of a K chunk of 64, 32 or 16 per stage, each
    // loaded once for all pairs; two to four stages, where they fit)
    const int stages[6] = {0, 3, 2, -1, -2, -3};
    const int npairs = f64 ? np64 : kFixedPairs;
    const int *tpa = f64 ? pa64 : kPairA, *tpb = f64 ? pb64 : kPairB;
    const int limit = 64;  // six or more accumulators of bn columns in tensor memory
    float bs = 0.0f;
    int bbn = 0, bst = 0;
    for (int c = 0; c < 7; ++c)
      for (int q = 0; q < 6; ++q) {
        if (cands[c] > limit) continue;
        if (stages[q] < 0 && !umma_chunk_fits(npairs, tpa, tpb, cands[c], stages[q])) continue;
        float ms = 0.0f;
        JAGP_CU(time_calls(
            [&] {
              T *dst = left ? at<T>(state, L.a_up) : bt;
              if (f64)
                return launch_umma_gemm(pack, rows, nullptr, h->tc_slices, left ? h->split_lamT : h->split_lam, Lb,
                                        h->tc_slices, h->kp, np64, pa64, pb64, nullptr, Lb, nullptr, h->d_err, st,
                                        exps, left ? h->exp_lamT : h->exp_lam, nullptr, cands[c],
                                        reinterpret_cast<double *>(dst), h->tc_bits, 0, 0, stages[q]);
              return launch_umma_gemm(pack, rows, nullptr, kFixedSlices, left ? h->split_lamT : h->split_lam, Lb,
                                      kFixedSlices, h->kp, kFixedPairs, kPairA, kPairB,
                                      reinterpret_cast<float *>(dst), Lb, nullptr, h->d_err, st, exps,
                                      left ? h->exp_lamT : h->exp_lam, at<float>(state, left ? L.a_up_lo : L.bt_lo),
                                      cands[c], nullptr, 8, 0, 0, stages[q]);
            },
            st, &ms));
        if (bbn == 0 || ms < bs) {
          bs = ms;
          bbn = cands[c];
          bst = stages[q];
        }
      }
    if (left) {
      h->tune_bn_left = bbn;
      h->tune_st_left = bst;
      out->umma_bn_left = bbn;
      out->umma_stages_left = bst;
      out->ms[2] = bs;
    } else {
      h->tune_bn_right = bbn;
      h->tune_st_right = bst;
      out->umma_bn_right = bbn;
      out->umma_stages_right = bst;
      out->ms[3] = bs;
    }
  }
  return JAGP_OK;
}

}  // namespace

extern "C" {

static jagp_status_t jagp_autotune_impl(jagp_handle_t h, void *d_state, int W, jagp_tuning_t *out, void *stream) {
  jagp_status_t s = check_walkers(h, W, d_state);
  if (s != JAGP_OK) return s;
  if (!out) return JAGP_ERR_INVALID_ARG;
  memset(out, 0, sizeof(*out));
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  s = h->precision == JAGP_PREC_MIXED ? tune_products<float>(h, d_state, W, st, out)
                                      : tune_products<double>(h, d_state, W, st, out);
  if (s != JAGP_OK) return s;
  JAGP_CU(cudaStreamSynchronize(st));
  return JAGP_OK;
}

static jagp_status_t jagp_set_tuning_impl(jagp_handle_t h, const jagp_tuning_t *t) {
  if (!h || !t) return JAGP_ERR_INVALID_ARG;
  const bool mixed = h->precision == JAGP_PREC_MIXED;
  auto tile_ok = [](int v, bool allow16) { return v == -1 || v == 0 || v == 32 || v == 64 || (allow16 && v == 16); };
  if (!tile_ok(t->tile_proposals, false) || !tile_ok(t->tile_refresh, mixed && h->ds.n_up <= 16))
    return JAGP_ERR_INVALID_ARG;
  const int bn[2] = {t->umma_bn_left, t->umma_bn_right}, stg[2] = {t->umma_stages_left, t->umma_stages_right};
  if (!h->tc_lambda) {
    if (bn[0] || bn[1] || stg[0] || stg[1]) return JAGP_ERR_INVALID_ARG;
  } else {
    int pa64[kMaxPairs], pb64[kMaxPairs];
    const int np64 = slice_pairs(h->tc_slices, pa64, pb64);
    for (int side = 0; side < 2; ++side) {
      const bool left = side == 0;
      // six (mixed) or up to eight (FP64-equivalent) accumulators of bn columns in tensor memory
      const int limit = 64;
      if (bn[side] < 0 || bn[side] % 16 || bn[side] > limit) return JAGP_ERR_INVALID_ARG;
      if (stg[side] < -3 || stg[side] == 1 || stg[side] > 6) return JAGP_ERR_INVALID_ARG;
      const int npairs = mixed ? kFixedPairs : np64;
      const int actual = umma_pick_bn(h->ds.L, bn[side] ? bn[side] : limit);
      if (stg[side] < 0 && !umma_chunk_fits(npairs, mixed ? kPairA : pa64, mixed ? kPairB : pb64, actual, stg[side]))
        return JAGP_ERR_INVALID_ARG;
    }
  }
  h->tune_tile_prop = t->tile_proposals;
  h->tune_tile_refresh = t->tile_refresh;
  h->tune_bn_left = bn[0];
  h->tune_bn_right = bn[1];
  h->tune_st_left = stg[0];
  h->tune_st_right = stg[1];
  return JAGP_OK;
}

static jagp_status_t vmc_sweep_impl(jagp_handle_t h, double *d_r, void *d_state, int W, int nsweeps, uint64_t walker0,
                        uint64_t sweep0, double *d_eL, double *d_acc, void *stream) {
  jagp_status_t s = check_walkers(h, W, d_state);
  if (s != JAGP_OK) return s;
  if (!d_r || nsweeps < 0) return JAGP_ERR_INVALID_ARG;
  if (walker0 + (uint64_t)W > 0x100000000ull || sweep0 + (uint64_t)nsweeps > 0x100000000ull)
    return JAGP_ERR_INVALID_ARG;  // Philox counter words are 32-bit
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (h->precision == JAGP_PREC_MIXED)
    return run_sweeps<float>(h, d_r, d_state, W, nsweeps, walker0, sweep0, d_eL, d_acc, st);
  return run_sweeps<double>(h, d_r, d_state, W, nsweeps, walker0, sweep0, d_eL, d_acc, st);
}

static jagp_status_t local_energy_impl(jagp_handle_t h, const double *d_r, void *d_state, int W, double *d_eL,
                           double *d_parts, void *stream) {
  jagp_status_t s = check_walkers(h, W, d_state);
  if (s != JAGP_OK) return s;
  if (!d_r || !d_eL) return JAGP_ERR_INVALID_ARG;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (h->precision == JAGP_PREC_MIXED) return run_local_energy<float>(h, d_r, d_state, W, d_eL, d_parts, st);
  return run_local_energy<double>(h, d_r, d_state, W, d_eL, d_parts, st);
}

jagp_status_t jagp_gemm_bf16x(const uint16_t *d_A, int M, int a_terms, const uint16_t *d_B, int N, int b_terms,
                              int Kp, int npairs, const int *h_pair_a, const int *h_pair_b, float *d_C,
                              long long ldc, const int *d_rows, const int *d_count, const int *d_row_exp,
                              const int *d_col_exp, int *d_err, void *stream) {
  if (!d_A || !d_B || !d_C || !d_err || !h_pair_a || !h_pair_b) return JAGP_ERR_INVALID_ARG;
  if (M <= 0 || N <= 0 || Kp <= 0 || Kp % 64 != 0 || ldc < N || npairs < 1 || npairs > kFixedPairs)
    return JAGP_ERR_INVALID_ARG;
  if (a_terms < 1 || a_terms > kFixedSlices || b_terms < 1 || b_terms > kFixedSlices) return JAGP_ERR_INVALID_ARG;
  if ((d_row_exp == nullptr) != (d_col_exp == nullptr)) return JAGP_ERR_INVALID_ARG;
  if (d_row_exp)
    for (int p = 0; p < npairs; ++p)
      if (h_pair_a[p] + h_pair_b[p] > kFixedSlices - 1) return JAGP_ERR_INVALID_ARG;
  std::call_once(g_attr_once, [] {
    g_attr_err = setup_kernel_attributes();
    if (g_attr_err == cudaSuccess) g_attr_err = setup_walker_attributes();
    if (g_attr_err == cudaSuccess) g_attr_err = setup_energy_attributes();
    if (g_attr_err == cudaSuccess) g_attr_err = setup_umma_attributes();
    if (g_attr_err == cudaSuccess) g_attr_err = setup_adjoint_attributes();
    if (g_attr_err == cudaSuccess) g_attr_err = setup_forces_attributes();
  });
  if (g_attr_err != cudaSuccess) return JAGP_ERR_CUDA;
  const cudaError_t e = launch_umma_gemm(d_A, M, d_count, a_terms, d_B, N, b_terms, Kp, npairs, h_pair_a, h_pair_b,
                                         d_C, ldc, d_rows, d_err, static_cast<cudaStream_t>(stream), d_row_exp,
                                         d_col_exp);
  if (e == cudaErrorInvalidValue) return JAGP_ERR_INVALID_ARG;
  return e == cudaSuccess ? JAGP_OK : JAGP_ERR_CUDA;
}

static jagp_status_t jagp_profile_impl(jagp_handle_t h, int kernel, int enable) {
  if (!h || kernel < 1 || kernel > JAGP_KERNEL_ENERGY) return JAGP_ERR_INVALID_ARG;
  h->prof_kernel = enable ? kernel : 0;
  return JAGP_OK;
}

static jagp_status_t jagp_profile_read_impl(jagp_handle_t h, double *h_total_ms, long long *h_launches) {
  if (!h || !h_total_ms || !h_launches) return JAGP_ERR_INVALID_ARG;
  double tot = 0.0;
  jagp_status_t rc = JAGP_OK;
  for (auto &p : h->prof_events) {
    float ms = 0.f;
    if (cudaEventSynchronize(p.second) != cudaSuccess || cudaEventElapsedTime(&ms, p.first, p.second) != cudaSuccess)
      rc = JAGP_ERR_CUDA;
    tot += ms;
    cudaEventDestroy(p.first);
    cudaEventDestroy(p.second);
  }
  *h_launches = (long long)h->prof_events.size();
  *h_total_ms = tot;
  h->prof_events.clear();
  return rc;
}

long long jagp_launch_count(jagp_handle_t h) { return h ? h->launches : -1;
}

static jagp_status_t jagp_walker_info_impl(jagp_handle_t h, const void *d_state, int W, double *d_logabs, double *d_sign,
                               double *d_naccept, double *d_drift, int *d_status, void *stream) {
  jagp_status_t s = check_walkers(h, W, d_state);
  if (s != JAGP_OK) return s;
  const Layout L = layout_of(h, W);
  void *sp = const_cast<void *>(d_state);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  LAUNCH(0, 1, launch_walker_info(at<double>(sp, L.scal), at<int>(sp, L.status), W, d_logabs, d_sign, d_naccept,
                                  d_drift, d_status, st));
  return JAGP_OK;
}

static jagp_status_t jagp_walker_status_impl(jagp_handle_t h, const void *d_state, int W, int *h_bits, void *stream) {
  jagp_status_t s = check_walkers(h, W, d_state);
  if (s != JAGP_OK) return s;
  if (!h_bits) return JAGP_ERR_INVALID_ARG;
  const Layout L = layout_of(h, W);
  std::vector<int> bits(W);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  JAGP_CU(cudaMemcpyAsync(bits.data(), static_cast<const char *>(d_state) + L.status, (size_t)W * sizeof(int),
                          cudaMemcpyDeviceToHost, st));
  JAGP_CU(cudaStreamSynchronize(st));
  int o = 0, nbad = 0;
  for (int w = 0; w < W; ++w) {
    o |= bits[w];
    nbad += bits[w] != 0;
  }
  *h_bits = o;
  // a tensor-core pipeline wait that ran out of time leaves its flag set
  int err = 0;
  JAGP_CU(cudaMemcpy(&err, h->d_err, sizeof(int), cudaMemcpyDeviceToHost));
  if (err) {
    jagp_set_detail("a tensor-core pipeline wait expired (flag %d)", err);
    return JAGP_ERR_TIMEOUT;
  }
  if (nbad) {
    // not a failure of the call: the text records which walkers carry bits
    h->last_status = JAGP_OK;
    snprintf(h->last_error, sizeof(h->last_error),
             "jagp_walker_status: %d of %d walkers with status bits 0x%x (1 NONFINITE, 2 SINGULAR, 4 DRIFT)", nbad, W,
             o);
  }
  return JAGP_OK;
}


// ---------------------------------------------------------------------------
// Batches of independent systems: one sweep of every system captured once into
// a CUDA graph (the systems' launch sequences forked over concurrent streams),
// replayed once per sweep; the Philox sweep index comes from a device counter
// that the graph advances at its end.
// ---------------------------------------------------------------------------
}  // extern "C"

// one launch of the grouped sweep: kernel fn over the entries of table
struct GroupLaunch {
  const void *fn;
  dim3 block;
  size_t smem;
  int blocks;
  size_t tab_off;     // byte offset of the argument packs in the blob
  int lane;
  GroupTable table;
};

struct jagp_batch {
  int S = 0;
  bool grouped = false;          // one launch per kernel and point of the sweep over all systems
  void *blob = nullptr;          // device: entry tables and argument packs of the grouped launches
  std::vector<GroupLaunch> glaunch;
  int group_lanes = 1;           // concurrent chains of grouped launches
  std::vector<cudaStream_t> lane_streams;
  std::vector<cudaEvent_t> lane_events;
  std::vector<jagp_ctx *> h;
  std::vector<void *> state;
  std::vector<double *> r, eL;
  std::vector<int> W;
  std::vector<uint64_t> walker0;
  std::vector<int> order;  // systems by decreasing cost
  std::vector<int> lane;   // stream of order[q]: least-loaded stream at its turn
  double *acc = nullptr;
  uint32_t *counter = nullptr;
  std::vector<cudaStream_t> streams;
  std::vector<cudaEvent_t> ev;
  cudaEvent_t ev0 = nullptr;
  cudaStream_t cap = nullptr;  // capture stream (capture is not allowed on the legacy default stream)
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
};

namespace {
// the per-system streams: systems by decreasing cost (order), each onto the
// least-loaded of K streams at its turn, so that the streams of the graph end
// at about the same time (round robin leaves the stream with the largest
// systems about half again above the mean)
std::vector<int> batch_lanes(jagp_batch *b, int K) {
  auto cost = [&](int q) {
    const double n = b->h[q]->ds.n_up, L = b->h[q]->ds.L;
    return (double)b->W[q] * (n * L * L + n * n * L);
  };
  b->order.resize(b->S);
  for (int q = 0; q < b->S; ++q) b->order[q] = q;
  std::stable_sort(b->order.begin(), b->order.end(), [&](int a, int c) { return cost(a) > cost(c); });
  std::vector<int> lane;
  std::vector<double> load(K, 0.0);
  for (int q = 0; q < b->S; ++q) {
    int best = 0;
    for (int k = 1; k < K; ++k)
      if (load[k] < load[best]) best = k;
    lane.push_back(best);
    load[best] += cost(b->order[q]);
  }
  return lane;
}

__global__ void k_set_counter(uint32_t *c, uint32_t v) {
  if (threadIdx.x == 0) *c = v;
}

// Grouped sweep: record each system's launch sequence of one sweep (nothing
// runs; a launcher that cannot be recorded would be caught by the capture of
// the scratch stream), order all records by their point of the sweep (the
// keys set in run_sweeps / run_refresh, then the order within that point),
// and issue the records of the same kernel at the same point as one grouped
// launch.  Each system's own launches keep their order, and launches of
// different systems are independent, so every system sees exactly its
// per-system sequence.  Returns UNSUPPORTED when a sequence cannot be grouped.
jagp_status_t batch_build_grouped(jagp_batch *b) {
  cudaStream_t st = b->cap;
  std::vector<GroupRecord> all;
  for (int q = 0; q < b->S; ++q) {
    jagp_ctx *h = b->h[q];
    GroupRecorder R;
    R.sys = q;
    const int prof = h->prof_kernel;
    h->prof_kernel = 0;
    JAGP_CU(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
    set_group_recorder(&R);
    jagp_status_t rc;
    if (h->precision == JAGP_PREC_MIXED)
      rc = run_sweeps<float>(h, b->r[q], b->state[q], b->W[q], 1, b->walker0[q], 0, b->eL[q],
                             b->acc ? b->acc + 4 * (size_t)q : nullptr, st, b->counter, 1);
    else
      rc = run_sweeps<double>(h, b->r[q], b->state[q], b->W[q], 1, b->walker0[q], 0, b->eL[q],
                              b->acc ? b->acc + 4 * (size_t)q : nullptr, st, b->counter, 1);
    set_group_recorder(nullptr);
    h->prof_kernel = prof;
    cudaGraph_t g = nullptr;
    const cudaError_t e = cudaStreamEndCapture(st, &g);
    size_t nodes = 0;
    if (g) {
      cudaGraphGetNodes(g, nullptr, &nodes);
      cudaGraphDestroy(g);
    }
    if (e != cudaSuccess) {
      g_last_cuda_error = cudaGetErrorString(e);
      return JAGP_ERR_CUDA;
    }
    if (rc != JAGP_OK) return rc;
    if (nodes != 0) return JAGP_ERR_UNSUPPORTED;  // a launch that bypassed the recorder
    for (auto &r : R.recs) all.push_back(std::move(r));
  }
  // lanes: disjoint sets of systems (balanced by cost), each its own chain of
  // grouped launches on its own stream of the graph, so that the lanes' kernels overlap
  const int lanes = std::max(1, std::min(b->group_lanes, b->S));
  std::vector<int> lane_of(b->S, 0);
  if (lanes > 1) {
    const std::vector<int> ln = batch_lanes(b, lanes);
    for (int q = 0; q < b->S; ++q) lane_of[b->order[q]] = ln[q];
  }
  for (auto &r : all) r.lane = lane_of[r.sys];
  auto point_less = [](const GroupRecord &a, const GroupRecord &c) {
    if (a.lane != c.lane) return a.lane < c.lane;
    for (int i = 0; i < 5; ++i)
      if (a.key[i] != c.key[i]) return a.key[i] < c.key[i];
    return a.seq < c.seq;
  };
  // every system's sequence must advance through the points in order
  {
    std::vector<const GroupRecord *> last(b->S, nullptr);
    for (const auto &r : all) {
      if (last[r.sys] && !point_less(*last[r.sys], r)) return JAGP_ERR_UNSUPPORTED;
      last[r.sys] = &r;
    }
  }
  auto same_launch = [](const GroupRecord &a, const GroupRecord &c) {
    return a.fn == c.fn && a.block.x == c.block.x && a.block.y == c.block.y && a.block.z == c.block.z;
  };
  std::stable_sort(all.begin(), all.end(), [&](const GroupRecord &a, const GroupRecord &c) {
    if (point_less(a, c)) return true;
    if (point_less(c, a)) return false;
    if (a.fn != c.fn) return std::less<const void *>()(a.fn, c.fn);
    if (a.block.x != c.block.x) return a.block.x < c.block.x;
    return a.block.y * 1024 + a.block.z < c.block.y * 1024 + c.block.z;
  });
  // lay out the entry tables and argument packs
  std::vector<unsigned char> host;
  auto place = [&](size_t bytes, size_t align) {
    size_t off = (host.size() + align - 1) / align * align;
    host.resize(off + bytes);
    return off;
  };
  b->glaunch.clear();
  for (size_t i = 0; i < all.size();) {
    // records of one kernel at one point (at most kGroupMax per launch)
    size_t j = i + 1;
    while (j < all.size() && j - i < (size_t)kGroupMax && !point_less(all[i], all[j]) && same_launch(all[i], all[j]))
      ++j;
    GroupLaunch gl{};
    gl.fn = all[i].fn;
    gl.block = all[i].block;
    gl.lane = all[i].lane;
    gl.table.n = (int)(j - i);
    const size_t psz = all[i].args.size();
    if (psz % all[i].align) return JAGP_ERR_UNSUPPORTED;
    gl.tab_off = place((size_t)gl.table.n * psz, 256);
    long long blocks = 0;
    for (size_t k = i; k < j; ++k) {
      const GroupRecord &r = all[k];
      if (r.args.size() != psz) return JAGP_ERR_UNSUPPORTED;
      gl.table.start[k - i] = (int)blocks;
      gl.table.dims[k - i][0] = (int)r.grid.x;
      gl.table.dims[k - i][1] = (int)r.grid.y;
      gl.table.dims[k - i][2] = (int)r.grid.z;
      memcpy(host.data() + gl.tab_off + (k - i) * psz, r.args.data(), psz);
      blocks += (long long)r.grid.x * r.grid.y * r.grid.z;
      if (blocks > 0x7fffffffLL) return JAGP_ERR_UNSUPPORTED;
      gl.smem = std::max(gl.smem, r.smem);
    }
    gl.table.start[gl.table.n] = (int)blocks;
    gl.blocks = (int)blocks;
    b->glaunch.push_back(gl);
    i = j;
  }
  if (b->blob) cudaFree(b->blob);
  b->blob = nullptr;
  JAGP_CU(cudaMalloc(&b->blob, std::max<size_t>(host.size(), 256)));
  JAGP_CU(cudaMemcpy(b->blob, host.data(), host.size(), cudaMemcpyHostToDevice));
  // dynamic shared memory beyond 48 KB: the kernel's limit raised to the device's
  for (const auto &gl : b->glaunch)
    if (gl.smem > 48 * 1024) {
      std::atomic<unsigned char> done[64];
      for (auto &d : done) d.store(0, std::memory_order_relaxed);
      JAGP_CU(group_raise_smem(gl.fn, done));
    }
  // capture: each lane's grouped launches in order on its stream (forked from
  // and joined back into the capture stream), then the sweep counter
  while ((int)b->lane_streams.size() < lanes) {
    cudaStream_t s2;
    cudaEvent_t e2;
    JAGP_CU(cudaStreamCreateWithFlags(&s2, cudaStreamNonBlocking));
    b->lane_streams.push_back(s2);
    JAGP_CU(cudaEventCreateWithFlags(&e2, cudaEventDisableTiming));
    b->lane_events.push_back(e2);
  }
  JAGP_CU(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
  cudaError_t le = cudaEventRecord(b->ev0, st);
  for (int k = 0; k < lanes && le == cudaSuccess; ++k) le = cudaStreamWaitEvent(b->lane_streams[k], b->ev0, 0);
  for (auto &gl : b->glaunch) {
    if (le != cudaSuccess) break;
    void *tab = static_cast<char *>(b->blob) + gl.tab_off;
    void *args[2] = {&tab, &gl.table};
    le = cudaLaunchKernel(gl.fn, dim3(gl.blocks), gl.block, args, gl.smem, b->lane_streams[gl.lane]);
  }
  for (int k = 0; k < lanes && le == cudaSuccess; ++k) {
    le = cudaEventRecord(b->lane_events[k], b->lane_streams[k]);
    if (le == cudaSuccess) le = cudaStreamWaitEvent(st, b->lane_events[k], 0);
  }
  if (le == cudaSuccess) le = launch_increment(b->counter, 1, st);
  cudaGraph_t g = nullptr;
  const cudaError_t e = cudaStreamEndCapture(st, &g);
  if (le != cudaSuccess || e != cudaSuccess || !g) {
    g_last_cuda_error = cudaGetErrorString(le != cudaSuccess ? le : e);
    if (g) cudaGraphDestroy(g);
    return JAGP_ERR_CUDA;
  }
  b->graph = g;
  JAGP_CU(cudaGraphInstantiate(&b->exec, g, 0));
  b->grouped = true;
  return JAGP_OK;
}

jagp_status_t batch_capture(jagp_batch *b) {
  cudaStream_t st = b->cap;
  if (b->streams.empty()) {
    // grouped launches, or the per-system streams when a sequence cannot be grouped
    const jagp_status_t rc = batch_build_grouped(b);
    if (rc != JAGP_ERR_UNSUPPORTED) return rc;
    cudaGetLastError();
    const int K = std::max(1, std::min(8, b->S));
    for (int k = 0; k < K; ++k) {
      cudaStream_t s2;
      cudaEvent_t e2;
      JAGP_CU(cudaStreamCreateWithFlags(&s2, cudaStreamNonBlocking));
      b->streams.push_back(s2);
      JAGP_CU(cudaEventCreateWithFlags(&e2, cudaEventDisableTiming));
      b->ev.push_back(e2);
    }
    b->lane = batch_lanes(b, K);
  }
  JAGP_CU(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
  jagp_status_t rc = JAGP_OK;
  cudaEventRecord(b->ev0, st);
  const int K = (int)b->streams.size();
  for (int k = 0; k < K; ++k) cudaStreamWaitEvent(b->streams[k], b->ev0, 0);
  for (int q = 0; q < b->S && rc == JAGP_OK; ++q) {
    const int sidx = b->order[q];
    jagp_ctx *h = b->h[sidx];
    const int prof = h->prof_kernel;
    h->prof_kernel = 0;  // no event pairs inside a graph
    cudaStream_t ss = b->streams[b->lane[q]];
    double *acc = b->acc ? b->acc + 4 * (size_t)sidx : nullptr;
    if (h->precision == JAGP_PREC_MIXED)
      rc = run_sweeps<float>(h, b->r[sidx], b->state[sidx], b->W[sidx], 1, b->walker0[sidx], 0, b->eL[sidx], acc, ss,
                             b->counter, 1);
    else
      rc = run_sweeps<double>(h, b->r[sidx], b->state[sidx], b->W[sidx], 1, b->walker0[sidx], 0, b->eL[sidx], acc,
                              ss, b->counter, 1);
    h->prof_kernel = prof;
  }
  for (int k = 0; k < K; ++k) {
    cudaEventRecord(b->ev[k], b->streams[k]);
    cudaStreamWaitEvent(st, b->ev[k], 0);
  }
  if (rc == JAGP_OK && launch_increment(b->counter, 1, st) != cudaSuccess) rc = JAGP_ERR_CUDA;
  cudaGraph_t g = nullptr;
  const cudaError_t e = cudaStreamEndCapture(st, &g);
  if (rc != JAGP_OK || e != cudaSuccess || !g) {
    if (e != cudaSuccess) g_last_cuda_error = cudaGetErrorString(e);
    if (g) cudaGraphDestroy(g);
    return rc != JAGP_OK ? rc : JAGP_ERR_CUDA;
  }
  b->graph = g;
  JAGP_CU(cudaGraphInstantiate(&b->exec, g, 0));
  return JAGP_OK;
}
}  // namespace

extern "C" {

jagp_status_t jagp_batch_create(jagp_batch_t *out, int S, const jagp_handle_t *handles, void *const *d_states,
                                double *const *d_r, const int *W, const uint64_t *walker0, double *const *d_eL,
                                double *d_acc, int n_streams) {
  if (!out || S <= 0 || !handles || !d_states || !d_r || !W) return JAGP_ERR_INVALID_ARG;
  *out = nullptr;
  for (int q = 0; q < S; ++q) {
    const jagp_status_t s = check_walkers(handles[q], W[q], d_states[q]);
    if (s != JAGP_OK || !d_r[q]) return JAGP_ERR_INVALID_ARG;
    if (handles[q]->device != handles[0]->device) return JAGP_ERR_INVALID_ARG;
    if (walker0 && walker0[q] + (uint64_t)W[q] > 0x100000000ull) return JAGP_ERR_INVALID_ARG;
  }
  jagp_batch *b = new jagp_batch();
  b->S = S;
  for (int q = 0; q < S; ++q) {
    b->h.push_back(handles[q]);
    b->state.push_back(d_states[q]);
    b->r.push_back(d_r[q]);
    b->eL.push_back(d_eL ? d_eL[q] : nullptr);
    b->W.push_back(W[q]);
    b->walker0.push_back(walker0 ? walker0[q] : 0);
    b->order.push_back(q);
  }
  b->acc = d_acc;
  // n_streams > 0: per-system launches over that many streams; 0 or -k:
  // grouped launches in one or k lanes (the streams only as the fallback)
  const int K = n_streams > 0 ? std::max(1, std::min(n_streams, S)) : 0;
  b->group_lanes = n_streams < 0 ? -n_streams : 1;
  if (K > 0) b->lane = batch_lanes(b, K);
  bool ok = cudaMalloc(&b->counter, sizeof(uint32_t)) == cudaSuccess &&
            cudaMemset(b->counter, 0, sizeof(uint32_t)) == cudaSuccess &&
            cudaEventCreateWithFlags(&b->ev0, cudaEventDisableTiming) == cudaSuccess &&
            cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking) == cudaSuccess;
  for (int k = 0; ok && k < K; ++k) {
    cudaStream_t s2;
    cudaEvent_t e2;
    ok = cudaStreamCreateWithFlags(&s2, cudaStreamNonBlocking) == cudaSuccess &&
         cudaEventCreateWithFlags(&e2, cudaEventDisableTiming) == cudaSuccess;
    if (ok) {
      b->streams.push_back(s2);
      b->ev.push_back(e2);
    }
  }
  if (!ok) {
    jagp_batch_destroy(b);
    return JAGP_ERR_CUDA;
  }
  *out = b;
  return JAGP_OK;
}

jagp_status_t jagp_batch_sweep(jagp_batch_t b, int nsweeps, uint64_t sweep0, void *stream) {
  if (!b || nsweeps < 0 || sweep0 + (uint64_t)nsweeps > 0x100000000ull) return JAGP_ERR_INVALID_ARG;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (!b->exec) {
    const jagp_status_t rc = batch_capture(b);
    if (rc != JAGP_OK) return rc;
  }
  k_set_counter<<<1, 32, 0, st>>>(b->counter, (uint32_t)sweep0);
  JAGP_CU(cudaGetLastError());
  for (int t = 0; t < nsweeps; ++t) JAGP_CU(cudaGraphLaunch(b->exec, st));
  return JAGP_OK;
}

jagp_status_t jagp_batch_launches(jagp_batch_t b, long long *h_kernels, long long *h_nodes) {
  if (!b || !h_kernels) return JAGP_ERR_INVALID_ARG;
  *h_kernels = 0;
  if (h_nodes) *h_nodes = 0;
  if (!b->graph) return JAGP_OK;
  size_t n = 0;
  JAGP_CU(cudaGraphGetNodes(b->graph, nullptr, &n));
  std::vector<cudaGraphNode_t> nodes(n);
  JAGP_CU(cudaGraphGetNodes(b->graph, nodes.data(), &n));
  long long k = 0;
  for (size_t i = 0; i < n; ++i) {
    cudaGraphNodeType t;
    JAGP_CU(cudaGraphNodeGetType(nodes[i], &t));
    k += t == cudaGraphNodeTypeKernel;
  }
  *h_kernels = k;
  if (h_nodes) *h_nodes = (long long)n;
  return JAGP_OK;
}

jagp_status_t jagp_batch_destroy(jagp_batch_t b) {
  if (!b) return JAGP_ERR_INVALID_ARG;
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  for (auto s2 : b->streams) cudaStreamDestroy(s2);
  for (auto e2 : b->ev) cudaEventDestroy(e2);
  if (b->ev0) cudaEventDestroy(b->ev0);
  if (b->cap) cudaStreamDestroy(b->cap);
  if (b->counter) cudaFree(b->counter);
  if (b->blob) cudaFree(b->blob);
  for (auto s2 : b->lane_streams) cudaStreamDestroy(s2);
  for (auto e2 : b->lane_events) cudaEventDestroy(e2);
  delete b;
  return JAGP_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Entry points: each records a failure in the handle for jagp_last_error.
// ---------------------------------------------------------------------------
extern "C" {
jagp_status_t jagp_eval(jagp_handle_t h, const double *d_r, int W, void *d_state, double *d_logabs,
                        double *d_sign, void *stream) {
  return jagp_note(h, "jagp_eval", jagp_eval_impl(h, d_r, W, d_state, d_logabs, d_sign, stream));
}

jagp_status_t vmc_sweep(jagp_handle_t h, double *d_r, void *d_state, int W, int nsweeps, uint64_t walker0,
                        uint64_t sweep0, double *d_eL, double *d_acc, void *stream) {
  return jagp_note(h, "vmc_sweep", vmc_sweep_impl(h, d_r, d_state, W, nsweeps, walker0, sweep0, d_eL, d_acc, stream));
}

jagp_status_t local_energy(jagp_handle_t h, const double *d_r, void *d_state, int W, double *d_eL,
                           double *d_parts, void *stream) {
  return jagp_note(h, "local_energy", local_energy_impl(h, d_r, d_state, W, d_eL, d_parts, stream));
}

jagp_status_t jagp_grad(jagp_handle_t h, const double *d_r, void *d_state, int W, const double *d_seed_logpsi,
                        const double *d_seed_eL, void *d_work, double *d_eL, double *d_dlambda, double *d_djas,
                        double *d_dR, double *d_dR_walker, double *d_dr, void *stream) {
  return jagp_note(h, "jagp_grad", jagp_grad_impl(h, d_r, d_state, W, d_seed_logpsi, d_seed_eL, d_work, d_eL, d_dlambda, d_djas, d_dR, d_dR_walker, d_dr, stream));
}

jagp_status_t jagp_walker_info(jagp_handle_t h, const void *d_state, int W, double *d_logabs, double *d_sign,
                               double *d_naccept, double *d_drift, int *d_status, void *stream) {
  return jagp_note(h, "jagp_walker_info", jagp_walker_info_impl(h, d_state, W, d_logabs, d_sign, d_naccept, d_drift, d_status, stream));
}

jagp_status_t jagp_walker_status(jagp_handle_t h, const void *d_state, int W, int *h_bits, void *stream) {
  return jagp_note(h, "jagp_walker_status", jagp_walker_status_impl(h, d_state, W, h_bits, stream));
}

jagp_status_t jagp_autotune(jagp_handle_t h, void *d_state, int W, jagp_tuning_t *out, void *stream) {
  return jagp_note(h, "jagp_autotune", jagp_autotune_impl(h, d_state, W, out, stream));
}

jagp_status_t jagp_set_tuning(jagp_handle_t h, const jagp_tuning_t *t) {
  return jagp_note(h, "jagp_set_tuning", jagp_set_tuning_impl(h, t));
}

jagp_status_t jagp_profile(jagp_handle_t h, int kernel, int enable) {
  return jagp_note(h, "jagp_profile", jagp_profile_impl(h, kernel, enable));
}

jagp_status_t jagp_profile_read(jagp_handle_t h, double *h_total_ms, long long *h_launches) {
  return jagp_note(h, "jagp_profile_read", jagp_profile_read_impl(h, h_total_ms, h_launches));
}

size_t jagp_logpsi_derivs_workspace_bytes(jagp_handle_t h, int W) {
  if (!h || W <= 0 || W > h->max_walkers) return 0;
  const size_t blk = align256((size_t)W * h->ds.n_up * h->ds.L * 8);
  return 2 * blk;
}

static jagp_status_t jagp_logpsi_derivs_impl(jagp_handle_t h, const double *d_r, void *d_state, int W, void *d_work,
                                             double *d_O, long long ldo, void *stream) {
  jagp_status_t s = check_walkers(h, W, d_state);
  if (s != JAGP_OK) return s;
  if (!d_r || !d_work || !d_O || (reinterpret_cast<uintptr_t>(d_work) & 255u)) return JAGP_ERR_INVALID_ARG;
  const DevSystem &d = h->ds;
  const int n = d.n_up, nd = d.n_dn, Lb = d.L;
  const long long P = (long long)Lb * Lb + 3;
  if (ldo < P) {
    jagp_set_detail("ldo = %lld below the %lld parameters", ldo, P);
    return JAGP_ERR_INVALID_ARG;
  }
  if (h->precision != JAGP_PREC_FP64) return JAGP_ERR_UNSUPPORTED;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const Layout L = layout_of(h, W);
  const size_t blk = align256((size_t)W * n * Lb * 8);
  double *phidn = reinterpret_cast<double *>(d_work);
  double *ybuf = reinterpret_cast<double *>(static_cast<char *>(d_work) + blk);
  // orbitals of the down electrons (rows j < N_dn of each walker's block)
  LAUNCH(JAGP_KERNEL_BASIS, nd > 0, launch_basis_points<double>(d, false, d_r, W, n, nd, phidn, nullptr, nullptr, 0, 0, st));
  // Y[i][nu] = sum_{j < N_dn} Ginv[j][i] phi_nu(r_j^dn); O_lambda[mu][nu] = sum_i phi_mu(r_i^up) Y[i][nu]
  LAUNCH(0, 1,
         launch_bgemm_tn(at<double>(d_state, L.ginv), (size_t)n * n, n, phidn, (size_t)n * Lb, Lb, nd, n, Lb, ybuf,
                         (size_t)n * Lb, Lb, W, st));
  LAUNCH(0, 1,
         launch_bgemm_tn(at<double>(d_state, L.phi_up), (size_t)n * Lb, Lb, ybuf, (size_t)n * Lb, Lb, n, Lb, Lb, d_O,
                         (size_t)ldo, Lb, W, st));
  LAUNCH(0, 1, launch_sr_jastrow(d, d_r, d_O, ldo, (long long)Lb * Lb, W, st));
  return JAGP_OK;
}

size_t jagp_sr_workspace_bytes(int M, int P) {
  if (M <= 0 || P <= 0) return 0;
  return sr_layout(M, P).total * sizeof(double);
}

jagp_status_t jagp_sr_step(const double *d_O, long long ldo, const double *d_eL, int M, int P, double eps,
                           double delta, int max_iter, double tol, void *d_work, double *d_f, double *d_dalpha,
                           int *h_iters, double *h_resid, void *stream) {
  if (!d_O || !d_eL || !d_work || !d_f || !d_dalpha || M < 2 || P < 1 || ldo < P || max_iter < 0 || !(eps >= 0.0) ||
      !(tol >= 0.0) || (reinterpret_cast<uintptr_t>(d_work) & 255u))
    return JAGP_ERR_INVALID_ARG;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const SrLayout L = sr_layout(M, P);
  double *w = static_cast<double *>(d_work);
  JAGP_CU(sr_prepare(d_O, ldo, d_eL, M, P, w, L, d_f, st));
  JAGP_CU(sr_cg_init(d_f, eps, P, w, L, st));
  double rr0 = 0.0, rr = 0.0;
  JAGP_CU(cudaMemcpyAsync(&rr0, w + L.sc + 3, sizeof(double), cudaMemcpyDeviceToHost, st));
  JAGP_CU(cudaStreamSynchronize(st));
  rr = rr0;
  int it = 0;
  while (it < max_iter && rr > tol * tol * rr0 && rr > 0.0) {
    JAGP_CU(sr_cg_iter(d_O, ldo, M, P, eps, w, L, st));
    JAGP_CU(cudaMemcpyAsync(&rr, w + L.sc + 3, sizeof(double), cudaMemcpyDeviceToHost, st));
    JAGP_CU(cudaStreamSynchronize(st));
    ++it;
  }
  JAGP_CU(sr_finish(delta, P, w, L, d_dalpha, st));
  if (h_iters) *h_iters = it;
  if (h_resid) *h_resid = rr0 > 0.0 ? sqrt(rr / rr0) : 0.0;
  return JAGP_OK;
}

int jagp_reblock_levels(int T) { return T >= 1 ? reblock_levels(T) : 0; }

jagp_status_t jagp_reblock(const double *d_eL, int T, int W, double *d_work, double *d_levels, double *d_stats,
                           void *stream) {
  if (!d_eL || !d_work || !d_stats || T <= 0 || W <= 0) return JAGP_ERR_INVALID_ARG;
  if (reblock_levels(T) > 0 && !d_levels) return JAGP_ERR_INVALID_ARG;
  JAGP_CU(launch_reblock(d_eL, T, W, d_work, d_levels, d_stats, static_cast<cudaStream_t>(stream)));
  return JAGP_OK;
}

static jagp_status_t jagp_space_warp_impl(jagp_handle_t h, const double *d_r, int W, const double *d_rbar,
                                          const double *d_seed_logpsi, double *d_dR_walker, double *d_dR,
                                          void *stream) {
  if (!h || W <= 0 || W > h->max_walkers || !d_r || !d_rbar || !d_dR_walker) return JAGP_ERR_INVALID_ARG;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  LAUNCH(0, 1 + (d_dR != nullptr), launch_space_warp(h->ds, d_r, d_rbar, d_seed_logpsi, d_dR_walker, d_dR, W, st));
  return JAGP_OK;
}

static jagp_status_t jagp_guiding_weights_impl(jagp_handle_t h, void *d_state, int W, double theta, double eps,
                                               double *d_R, double *d_W, void *stream) {
  jagp_status_t s = check_walkers(h, W, d_state);
  if (s != JAGP_OK) return s;
  if (!(theta > 0.0) || !(eps >= 0.0) || (!d_R && !d_W)) return JAGP_ERR_INVALID_ARG;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const Layout L = layout_of(h, W);
  const int n = h->ds.n_up, Lb = h->ds.L;
  double *gm = refresh_g(L, d_state);
  // G~ = Phi_up Bt^T from the current tables (FP64, or compensated from the two-float tables)
  if (h->precision == JAGP_PREC_MIXED) {
    LAUNCH(0, 1,
           refresh_geminal(at<float>(d_state, L.phi_up), lo_table(h, d_state, L.phi_lo), (size_t)n * Lb,
                           at<float>(d_state, L.bt), lo_table(h, d_state, L.bt_lo), (size_t)n * Lb, n, Lb, gm, W, st,
                           -1));
    LAUNCH(0, 1, launch_guiding<float>(gm, at<float>(d_state, L.ginv), n, W, theta, eps, d_R, d_W, st));
  } else {
    LAUNCH(0, 1,
           refresh_geminal(at<double>(d_state, L.phi_up), nullptr, (size_t)n * Lb, at<double>(d_state, L.bt), nullptr,
                           (size_t)n * Lb, n, Lb, gm, W, st, -1));
    LAUNCH(0, 1, launch_guiding<double>(gm, at<double>(d_state, L.ginv), n, W, theta, eps, d_R, d_W, st));
  }
  return JAGP_OK;
}

jagp_status_t jagp_set_guiding(jagp_handle_t h, double theta, double eps) {
  if (!h) return JAGP_ERR_INVALID_ARG;
  if (!(theta > 0.0) || !(eps >= 0.0) || !std::isfinite(eps)) {
    jagp_set_detail("theta = %g, eps = %g (theta > 0, eps >= 0)", theta, eps);
    return jagp_note(h, "jagp_set_guiding", JAGP_ERR_INVALID_ARG);
  }
  if (eps > 0.0 && (h->precision != JAGP_PREC_FP64 || h->ds.n_up > kGuidedMaxUp || h->ds.use_j3)) {
    jagp_set_detail("guided sampling needs an FP64 handle with N_up <= %d and no three-body Jastrow", kGuidedMaxUp);
    return jagp_note(h, "jagp_set_guiding", JAGP_ERR_UNSUPPORTED);
  }
  h->guide_theta = theta;
  h->guide_eps = eps;
  return JAGP_OK;
}

jagp_status_t jagp_space_warp(jagp_handle_t h, const double *d_r, int W, const double *d_rbar,
                              const double *d_seed_logpsi, double *d_dR_walker, double *d_dR, void *stream) {
  return jagp_note(h, "jagp_space_warp",
                   jagp_space_warp_impl(h, d_r, W, d_rbar, d_seed_logpsi, d_dR_walker, d_dR, stream));
}

jagp_status_t jagp_guiding_weights(jagp_handle_t h, void *d_state, int W, double theta, double eps, double *d_R,
                                   double *d_W, void *stream) {
  return jagp_note(h, "jagp_guiding_weights", jagp_guiding_weights_impl(h, d_state, W, theta, eps, d_R, d_W, stream));
}

jagp_status_t jagp_force_seeds(const double *d_eL, const double *d_weight, int M, double *d_seed_logpsi,
                               double *d_seed_eL, double *d_mean, void *stream) {
  if (!d_eL || M <= 0 || !d_seed_logpsi || !d_seed_eL) return JAGP_ERR_INVALID_ARG;
  JAGP_CU(launch_force_seeds(d_eL, d_weight, M, d_seed_logpsi, d_seed_eL, d_mean, static_cast<cudaStream_t>(stream)));
  return JAGP_OK;
}

jagp_status_t jagp_logpsi_derivs(jagp_handle_t h, const double *d_r, void *d_state, int W, void *d_work, double *d_O,
                                 long long ldo, void *stream) {
  return jagp_note(h, "jagp_logpsi_derivs", jagp_logpsi_derivs_impl(h, d_r, d_state, W, d_work, d_O, ldo, stream));
}

jagp_status_t jagp_last_error(jagp_handle_t h, char *buf, size_t len) {
  if (!h) return JAGP_ERR_INVALID_ARG;
  if (buf && len > 0) snprintf(buf, len, "%s", h->last_error);
  return h->last_status;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Lattice-regularised diffusion Monte Carlo (Sec. "Lattice regularized Monte
// Carlo"): the round loop of a projection and the reconfiguration.
// ---------------------------------------------------------------------------
namespace {

LrdmcWork lrdmc_work(const jagp_ctx *h, int W, void *base, size_t *total) {
  const size_t w = (size_t)W, N = h->ds.N;
  size_t o = 0;
  auto take = [&](size_t bytes) { size_t r = o; o = align256(o + bytes); return r; };
  const size_t left = take(w * 8), lw = take(w * 8), eL = take(w * 8), rho = take(w * 6 * N * 8),
               rt = take(w * N * 3 * 8), hops = take(w * 4), flags = take(w * 4), active = take(w * 4),
               moved = take(w * 4), lu = take(w * 4), ld = take(w * 4), lwk = take(w * 4), cnt = take(16),
               rs = take(w * N * 3 * 8), es = take(w * 8), ss = take(layout_of(h, W).total);
  if (total) *total = o;
  LrdmcWork k;
  char *b = static_cast<char *>(base);
  k.left = reinterpret_cast<double *>(b + left);
  k.lw = reinterpret_cast<double *>(b + lw);
  k.eL = reinterpret_cast<double *>(b + eL);
  k.rho = reinterpret_cast<double *>(b + rho);
  k.r_tmp = reinterpret_cast<double *>(b + rt);
  k.hops = reinterpret_cast<int *>(b + hops);
  k.flags = reinterpret_cast<int *>(b + flags);
  k.active = reinterpret_cast<int *>(b + active);
  k.moved = reinterpret_cast<int *>(b + moved);
  k.list_up = reinterpret_cast<int *>(b + lu);
  k.list_dn = reinterpret_cast<int *>(b + ld);
  k.list_w = reinterpret_cast<int *>(b + lwk);
  k.cnt = reinterpret_cast<int *>(b + cnt);
  k.r_sub = reinterpret_cast<double *>(b + rs);
  k.eL_sub = reinterpret_cast<double *>(b + es);
  k.sub_state = b + ss;
  return k;
}

jagp_status_t lrdmc_project(jagp_ctx *h, double *d_r, void *d_state, int W, uint64_t walker0, uint64_t gen,
                            double a, double gamma, double tau, double e_ref, int max_hops, double *d_weight,
                            double *d_eL, int *d_hops, int *d_flags, void *d_work, cudaStream_t st) {
  const Layout L = layout_of(h, W);
  const DevSystem &d = h->ds;
  LrdmcWork k = lrdmc_work(h, W, d_work, nullptr);
  double *phi_up = at<double>(d_state, L.phi_up), *pprop = at<double>(d_state, L.pprop);
  int *status = at<int>(d_state, L.status);
  // the walkers' tables, G~^{-1}, e_L and the kinetic vectors M at the start
  jagp_status_t s = run_eval<double>(h, d_r, W, d_state, nullptr, nullptr, st);
  if (s != JAGP_OK) return s;
  s = run_local_energy<double>(h, d_r, d_state, W, k.eL, nullptr, st);
  if (s != JAGP_OK) return s;
  LAUNCH(0, 1, launch_lrdmc_start(status, W, tau, k, st));
  for (;;) {
    JAGP_CU(cudaMemsetAsync(k.cnt, 0, 4 * sizeof(int), st));
    LAUNCH(JAGP_KERNEL_BASIS, 1, launch_lrdmc_ratios(d, d_r, at<double>(d_state, L.mbuf), k.active, a, k.rho, W, st));
    LAUNCH(JAGP_KERNEL_METROPOLIS, 1,
           launch_lrdmc_decide(d, d_r, k.eL, status, W, (uint32_t)walker0, (uint32_t)gen, a, gamma, e_ref, max_hops,
                               k, st));
    int h_cnt[4] = {0, 0, 0, 0};
    JAGP_CU(cudaMemcpyAsync(h_cnt, k.cnt, sizeof(h_cnt), cudaMemcpyDeviceToHost, st));
    JAGP_CU(cudaStreamSynchronize(st));
    if (h_cnt[2] == 0) break;
    // the moved electrons' orbital rows, their lambda products, G~^{-1}, J, e_L and M
    LAUNCH(JAGP_KERNEL_BASIS, 1, launch_lrdmc_rows(d, d_r, k.moved, pprop, phi_up, W, st));
    if (h_cnt[0] > 0) {
      s = lambda_products(h, pprop, nullptr, at<double>(d_state, L.a_up), true, k.list_up, k.cnt, 0, 1, 0, h_cnt[0],
                          d_state, W, st);
      if (s != JAGP_OK) return s;
    }
    if (h_cnt[1] > 0) {
      s = lambda_products(h, pprop, nullptr, at<double>(d_state, L.bt), false, k.list_dn, k.cnt + 1, 0, 1, 0,
                          h_cnt[1], d_state, W, st);
      if (s != JAGP_OK) return s;
    }
    // only the moved walkers changed: their tables and positions into a
    // compact state, G~^{-1}, J, e_L and M there, and back
    const int Wc = h_cnt[2];
    const Layout C = layout_of(h, Wc);
    const size_t n = d.n_up, Lb = d.L, N = d.N;
    WalkerCopies in{};
    in.c[0] = {phi_up, at<double>(k.sub_state, C.phi_up), n * Lb * 8};
    in.c[1] = {at<double>(d_state, L.a_up), at<double>(k.sub_state, C.a_up), n * Lb * 8};
    in.c[2] = {at<double>(d_state, L.bt), at<double>(k.sub_state, C.bt), n * Lb * 8};
    in.c[3] = {d_r, k.r_sub, N * 3 * 8};
    in.c[4] = {at<double>(d_state, L.scal), at<double>(k.sub_state, C.scal), (size_t)S_STRIDE * 8};
    in.c[5] = {status, at<int>(k.sub_state, C.status), 4};
    in.n = 6;
    LAUNCH(0, 1, launch_walker_copy(in, k.list_w, Wc, false, st));
    s = run_refresh<double>(h, k.r_sub, k.sub_state, Wc, 0, true, st);
    if (s != JAGP_OK) return s;
    s = run_local_energy<double>(h, k.r_sub, k.sub_state, Wc, k.eL_sub, nullptr, st);
    if (s != JAGP_OK) return s;
    WalkerCopies out{};
    out.c[0] = {at<double>(k.sub_state, C.ginv), at<double>(d_state, L.ginv), n * n * 8};
    out.c[1] = {at<double>(k.sub_state, C.scal), at<double>(d_state, L.scal), (size_t)S_STRIDE * 8};
    out.c[2] = {at<int>(k.sub_state, C.status), status, 4};
    out.c[3] = {at<double>(k.sub_state, C.mbuf), at<double>(d_state, L.mbuf), N * Lb * 8};
    out.c[4] = {at<double>(k.sub_state, C.kin), at<double>(d_state, L.kin), N * 4 * 8};
    out.c[5] = {k.eL_sub, k.eL, 8};
    out.n = 6;
    LAUNCH(0, 1, launch_walker_copy(out, k.list_w, Wc, true, st));
  }
  LAUNCH(0, 1, launch_lrdmc_finish(W, k.lw, k.eL, d_weight, d_eL, st));
  if (d_hops) JAGP_CU(cudaMemcpyAsync(d_hops, k.hops, (size_t)W * sizeof(int), cudaMemcpyDeviceToDevice, st));
  if (d_flags) JAGP_CU(cudaMemcpyAsync(d_flags, k.flags, (size_t)W * sizeof(int), cudaMemcpyDeviceToDevice, st));
  return JAGP_OK;
}

}  // namespace

extern "C" {

size_t jagp_lrdmc_workspace_bytes(jagp_handle_t h, int W) {
  if (!h || W <= 0) return 0;
  size_t total = 0;
  lrdmc_work(h, W, nullptr, &total);
  return total;
}

static jagp_status_t jagp_lrdmc_project_impl(jagp_handle_t h, double *d_r, void *d_state, int W, uint64_t walker0,
                                             uint64_t generation, double a, double gamma, double tau, double e_ref,
                                             int max_hops, double *d_weight, double *d_eL, int *d_hops, int *d_flags,
                                             void *d_work, void *stream) {
  jagp_status_t s = check_walkers(h, W, d_state);
  if (s != JAGP_OK) return s;
  if (!d_r || !d_weight || !d_work || (reinterpret_cast<uintptr_t>(d_work) & 255u)) {
    jagp_set_detail("positions, weights or an aligned workspace missing");
    return JAGP_ERR_INVALID_ARG;
  }
  if (!(a > 0.0) || !std::isfinite(a) || !(gamma >= 0.0) || !std::isfinite(gamma) || !(tau >= 0.0) ||
      !std::isfinite(tau) || !std::isfinite(e_ref) || max_hops < 0) {
    jagp_set_detail("a = %g, gamma = %g, tau = %g, e_ref = %g, max_hops = %d", a, gamma, tau, e_ref, max_hops);
    return JAGP_ERR_INVALID_ARG;
  }
  if (h->precision != JAGP_PREC_FP64 || h->ds.use_j3) {
    jagp_set_detail("lattice-regularised DMC runs on FP64 handles without the three-body Jastrow");
    return JAGP_ERR_UNSUPPORTED;
  }
  if ((size_t)h->ds.N * 3 * 16 > 48 * 1024) {
    jagp_set_detail("N = %d: the hop-ratio kernel keeps a walker's positions (FP64 and double-word) in 48 KB of "
                    "shared memory (N <= 1024)", h->ds.N);
    return JAGP_ERR_UNSUPPORTED;
  }
  return lrdmc_project(h, d_r, d_state, W, walker0, generation, a, gamma, tau, e_ref, max_hops, d_weight, d_eL,
                       d_hops, d_flags, d_work, static_cast<cudaStream_t>(stream));
}

jagp_status_t jagp_lrdmc_project(jagp_handle_t h, double *d_r, void *d_state, int W, uint64_t walker0,
                                 uint64_t generation, double a, double gamma, double tau, double e_ref, int max_hops,
                                 double *d_weight, double *d_eL, int *d_hops, int *d_flags, void *d_work,
                                 void *stream) {
  return jagp_note(h, "jagp_lrdmc_project",
                   jagp_lrdmc_project_impl(h, d_r, d_state, W, walker0, generation, a, gamma, tau, e_ref, max_hops,
                                           d_weight, d_eL, d_hops, d_flags, d_work, stream));
}

static jagp_status_t jagp_lrdmc_branch_impl(jagp_handle_t h, double *d_r, int W, uint64_t generation,
                                            double *d_weight, const double *d_eL, int *d_parent, double *d_stats,
                                            void *d_work, void *stream) {
  if (!h) return JAGP_ERR_INVALID_ARG;
  if (W <= 0 || W > h->max_walkers || !d_r || !d_weight || !d_eL || !d_stats || !d_work ||
      (reinterpret_cast<uintptr_t>(d_work) & 255u)) {
    jagp_set_detail("W = %d (1..%d), positions, weights, energies, stats and an aligned workspace needed", W,
                    h->max_walkers);
    return JAGP_ERR_INVALID_ARG;
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  LrdmcWork k = lrdmc_work(h, W, d_work, nullptr);
  const size_t bytes = (size_t)W * h->ds.N * 3 * sizeof(double);
  JAGP_CU(cudaMemcpyAsync(k.r_tmp, d_r, bytes, cudaMemcpyDeviceToDevice, st));
  LAUNCH(0, 2,
         launch_lrdmc_branch(W, h->ds.N, (uint32_t)generation, h->ds.key0, h->ds.key1, d_weight, d_eL,
                             d_parent ? d_parent : k.moved, d_stats, k.r_tmp, d_r, st));
  return JAGP_OK;
}

jagp_status_t jagp_lrdmc_branch(jagp_handle_t h, double *d_r, int W, uint64_t generation, double *d_weight,
                                const double *d_eL, int *d_parent, double *d_stats, void *d_work, void *stream) {
  return jagp_note(h, "jagp_lrdmc_branch",
                   jagp_lrdmc_branch_impl(h, d_r, W, generation, d_weight, d_eL, d_parent, d_stats, d_work, stream));
}

jagp_status_t jagp_lrdmc_energy(const double *d_wbar, const double *d_ebar, int T, int p, double *d_E, void *stream) {
  if (!d_wbar || !d_ebar || !d_E || T <= 0 || p < 0 || p >= T) return JAGP_ERR_INVALID_ARG;
  JAGP_CU(launch_lrdmc_energy(d_wbar, d_ebar, T, p, d_E, static_cast<cudaStream_t>(stream)));
  return JAGP_OK;
}

}  // extern "C"
