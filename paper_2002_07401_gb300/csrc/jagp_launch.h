// jagp_launch.h -- host-side launchers of the libjagp kernels (internal).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "jagp_common.cuh"

namespace jagp {

// Orbital values at electron positions (PROPOSE = false) or at freshly drawn
// proposals (PROPOSE = true, also writes rprop).  Rows go to
// out[(w * n_up + i) * L], i < npts, for electrons e0 .. e0 + npts - 1; in the
// FP32 path out_lo (same layout, may be null) gets the low parts.
template <typename T>
cudaError_t launch_basis_points(const DevSystem &s, bool propose, const double *r, int W, int e0,
                                int npts, T *out, float *out_lo, double *rprop, uint32_t walker0,
                                uint32_t sweep, cudaStream_t st, const uint32_t *sweep_dev = nullptr);

// Sequential Metropolis over one spin species with Sherman-Morrison updates,
// moves m_begin .. m_end - 1 of the half-sweep (m_end < 0: to the last).
// Accepted moves are appended to list (*count) and counted in *total (when
// given); accepted up moves copy their proposal row of pprop (and pprop_lo,
// when given) into phi_up (phi_lo).
template <typename T>
cudaError_t launch_metropolis(const DevSystem &s, bool up, double *r, const double *rprop, const T *gprop,
                              T *ginv, double *scal, int *status, const T *pprop, T *phi_up, int *list,
                              int *count, int W, cudaStream_t st, const float *pprop_lo = nullptr,
                              float *phi_lo = nullptr, int m_begin = 0, int m_end = -1, int *total = nullptr,
                              double *j3buf = nullptr);

// The Metropolis half-sweep (FP64, N_up <= kGuidedMaxUp) sampling the guiding
// function: acceptance |Psi_T'/Psi_T|^2 W / W', W = (R / max(R, eps))^2; gmat
// ([W][n][n], in/out) holds G~ of the current configurations.
cudaError_t launch_metropolis_guided(const DevSystem &s, bool up, double *r, const double *rprop,
                                     const double *gprop, double *ginv, double *scal, int *status,
                                     const double *pprop, double *phi_up, int *list, int *count, double *gmat,
                                     double theta, double eps, int W, cudaStream_t st, int m_begin, int m_end,
                                     int *total);

// Out[w][a][b] = sum_k X[w][a][k] Y[w][b][k]  (a < ma, b < nb, k < K); row stride K.
// tile: -1 picks by shape, 0 one output per thread (16 x 16 tiles), 32 or 64
// register-blocked tiles (the autotuner's choice)
template <typename T>
cudaError_t launch_gemm_rows(const T *X, size_t xw, const T *Y, size_t yw, int ma, int nb, int K, T *Out,
                             size_t ow, int ldo, int W, cudaStream_t st, int tile = -1);

// FP32 variant with a compensated (error-free transformation) dot product; X and
// Y may carry low parts Xlo, Ylo (same layouts) so that they are two-float operands
cudaError_t launch_gemm_rows_dot2(const float *X, const float *Xlo, size_t xw, const float *Y, const float *Ylo,
                                  size_t yw, int ma, int nb, int K, double *Out, size_t ow, int ldo, int W,
                                  cudaStream_t st, int tile = -1);
// low parts of the unpaired-orbital rows of Bt (two-float table of the FP32 path)
cudaError_t launch_fill_unpaired_lo(const DevSystem &s, float *bt_lo, int W, cudaStream_t st);

// Out[row] = P[row] * Lam (L x L).  Rows are list[0 .. *count) when list is
// given, else rows r < nrows mapped to (r / nsub) * stride + r % nsub.
cudaError_t launch_lambda_rows(const double *P, const double *Lam, double *Out, const int *list,
                               const int *count, int nrows, int nsub, int stride, int L,
                               int max_rows, cudaStream_t st);

// Fill rows n_dn .. n_up - 1 of every walker's Bt block with the unpaired orbitals.
template <typename T>
cudaError_t launch_fill_unpaired(const DevSystem &s, T *bt, int W, cudaStream_t st);

// Gauss-Jordan inverse with partial pivoting of G~ (in gm), log|det|, sign and
// the Sherman-Morrison drift against the inverse held in ginv; ginv64 (or
// null) also receives the inverse in FP64 (the mixed path's local energy)
template <typename T>
cudaError_t launch_refresh_inverse(double *gm, T *ginv, double *scal, int *status, int n, int W,
                                   int check_drift, double drift_tol, cudaStream_t st, double *ginv64 = nullptr);

// J = J1 + J2 (+ J3 from the walker's j3 vectors j3buf [W][6][LJ], when the system has it)
cudaError_t launch_jastrow_full(const DevSystem &s, const double *r, double *scal, int W,
                                cudaStream_t st, const double *j3buf = nullptr);
// the three-body Jastrow's per-walker vectors (U_s and M U_s, see j3.cuh) from the positions
cudaError_t launch_j3_prep(const DevSystem &s, const double *r, double *buf, int W, cudaStream_t st);

// M vectors of the kinetic energy (see k_linalg.cu), then the orbital
// derivative contractions and the final per-walker local energy.
template <typename T>
cudaError_t launch_mmat(const DevSystem &s, const T *ginv, const T *bt, const T *a_up, T *mbuf, int W,
                        cudaStream_t st);
template <typename T>
cudaError_t launch_kinetic(const DevSystem &s, const double *r, const T *mbuf, double *kin, int W,
                           cudaStream_t st);
// the mixed path's two-float M vectors on the CUDA cores (small N_up): compensated
// sums of the FP64 inverse against the two-float Bt / A_up tables
cudaError_t launch_mmat_dw(const DevSystem &s, const double *ginv64, const float *bt, const float *bt_lo,
                           const float *a_up, const float *a_lo, float *mbuf, float *mlo, int W, cudaStream_t st);
// the mixed path's contraction with two-float M vectors, in double-word arithmetic
cudaError_t launch_kinetic_m2(const DevSystem &s, const double *r, const float *mbuf, const float *mlo, double *kin,
                              int W, cudaStream_t st);
cudaError_t launch_elocal(const DevSystem &s, const double *r, const double *kin, double *eL,
                          double *parts, int W, cudaStream_t st, double *scal = nullptr,
                          const double *j3buf = nullptr);
// the FP32 path's version (double-word distances, Coulomb sums and Jastrow values)
cudaError_t launch_elocal_dw(const DevSystem &s, const double *r, const double *kin, double *eL,
                             double *parts, int W, cudaStream_t st, double *scal = nullptr,
                             const double *j3buf = nullptr);

// zero the per-walker counters; status = JAGP_WS_NONFINITE for a walker with a
// non-finite coordinate in r [W][N][3] (when r is given), else 0
cudaError_t launch_walker_init(double *scal, int *status, int W, cudaStream_t st, const double *r = nullptr,
                               int N = 0);
cudaError_t launch_logpsi_out(const double *scal, int W, double *logabs, double *sign,
                              cudaStream_t st);
cudaError_t launch_walker_info(const double *scal, const int *status, int W, double *logabs,
                               double *sign, double *nacc, double *drift, int *st_out,
                               cudaStream_t st);
cudaError_t launch_reduce_acc(const double *eL, const double *scal, const int *count, int W,
                              double *acc, cudaStream_t st, int accumulate = 0);
// *c += by (one thread): advances a device-side sweep counter between graph replays
cudaError_t launch_increment(uint32_t *c, uint32_t by, cudaStream_t st);

// Tensor-core contraction (k_umma.cu):
//   out[out_rows[m]][c] = sum_p sum_k A[m][pair_a[p] kp + k] B[c][pair_b[p] kp + k]
// (batched: A is `batches` stacked blocks of batch_rows rows, B of b_batch_rows
// rows (default batch_rows), block b of A against block b of B, c < n <=
// b_batch_rows; out rows as A's, or with o_cstride != 0 the element of local row
// r and column c of block b at out[b o_bstride + r o_rstride + c o_cstride])
// A: BF16 [m_max][a_terms kp], B: BF16 [n][b_terms kp] (kp % 64 == 0, 16-byte
// aligned bases); rows m < *m_dev (or m_max) are written; out FP32, pitch ldo.
// With a_exp/b_exp (row / column exponents) the terms are fixed-point slices and
// pairs of equal a + b share an exact accumulator (see k_umma.cu).
// stages_max: pipeline depth (0: as many as fit); -1, -2, -3: chunk-major stages (K chunks of 64, 32, 16).
int umma_pick_bn(int n, int max_bn);
cudaError_t launch_umma_gemm(const uint16_t *A, int m_max, const int *m_dev, int a_terms, const uint16_t *B, int n,
                             int b_terms, int kp, int npairs, const int *pair_a, const int *pair_b, float *out,
                             long long ldo, const int *out_rows, int *err, cudaStream_t st,
                             const int *a_exp = nullptr, const int *b_exp = nullptr, float *out_lo = nullptr,
                             int bn_max = 0, double *out64 = nullptr, int slice_bits = 8, int batch_rows = 0,
                             int batches = 0, int stages_max = 0, int b_batch_rows = 0, long long o_bstride = 0,
                             long long o_rstride = 0, long long o_cstride = 0, const int *pair_group = nullptr);
// whether two chunk-major stages (stages_max = -1, -2, -3: K chunks of 64, 32,
// 16) of these pairs fit at tile width bn
bool umma_chunk_fits(int npairs, const int *pair_a, const int *pair_b, int bn, int stages_max);
// FP64 rows -> nsl exact slices of `bits` bits per element plus a row exponent;
// rows_out[m] = the source row, or (dst_stride > 0) (m / nsub) dst_stride + dst_off + m % nsub
cudaError_t launch_pack_fixed64(const double *P, const int *list, const int *count, int nrows, int nsub, int stride,
                                int L, int kp, int nsl, int bits, uint16_t *A, int *rows_out, int *exps,
                                int max_rows, cudaStream_t st, long dst_stride = 0, long dst_off = 0);
// columns c < C of the per-walker matrices X_w ([R][C], X_w = X + w xw; FP64 X64,
// or two-float X32 + Xlo) -> operand rows w C + c of nsl exact slices of
// `bits` bits (8, or 7 for FP64 X; nsl <= 8) over the R rows (K padded to kp),
// exponents exps[w C + c], and rows_out[w C + c] = w dst_stride + dst_off + c
// (when given)
cudaError_t launch_pack_cols(const double *X64, const float *X32, const float *Xlo, size_t xw, int R, int C, int kp,
                             int W, uint16_t *A, int *exps, int *rows_out, long dst_stride, long dst_off,
                             cudaStream_t st, int nsl = kFixedSlices, int bits = 8);
// FP32 rows (two-float rows P + P_lo when P_lo is given) -> kFixedSlices exact
// 8-bit slices per element (BF16) plus a row exponent
cudaError_t launch_pack_fixed(const float *P, const float *P_lo, const int *list, const int *count, int nrows,
                               int nsub, int stride, int L, int kp, uint16_t *A, int *rows_out, int *exps,
                               int max_rows, cudaStream_t st);
cudaError_t setup_umma_attributes();

// Reverse-mode derivatives (k_adjoint.cu); see that file for the formulas.
cudaError_t launch_adj_kvec(const DevSystem &s, const double *r, const double *sE, double *jg, double *kbar,
                            double *dnphi, int W, cudaStream_t st);
cudaError_t launch_adj_gbar(const double *ginv, const double *h1, const double *h2, const double *sL, int n, int nd,
                            double *gbar, int W, cudaStream_t st);
cudaError_t launch_adj_rows(const DevSystem &s, const double *ginv, const double *gbar, const double *phi_up,
                            const double *bt, const double *kbar, double *btbar, double *abar, double *phibar, int W,
                            cudaStream_t st);
// steps 2 and 3 as per-walker GEMMs for N_up too large for shared-memory staging
// (h1, h2 are overwritten; gbarT receives Gbar transposed)
cudaError_t launch_adj_rows_gemm(const DevSystem &s, const double *ginv, double *h1, double *h2, const double *sL,
                                 const double *phi_up, const double *bt, const double *kbar, double *gbarT,
                                 double *btbar, double *abar, double *phibar, int W, cudaStream_t st);
int adj_position_parts(const DevSystem &s);
cudaError_t launch_adj_positions(const DevSystem &s, const double *r, const double *sE, const double *jg,
                                 const double *mbuf, const double *phibar_a, const double *phibar_b,
                                 const double *phibar_dn, const int *shell_atom, double *rbar, double *part, int W,
                                 cudaStream_t st);
cudaError_t launch_adj_jastrow(const DevSystem &s, const double *r, const double *sL, const double *sE,
                               const double *jg, const double *kin, double *rbar, double *rbar_at, double *jpar, int W,
                               cudaStream_t st);
cudaError_t launch_adj_reduce(const double *part, int nparts, int n_atoms, double *rbar_at, const double *jpar,
                              int W, double *dR, double *djas, cudaStream_t st);
cudaError_t launch_adj_lambda(const double *btbar, const double *dnphi, const double *phi_up, const double *abar,
                              int W, int n, int nd, int L, double *part, int nz, double *dlam, cudaStream_t st);
// dlam[i] = sum_{z < nz} part[z][i] (fixed order), i < L^2
cudaError_t launch_adj_lambda_sum(const double *part, int nz, int L, double *dlam, cudaStream_t st);
cudaError_t setup_adjoint_attributes();

// Reblocking (k_stats.cu): walker means per sweep of eL [T][W] into work [T],
// then every level's (block size, blocks, sigma, error of sigma) into levels
// [reblock_levels(T)][4] and (mean, chosen sigma, chosen level, plateau) into stats [4]
int reblock_levels(int T);
cudaError_t launch_reblock(const double *eL, int T, int W, double *work, double *levels, double *stats,
                           cudaStream_t st);

// Stochastic reconfiguration (k_sr.cu).
// Out[w][a][b] = sum_{k < K} X[w][k][a] Y[w][k][b] (per-walker FP64 products
// with a shared leading index; row pitches ldx, ldy, ldo; walker strides xw, yw, ow)
cudaError_t launch_bgemm_tn(const double *X, size_t xw, int ldx, const double *Y, size_t yw, int ldy, int K, int Ma,
                            int Nb, double *Out, size_t ow, long long ldo, int W, cudaStream_t st);
// d ln|Psi| / d (b_ea, b_para, b_anti) per walker into O[w][off + 0..2]
cudaError_t launch_sr_jastrow(const DevSystem &s, const double *r, double *O, long long ldo, long long off, int W,
                              cudaStream_t st);
// workspace of the SR solve (offsets in doubles)
struct SrLayout {
  size_t obar, diag, dinv, x, r, z, p, q, u, part, ec, t, sc, total;
};
SrLayout sr_layout(int M, int P);
// Obar, diag S and f = -(2/M) sum_i (e_i - ebar)(O_i - Obar) from the samples
cudaError_t sr_prepare(const double *O, long long ldo, const double *e, int M, int P, double *w, const SrLayout &L,
                       double *f, cudaStream_t st);
// preconditioned CG on (S + eps diag S) x = f: start (x = 0), one iteration
// (device scalars at w + L.sc: [0] r.z, [3] r.r), and dalpha = delta x
cudaError_t sr_cg_init(const double *f, double eps, int P, double *w, const SrLayout &L, cudaStream_t st);
cudaError_t sr_cg_iter(const double *O, long long ldo, int M, int P, double eps, double *w, const SrLayout &L,
                       cudaStream_t st);
cudaError_t sr_finish(double delta, int P, const double *w, const SrLayout &L, double *dalpha, cudaStream_t st);

// Finite-variance forces (k_forces.cu).
// rbar_at[w][a] += sum_i omega_a(r_i) rbar[w][i] + sL_w / 2 sum_i grad omega_a(r_i) (the space
// warp); dR (or null) = sum_w rbar_at[w]
cudaError_t launch_space_warp(const DevSystem &s, const double *r, const double *rbar, const double *sL,
                              double *rbar_at, double *dR, int W, cudaStream_t st);
// R = (min_i sum_j G_ij^2 sum_jk Ginv_jk^2)^-theta and W = (R / max(R, eps))^2 per walker
template <typename T>
cudaError_t launch_guiding(const double *g, const T *ginv, int n, int W, double theta, double eps, double *R,
                           double *Wt, cudaStream_t st);
// sE = u / sum u, sL = 2 u (e - E) / sum u, E = sum u e / sum u; mean_out = (E, mean u)
cudaError_t launch_force_seeds(const double *e, const double *u, int M, double *sL, double *sE, double *mean_out,
                               cudaStream_t st);
cudaError_t setup_forces_attributes();

// Lattice-regularised diffusion Monte Carlo (k_lrdmc.cu), FP64 path.
// Per-walker projection state in the caller's workspace.
struct LrdmcWork {
  double *left;    // [W] imaginary time left in this projection
  double *lw;      // [W] log-weight gathered in this projection
  double *eL;      // [W] local energy of the current configuration
  double *rho;     // [W][6N] hop ratios Psi(x') / Psi(x)
  double *r_tmp;   // [W][N][3] positions before a reconfiguration
  int *hops, *flags, *active, *moved;  // [W]
  int *list_up, *list_dn;              // [W] rows w n_up + row of this round's moves
  int *list_w;                         // [W] walkers that moved this round
  int *cnt;                            // [4] up moves, down moves, walkers still active
  void *sub_state;                     // walker state of the moved walkers, compacted
  double *r_sub, *eL_sub;              // their positions [W][N][3] and local energies [W]
};
// per-walker arrays copied between a state and a compacted one
struct WalkerCopy {
  const void *src;
  void *dst;
  size_t bytes;  // per walker, a multiple of 4
};
struct WalkerCopies {
  WalkerCopy c[10];
  int n;
};
// gather (dst[j] = src[list[j]]) or scatter (dst[list[j]] = src[j]) for j < Wc
cudaError_t launch_walker_copy(const WalkerCopies &cp, const int *list, int Wc, bool scatter, cudaStream_t st);
cudaError_t launch_lrdmc_ratios(const DevSystem &s, const double *r, const double *mbuf, const int *active, double a,
                                double *rho, int W, cudaStream_t st);
cudaError_t launch_lrdmc_start(const int *status, int W, double tau, LrdmcWork &lw, cudaStream_t st);
cudaError_t launch_lrdmc_decide(const DevSystem &s, double *r, const double *eL, const int *status, int W,
                                uint32_t walker0, uint32_t gen, double a, double gamma, double e_ref, int max_hops,
                                LrdmcWork &lw, cudaStream_t st);
cudaError_t launch_lrdmc_rows(const DevSystem &s, const double *r, const int *moved, double *pprop, double *phi_up,
                              int W, cudaStream_t st);
cudaError_t launch_lrdmc_finish(int W, const double *lw, const double *eL_cur, double *weight, double *eL_out,
                                cudaStream_t st);
// parents by systematic resampling, (wbar, ebar) into stats, weights reset to
// 1, r_new[j] = r_old[parent[j]]
cudaError_t launch_lrdmc_branch(int W, int N, uint32_t gen, uint32_t key0, uint32_t key1, double *weight,
                                const double *eL, int *parent, double *stats, const double *r_old, double *r_new,
                                cudaStream_t st);
cudaError_t launch_lrdmc_energy(const double *wbar, const double *ebar, int T, int p, double *E, cudaStream_t st);

// one-time kernel attribute set-up (dynamic shared memory limits), per file
cudaError_t setup_kernel_attributes();
cudaError_t setup_walker_attributes();
cudaError_t setup_energy_attributes();

}  // namespace jagp
