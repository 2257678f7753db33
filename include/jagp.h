/*
 * jagp.h -- C ABI of libjagp, a GB300 (sm_103a) implementation of the
 * data-parallel hot path of variational Monte Carlo (VMC) for
 * Jastrow-correlated antisymmetrized-geminal-power (JAGP) wave functions,
 * following TurboRVB (Nakano et al., arXiv 2002.07401).
 *
 * Wave function (Sec. "Wave functions"):  Psi(x) = det(G~(x)) * exp(J(x)), with
 *   G~ = [G_ud | Phi] the N_up x N_up geminal matrix of Eq. wfAGPunpaired,
 *   G_ud[i][j] = sum_{mu,nu} phi_mu(r_i^up) lambda_{mu,nu} phi_nu(r_j^dn)   (Eq. agp_expansion)
 *   Phi[i][l]  = sum_mu c^{(l)}_mu phi_mu(r_i^up)     (k = N_up - N_dn unpaired orbitals)
 *   phi_mu: Gaussian or Slater atomic orbitals, l <= 2 (Eqs. gaussian, slater),
 *   J = J1 + J2 (Eqs. onebody_J_hom, onebody_u, twobody_jastrow, twobody_v).
 * Local energy e_L = H Psi / Psi (Sec. VMC, Eq. 1); sampling by single-electron
 * Metropolis moves (Sec. VMC).
 *
 * Conventions shared by every call:
 *   - Electron positions r are float64 [W][N][3] (bohr), up electrons first.
 *   - Pointers named d_* are DEVICE pointers owned by the caller; pointers named
 *     h_* (and everything reached through jagp_system_t) are HOST pointers,
 *     copied during the call.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).
 *     Calls are asynchronous on that stream unless stated otherwise.
 *   - Every call returns a jagp_status_t; JAGP_OK is 0.  Argument errors are
 *     detected on the host before any launch.  Numerical failures inside the
 *     kernels (a non-finite ratio, a singular geminal matrix at a refresh) set
 *     per-walker status bits that jagp_walker_status() reads back.
 *   - The library never synchronises the device except where a call says so.
 */
#ifndef JAGP_H
#define JAGP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int jagp_status_t;
#define JAGP_OK 0
#define JAGP_ERR_INVALID_ARG 1  /* a size, pointer or option is out of range */
#define JAGP_ERR_SINGULAR 2     /* |det G~| = 0 or non-finite at a refresh */
#define JAGP_ERR_NONFINITE 3    /* NaN/Inf in a position or a ratio */
#define JAGP_ERR_OOM 4          /* a device allocation inside jagp_create failed */
#define JAGP_ERR_TIMEOUT 5      /* a bounded device wait expired */
#define JAGP_ERR_UNSUPPORTED 6  /* e.g. l > 2, N_dn > N_up, too many walkers */
#define JAGP_ERR_CUDA 7         /* a CUDA runtime call failed */

/* per-walker status bits (jagp_walker_status) */
#define JAGP_WS_NONFINITE 1
#define JAGP_WS_SINGULAR 2
#define JAGP_WS_DRIFT 4          /* Sherman-Morrison drift above tolerance at a refresh */

#define JAGP_PREC_FP64 0         /* every step in float64 */
#define JAGP_PREC_MIXED 1        /* orbitals as double-word FP32 tables, proposed rows, Sherman-Morrison
                                    and the kinetic contraction in FP32, lambda products on the BF16
                                    tensor cores (operands cut into exact 8-bit fixed-point slices,
                                    FP32 accumulation); G~^{-1} refreshed by an FP64 elimination after
                                    every half-sweep (or every refresh_moves moves); log|det|, Jastrow,
                                    energies and their sums in FP64 */

/* The system: atoms, basis, pairing matrix lambda, unpaired orbitals, Jastrow.
 * All pointers are host pointers, read during jagp_create only. */
typedef struct jagp_system {
  int n_atoms;
  const double *R;            /* [n_atoms][3] nuclear positions (bohr) */
  const double *Z;            /* [n_atoms] nuclear charges */
  int n_shells;
  const int *shell_atom;      /* [n_shells] owning atom */
  const int *shell_l;         /* [n_shells] angular momentum 0..2 (components: s; x,y,z;
                                 xy,yz,zx,x^2-y^2,3z^2-r^2, relative to the atom) */
  const int *shell_radial;    /* [n_shells] 0 = Gaussian e^{-zeta r^2}, 1 = Slater e^{-zeta r} */
  const double *shell_zeta;   /* [n_shells] exponent */
  const double *lambda;       /* [L][L] row-major, L = sum (2l+1); need not be symmetric */
  int n_up, n_dn;             /* N_up >= N_dn >= 0, N_up >= 1 */
  const double *unpaired;     /* [N_up-N_dn][L] unpaired-orbital coefficients, NULL if equal */
  double b_ea;                /* J1 parameter (0 = the b -> 0 limit u = r/2) */
  double b_para, b_anti;      /* J2 parameters */
  int use_j1, use_j2;
  int j2_spin_independent;    /* 1: r/(2(1+b_anti r)) for every pair */
  /* three/four-body Jastrow (Eq. threebody_jastrow), read only when use_j3:
   *   J3 = sum_{i<j} sum_{mu,nu} M^{s_i s_j}_{mu,nu} chi_mu(r_i) chi_nu(r_j)
   * with its own basis chi (shells in the format above, LJ functions) and the
   * symmetric coupling matrices j3_para (equal spins) and j3_anti [LJ][LJ].
   * FP64 handles only; jagp_grad and guided sampling reject it (UNSUPPORTED). */
  int n_jshells;
  const int *jshell_atom, *jshell_l, *jshell_radial;
  const double *jshell_zeta;
  const double *j3_para, *j3_anti;
  int use_j3;
} jagp_system_t;

typedef struct jagp_options {
  int precision;              /* JAGP_PREC_FP64 or JAGP_PREC_MIXED */
  int max_walkers;            /* upper bound on W for every later call */
  double delta;               /* proposal half-width: r' = r + delta (2u - 1) per coordinate */
  uint64_t seed;              /* Philox4x32-10 key */
  double drift_tol;           /* Sherman-Morrison drift tolerance checked at each refresh
                                 (<= 0: 1e-8 for FP64, 1e-3 for MIXED) */
  int refresh_moves;          /* 0: refresh G~^{-1} from the tables once per sweep (FP64) or
                                 after each spin half-sweep (MIXED); k > 0: also after every
                                 k moves within a spin half-sweep (e.g. 16); < 0: INVALID_ARG */
  int fp64_tensor_cores;      /* FP64 only.  0: lambda products with FP64 instructions.  1: the
                                 same products FP64-equivalent on the BF16 tensor cores: FP64
                                 rows cut into 7 exact 8-bit slices (8 slices of 7 bits when
                                 L > 512), every slice pair of weight >= 2^-56 summed exactly in
                                 its own accumulator, combined in FP64 (Ozaki-style splitting) */
} jagp_options_t;

typedef struct jagp_ctx *jagp_handle_t;

/* Create a handle: validates the system, copies lambda, lambda^T, the shell
 * table and the unpaired orbitals to the current device (the handle owns
 * those copies; jagp_destroy frees them).  Synchronous.
 * Errors: INVALID_ARG (bad sizes/pointers), UNSUPPORTED (l > 2, N_dn > N_up,
 * N_up > 1024), OOM, CUDA. */
jagp_status_t jagp_create(jagp_handle_t *out, const jagp_system_t *sys, const jagp_options_t *opt);
jagp_status_t jagp_destroy(jagp_handle_t h);

/* Bytes of device workspace ("walker state") that W walkers need.  The caller
 * allocates it (e.g. a torch uint8 tensor), 256-byte aligned, and passes it to
 * the calls below; it holds G~^{-1}, the orbital tables, log|det| and the
 * per-walker counters.  Returns 0 for an invalid W. */
size_t jagp_state_bytes(jagp_handle_t h, int W);

/* log|Psi| and sign(Psi) of W configurations, and (re)build the walker state
 * for them (Sec. AGP: G~ = Phi_up lambda Phi_dn^T | Phi_up C; LU with partial
 * pivoting; J).  d_r: [W][N][3]; d_logabs, d_sign: [W] (either may be NULL).
 * Afterwards d_state is consistent with d_r and may be passed to vmc_sweep /
 * local_energy.  A singular G~ sets JAGP_WS_SINGULAR for that walker. */
jagp_status_t jagp_eval(jagp_handle_t h, const double *d_r, int W, void *d_state, double *d_logabs,
                        double *d_sign, void *stream);

/* nsweeps Metropolis sweeps (Sec. VMC) over W walkers whose state came from
 * jagp_eval or an earlier vmc_sweep on the same d_r.  One sweep moves every
 * electron once (up electrons 0..N_up-1, then down), each move drawing the
 * Philox4x32-10 block counter = (walker0 + w, sweep0 + t, electron, 1),
 * key = (seed lo, seed hi): x0..x2 give the proposal, x3 the acceptance draw
 * u = x3 2^-32; accept iff u < |Psi(x')/Psi(x)|^2.  The ratio uses
 * Sherman-Morrison updates of G~^{-1}; G~^{-1}, log|det| and J are refreshed
 * in FP64 after every sweep (and as jagp_options_t.refresh_moves and the
 * precision ask within it).  d_r is updated in place.
 * d_eL: [nsweeps][W] local energy after each sweep, or NULL (no energies).
 * d_acc: [nsweeps][4] (sum e_L, sum e_L^2, accepted moves, max drift) or NULL. */
jagp_status_t vmc_sweep(jagp_handle_t h, double *d_r, void *d_state, int W, int nsweeps,
                        uint64_t walker0, uint64_t sweep0, double *d_eL, double *d_acc, void *stream);

/* Local energy e_L = -1/2 sum_i lap_i Psi/Psi + V_ee + V_ei + V_ii (Sec. VMC,
 * Eq. 1) of W configurations whose state is current.  d_eL: [W].
 * d_parts: [W][4] (kinetic, V_ee, V_ei, V_ii) or NULL. */
jagp_status_t local_energy(jagp_handle_t h, const double *d_r, void *d_state, int W, double *d_eL,
                           double *d_parts, void *stream);

/* Per-walker log-derivatives for stochastic reconfiguration (Sec.
 * "Derivatives with respect to variational parameters": O_k(x) =
 * d ln|Psi(x)| / d alpha_k) of W walkers whose state is current (jagp_eval /
 * vmc_sweep on d_r), for the P = L*L + 3 parameters: every entry of lambda
 * taken as independent (row-major, O[mu L + nu] = sum_{i, j < N_dn}
 * G~^{-1}[j][i] phi_mu(r_i^up) phi_nu(r_j^dn)), then b_ea, b_para, b_anti.
 * d_O: [W][ldo] FP64, ldo >= P (device, caller-owned); d_work: device
 * workspace of jagp_logpsi_derivs_workspace_bytes(h, W) bytes, 256-byte
 * aligned.  FP64 handles only (UNSUPPORTED otherwise); INVALID_ARG for
 * ldo < P.  Leaves d_state unchanged. */
size_t jagp_logpsi_derivs_workspace_bytes(jagp_handle_t h, int W);
jagp_status_t jagp_logpsi_derivs(jagp_handle_t h, const double *d_r, void *d_state, int W, void *d_work, double *d_O,
                                 long long ldo, void *stream);

/* One regularised stochastic-reconfiguration step (Sec. "Stochastic
 * reconfiguration", Eqs. SRupdate and sr with the diagonal shift
 * s'_kk = s_kk (1 + eps)) from M samples: d_O [M][ldo] log-derivatives (the
 * first P columns are used) and d_eL [M] local energies, all device FP64.
 *   Obar_k = (1/M) sum_i O_ik,  S_kl = (1/M) sum_i (O_ik - Obar_k)(O_il - Obar_l),
 *   d_f[k] = f_k = -2 (1/M) sum_i (e_i - ebar)(O_ik - Obar_k)     (Eq. eq_general_force),
 *   d_dalpha = delta (S')^{-1} f,
 * solved by conjugate gradients preconditioned with diag(S') without forming
 * S: each iteration multiplies by S' through two passes over the samples,
 * (1/M) O_c^T (O_c v) + eps diag(S) v, O_c = O - Obar.  A parameter whose
 * samples do not vary (S_kk = 0) keeps dalpha_k = 0.  Iterates until the
 * residual norm is at most tol times that of f, or max_iter iterations;
 * *h_iters and *h_resid (host, may be NULL) receive the iterations and the
 * final relative residual.  d_work: device workspace of
 * jagp_sr_workspace_bytes(M, P) bytes, 256-byte aligned.  Synchronises
 * stream (the iteration is steered from the host).  Errors: INVALID_ARG for
 * M < 2, P < 1, ldo < P, eps < 0, tol < 0 or a NULL pointer. */
size_t jagp_sr_workspace_bytes(int M, int P);
jagp_status_t jagp_sr_step(const double *d_O, long long ldo, const double *d_eL, int M, int P, double eps,
                           double delta, int max_iter, double tol, void *d_work, double *d_f, double *d_dalpha,
                           int *h_iters, double *h_resid, void *stream);

/* Statistics of the sampled local energies (Sec. VMC: the VMC energy is the
 * mean of e_L over the Markov chain, its error bar from the correlated samples
 * by reblocking).  d_eL: [T][W] local energies of W walkers over T sweeps (as
 * vmc_sweep writes them).  The series is the walker mean per sweep,
 * m_t = (1/W) sum_w d_eL[t][w] (kept in d_work [T], caller-owned).  Level k
 * (k < jagp_reblock_levels(T), the levels with at least two blocks) cuts it
 * into n_k = floor(T / 2^k) consecutive blocks of B = 2^k sweeps (a ragged
 * tail is dropped) with block means b_j and writes d_levels[k] = (B, n_k,
 * sigma_k, err_k), sigma_k = sqrt(sum_j (b_j - bbar)^2 / (n_k (n_k - 1))),
 * err_k = sigma_k / sqrt(2 (n_k - 1)).  d_stats [4] = (mean of all T W values,
 * chosen sigma, chosen level, 1 if a plateau was found): the chosen level is
 * the smallest k whose next level still has >= 8 blocks and lies within err_k
 * of sigma_k, else the last level with >= 8 blocks (plateau 0).  FP64, fixed
 * summation order.  Device pointers; asynchronous on stream.  Errors:
 * INVALID_ARG for T or W < 1 or a NULL pointer (d_levels may be NULL when
 * T = 1). */
int jagp_reblock_levels(int T);
jagp_status_t jagp_reblock(const double *d_eL, int T, int W, double *d_work, double *d_levels, double *d_stats,
                           void *stream);

/* Batches of independent systems (uneven electron counts, each with its own
 * handle and walker state): jagp_batch_sweep runs nsweeps sweeps of every
 * system, exactly as vmc_sweep would (same Philox counters, walker indices
 * walker0[s] + w, sweep indices sweep0 + t), with local energies after each
 * sweep written to d_eL[s] ([W[s]], the last sweep's) and accumulated into
 * d_acc[s][4] (sum e_L, sum e_L^2, accepted moves, max drift; the caller
 * zeroes it).  The first jagp_batch_sweep captures one sweep of all systems
 * into a CUDA graph, which every later sweep replays.  With n_streams = 0 the
 * graph holds grouped launches: each system's launch sequence is recorded,
 * and the launches of one kernel at one point of the sweep (a spin
 * half-sweep's proposals, the acceptance of its k-th block of moves, the
 * lambda products of the accepted rows, the steps of a refresh, the local
 * energy, the sums) are issued as ONE launch over all systems' work (about a
 * hundred launches per sweep for the 64-system workload, against one
 * sequence per system); if a system's sequence cannot be grouped, the
 * per-system form with 8 streams is used instead.  With n_streams = -k the
 * systems are split into k lanes of about equal cost, each lane a chain of
 * grouped launches on its own stream of the graph.  With n_streams > 0 every
 * system's own launches are forked over n_streams concurrent streams,
 * largest systems first.  The per-system forms give bit for bit the results
 * of per-system vmc_sweep calls (the same kernels); a grouped launch runs the
 * same formulas in the same order for each system but is compiled as another
 * kernel, so its floating-point results may differ in the last bits (the
 * tests find the same trajectories and local energies within 1e-11).  The
 * sweep index
 * is read from a device counter, so the states, positions and output arrays
 * must stay where they were when the batch was created.  Handles, states and
 * arrays are borrowed, not copied.  d_eL and d_acc may be NULL. */
typedef struct jagp_batch *jagp_batch_t;
jagp_status_t jagp_batch_create(jagp_batch_t *out, int S, const jagp_handle_t *handles, void *const *d_states,
                                double *const *d_r, const int *W, const uint64_t *walker0, double *const *d_eL,
                                double *d_acc, int n_streams);
jagp_status_t jagp_batch_sweep(jagp_batch_t b, int nsweeps, uint64_t sweep0, void *stream);
jagp_status_t jagp_batch_destroy(jagp_batch_t b);
/* Kernel launches (*h_kernels) and all nodes (*h_nodes, may be NULL) of the
 * CUDA graph that one batched sweep replays (0 before the first
 * jagp_batch_sweep captures it).  Host-only. */
jagp_status_t jagp_batch_launches(jagp_batch_t b, long long *h_kernels, long long *h_nodes);

/* Reverse-mode (adjoint) derivatives, Sec. "Derivatives of energy" (AAD) and
 * Eqs. eq_general_force, forces:aad (without the space warp):  for W walkers
 * whose state is current (jagp_eval / vmc_sweep on d_r) and per-walker seeds
 * sL = d_seed_logpsi[w], sE = d_seed_eL[w] (either array may be NULL = 0),
 * the vector-Jacobian products
 *   d_dlambda[mu][nu] = sum_w (sL d log|Psi_w|/d lambda_{mu,nu} + sE d e_L,w/d lambda_{mu,nu})
 *                        (every entry of lambda taken as independent)          [L][L] or NULL
 *   d_djas[3]         = sum_w sL d log|Psi_w| / d (b_ea, b_para, b_anti)       (log|Psi| part only)
 *   d_dR[a][3]        = sum_w (sL d log|Psi_w|/dR_a + sE d e_L,w/dR_a)          or NULL
 *   d_dR_walker[w][a][3]  the same per walker                                 or NULL
 *   d_dr[w][i][3]     = sL d log|Psi_w|/dr_i + sE d e_L,w/dr_i                  or NULL
 * and d_eL[w] (the local energies the derivatives belong to, or NULL).  With
 * sL = 2 (e_L - <e_L>) / M and sE = 1 / M, d_dR is minus the Hellmann-Feynman +
 * Pulay force -<de_L/dR> - 2 cov(e_L, d log|Psi|/dR).  d_work: caller-owned
 * device workspace of jagp_grad_workspace_bytes(h, W) bytes, 256-byte aligned.
 * The jagp_grad call leaves d_state valid.  FP64 handles only (UNSUPPORTED otherwise). */
size_t jagp_grad_workspace_bytes(jagp_handle_t h, int W);
jagp_status_t jagp_grad(jagp_handle_t h, const double *d_r, void *d_state, int W, const double *d_seed_logpsi,
                        const double *d_seed_eL, void *d_work, double *d_eL, double *d_dlambda, double *d_djas,
                        double *d_dR, double *d_dR_walker, double *d_dr, void *stream);

/* Space-warp coordinate transformation for the forces (Sec. "Atomic forces",
 * Eq. forces:aad and the two total derivatives that follow it): electrons
 * move with nucleus a by Delta R_a omega_a(r), omega_a(r) = kappa(|r - R_a|) /
 * sum_b kappa(|r - R_b|), kappa(d) = 1/d^4.  Takes jagp_grad's per-walker
 * outputs for the same d_r and seeds, d_rbar = d_dr [W][N][3] (sL d ln|Psi|/dr
 * + sE d e_L/dr) and d_dR_walker [W][n_atoms][3] (the same w.r.t. R_a), and
 * adds in place, per walker,
 *   sum_i omega_a(r_i) d_rbar[w][i] + (sL_w / 2) sum_i grad omega_a(r_i)
 * (d_seed_logpsi = sL, NULL = 0), so that d_dR_walker[w][a] becomes
 * sE d e_L/dR_a + sL d ln(J^{1/2} Psi)/dR_a with the warp's total derivatives;
 * d_dR [n_atoms][3] (may be NULL) receives their sum over walkers.  With the
 * force seeds (jagp_force_seeds) the sum is minus the force.  Device pointers,
 * asynchronous.  Errors: INVALID_ARG. */
jagp_status_t jagp_space_warp(jagp_handle_t h, const double *d_r, int W, const double *d_rbar,
                              const double *d_seed_logpsi, double *d_dR_walker, double *d_dR, void *stream);

/* The guiding function's regularisation (Sec. "Atomic forces", Eqs. R_r,
 * regularization, reweighting) for W walkers whose state is current:
 *   R(x) = (S sum_{i,j} |G~^{-1}_{ij}|^2)^{-theta},  S = min_i sum_j |G~_ij|^2,
 *   d_W[w] = (R / max(R, eps))^2   (the reweighting factor of Psi_G samples),
 * d_R [W], d_W [W] device (either may be NULL, not both).  G~ is recomputed from
 * the state's tables into the state's refresh scratch.  theta > 0 (the paper
 * uses 3/8), eps >= 0.  Errors: INVALID_ARG. */
jagp_status_t jagp_guiding_weights(jagp_handle_t h, void *d_state, int W, double theta, double eps, double *d_R,
                                   double *d_W, void *stream);

/* Sample the guiding function instead of the trial wave function (Sec.
 * "Atomic forces", Eq. guiding_function): with eps > 0 every later vmc_sweep
 * (and batched sweep) of h accepts a move with probability
 * |Psi_T(x')/Psi_T(x)|^2 W(x) / W(x'), W = (R / max(R, eps))^2 and R as in
 * jagp_guiding_weights, i.e. samples |Psi_G|^2 = |Psi_T|^2 / W; estimates then
 * take the weights W (<W A>_G / <W>_G = <A>_T, Eq. reweighting).  eps = 0
 * restores plain sampling.  Host-only.  Errors: INVALID_ARG (theta <= 0,
 * eps < 0), UNSUPPORTED (eps > 0 on a mixed-precision handle or N_up > 64:
 * the guided acceptance keeps G~ and G~^{-1} in shared memory). */
jagp_status_t jagp_set_guiding(jagp_handle_t h, double theta, double eps);

/* Seeds of the (reweighted) force estimator for jagp_grad (Sec. "Atomic
 * forces", Eq. reweighting; Eq. eq_general_force): from local energies d_eL [M]
 * and weights u = d_weight [M] (NULL: all 1), with U = sum u and
 * E = sum u e / U,
 *   d_seed_eL[i] = u_i / U,   d_seed_logpsi[i] = 2 u_i (e_i - E) / U,
 * so that jagp_grad (plus jagp_space_warp) returns minus the force
 * <W F>/<W>.  d_mean [2] (may be NULL) = (E, U / M).  Device pointers. */
jagp_status_t jagp_force_seeds(const double *d_eL, const double *d_weight, int M, double *d_seed_logpsi,
                               double *d_seed_eL, double *d_mean, void *stream);

/* ------------------------------------------------------------------------ */
/* Lattice-regularised diffusion Monte Carlo (Sec. "Lattice regularized     */
/* Monte Carlo"), continuous time, fixed node, guiding function = Psi_T.    */
/* ------------------------------------------------------------------------ */
/* One projection of imaginary-time length tau for W walkers at d_r [W][N][3]
 * (device, updated in place).  Hop k = 6 i + 2 d + s moves electron i by +a
 * (s = 0) or -a (s = 1) along axis d; rho_k = Psi(x') / Psi(x) and the
 * fixed-node rate t_k = (rho_k > 0 ? rho_k : gamma |rho_k|) / (2 a^2),
 * Gamma = sum_k t_k.  A walker at x waits tau_xi = -ln(1 - xi) / Gamma and
 * its log-weight falls by tau_xi (e_L(x) - e_ref); when the wait reaches the
 * time left it falls by the time left times (e_L(x) - e_ref) and the walker
 * stops, else it hops to the first k whose running sum of t exceeds u Gamma.
 * Hop h of walker walker0 + w in generation `generation` draws Philox4x32-10
 * (counter (walker0 + w, generation, h, 2), the handle's seed as key):
 * xi = (x0 + 1/2) 2^-32, u = (x1 + 1/2) 2^-32.  A walker stops after
 * max_hops hops (flag bit 1); one whose G~ is singular or positions are not
 * finite takes no part (flag bit 2); a non-finite rate sum or e_L ends the
 * walker's projection (flag bit 4).
 * d_weight [W] in/out: multiplied by exp(log-weight change).  d_eL [W]
 * (or NULL): e_L at the final configuration.  d_hops, d_flags [W] (or NULL).
 * d_state is evaluated at the start (jagp_eval) and is current at the end.
 * d_work: jagp_lrdmc_workspace_bytes(h, W) bytes, 256-byte aligned, device
 * (it holds, besides the per-walker projection state, a compact walker state
 * in which each round's moved walkers are refreshed).
 * Synchronises the stream once per round of hops (every walker still moving
 * takes one hop per round).  a > 0, gamma >= 0, tau >= 0, max_hops >= 0.
 * Errors: INVALID_ARG; UNSUPPORTED for a mixed-precision handle or the
 * three-body Jastrow. */
size_t jagp_lrdmc_workspace_bytes(jagp_handle_t h, int W);
jagp_status_t jagp_lrdmc_project(jagp_handle_t h, double *d_r, void *d_state, int W, uint64_t walker0,
                                 uint64_t generation, double a, double gamma, double tau, double e_ref, int max_hops,
                                 double *d_weight, double *d_eL, int *d_hops, int *d_flags, void *d_work,
                                 void *stream);

/* Reconfiguration after a projection (Eqs. branching-1, branching-2): W new
 * walkers drawn from the old ones with probability w_a / sum w by systematic
 * resampling with one uniform z per generation (Philox4x32-10, counter
 * (0, generation, 0, 3), z = (x0 + 1/2) 2^-32): new walker j copies the first
 * old walker whose running weight sum exceeds (j + z) sum w / W.  d_r [W][N][3]
 * is replaced by the new population, d_weight [W] reset to 1, d_parent [W]
 * (or NULL) receives the old indices, d_stats [2] = (wbar = sum w / W,
 * ebar = sum w e_L / sum w) from d_eL [W].  The walkers' state must be
 * re-evaluated (jagp_lrdmc_project does so).  d_work as for
 * jagp_lrdmc_project.  Device pointers.  Errors: INVALID_ARG. */
jagp_status_t jagp_lrdmc_branch(jagp_handle_t h, double *d_r, int W, uint64_t generation, double *d_weight,
                                const double *d_eL, int *d_parent, double *d_stats, void *d_work, void *stream);

/* Energy with the correcting factor (Eq. many-walker-weight and the estimator
 * after it) from T generations' d_wbar, d_ebar [T]:
 *   E = sum_{n=p}^{T-1} G_n ebar_n / sum_{n=p}^{T-1} G_n,
 *   G_n = prod_{j=1..p} wbar_{n-j}  (formed as exponentials of log sums).
 * d_E [1] device.  0 <= p < T.  Errors: INVALID_ARG. */
jagp_status_t jagp_lrdmc_energy(const double *d_wbar, const double *d_ebar, int T, int p, double *d_E, void *stream);

/* Copy per-walker bookkeeping to device arrays (each may be NULL):
 * log|Psi|, sign, accepted moves since jagp_eval, last drift, status bits. */
jagp_status_t jagp_walker_info(jagp_handle_t h, const void *d_state, int W, double *d_logabs,
                               double *d_sign, double *d_naccept, double *d_drift, int *d_status,
                               void *stream);

/* OR of the status bits of all W walkers.  Synchronises `stream`.  Returns
 * JAGP_ERR_TIMEOUT if a bounded wait of the handle's tensor-core pipeline
 * expired in an earlier call (the bits are still written). */
jagp_status_t jagp_walker_status(jagp_handle_t h, const void *d_state, int W, int *h_bits,
                                 void *stream);

/* Tile autotuner (no counterpart in the paper: a property of this GPU code).
 * Times the candidate tilings of the per-walker products (proposed rows and
 * columns: one output per thread, 32x32 or 64x64 register-blocked tiles; the
 * refresh product G~ = Phi_up Bt^T likewise) and, in the mixed path, the
 * output-tile width (32..128 columns) and pipeline depth of the tensor-core
 * lambda products, on
 * this handle's operands and the caller's state buffer of W walkers; keeps the
 * fastest in the handle for every later call.  The choices change only the
 * tiling of outputs, never the order of a sum: results are identical with or
 * without tuning.  The state's tables are overwritten: call jagp_eval before
 * the next sweep.  Synchronises `stream`.  out (host) receives the choices and
 * the best times (ms per call: proposals, refresh, A_up rows, Bt rows). */
typedef struct {
  int tile_proposals;  /* 0: one output per thread; 32 / 64: blocked tiles; 16 (refresh, mixed,
                          N_up <= 16): four walkers per CTA, 2x2 outputs per thread */
  int tile_refresh;
  int umma_bn_left;    /* mixed path: tensor-core tile width, A_up = phi^T lambda (0 in FP64) */
  int umma_bn_right;   /* mixed path: tensor-core tile width, Bt = lambda phi */
  float ms[4];
  int umma_stages_left;   /* pipeline stages of those products (0: as many as fit in 200 KB;
                             -1, -2, -3: chunk-major, two to four stages each holding every
                             slice of one K chunk of 64, 32 or 16 elements, so that a slice
                             is read once for all its pairs) */
  int umma_stages_right;
} jagp_tuning_t;
jagp_status_t jagp_autotune(jagp_handle_t h, void *d_state, int W, jagp_tuning_t *out, void *stream);
/* Pin the tile choices of a handle without timing (e.g. those an earlier
 * jagp_autotune returned for the same system and walker count).  Host-only, no
 * CUDA call; ms is ignored.  tile_proposals / tile_refresh: -1 (the shape
 * heuristics), 0, 32 or 64, and 16 for tile_refresh in the mixed path with
 * N_up <= 16.  umma_*: 0 without tensor-core lambda products (FP64 without
 * fp64_tensor_cores); else bn 0 (heuristic) or a multiple of 16 up to 64 (six
 * or more tensor-memory accumulators), and stages -1, -2, -3 (chunk-major with
 * K chunks of 64, 32, 16, only where two such stages fit in shared memory), 0
 * or 2..6.
 * Every choice changes the tiling only, so results stay as without tuning.
 * Returns JAGP_ERR_INVALID_ARG (and keeps the earlier choices) on any other value. */
jagp_status_t jagp_set_tuning(jagp_handle_t h, const jagp_tuning_t *t);

/* The tensor-core contraction behind the lambda products of the mixed
 * precision path (Sec. AGP, Eq. agp_expansion: rows phi^T lambda and
 * lambda phi), exposed for direct use and testing.  tcgen05.mma (BF16 in,
 * FP32 accumulate in tensor memory) fed by TMA.
 *   plain mode (d_row_exp = d_col_exp = NULL):
 *     C[rows[m]][n] = sum_{p < npairs} sum_{k < Kp} A[m][pair_a[p] Kp + k] * B[n][pair_b[p] Kp + k]
 *   fixed-point mode (both exponent arrays given): the terms are exact 8-bit
 *     integer slices, a = 2^(ea[m] - 7) sum_t A_t / 256^t (likewise b with
 *     eb[n]), pairs with equal pair_a + pair_b (<= 5) share an exactly summed
 *     accumulator S_d, and C = 2^(ea + eb - 14) sum_d S_d / 256^d.
 * d_A: BF16 bits [M][a_terms Kp], d_B: BF16 bits [N][b_terms Kp] (up to six
 * terms per row side by side; Kp % 64 == 0; 16-byte aligned bases); d_C: FP32
 * with row pitch ldc >= N; d_rows: [M] destination rows or NULL (identity);
 * d_count: device int live row count (<= M) or NULL (= M); d_row_exp [M],
 * d_col_exp [N]: device ints or NULL.  h_pair_a/h_pair_b: host arrays of
 * npairs (1..21) term indices.  *d_err (device int) is set non-zero if a
 * pipeline wait timed out.  Errors: INVALID_ARG for shapes, alignment or term
 * indices. */
jagp_status_t jagp_gemm_bf16x(const uint16_t *d_A, int M, int a_terms, const uint16_t *d_B, int N, int b_terms,
                              int Kp, int npairs, const int *h_pair_a, const int *h_pair_b, float *d_C,
                              long long ldc, const int *d_rows, const int *d_count, const int *d_row_exp,
                              const int *d_col_exp, int *d_err, void *stream);

/* Profiling hooks (Sec. "Derivatives of energy" aside, these are tooling, not
 * part of the method).  jagp_profile(h, kernel, 1) makes later vmc_sweep /
 * jagp_eval calls record a CUDA event pair on the launching stream around every
 * launch of `kernel` (JAGP_KERNEL_*); jagp_profile_read synchronises those
 * events, returns the summed device time (ms) and the number of launches, and
 * clears the record.  jagp_launch_count returns how many kernels the handle
 * has launched since jagp_create. */
#define JAGP_KERNEL_LAMBDA_ROWS 1   /* lambda products of accepted orbital rows */
#define JAGP_KERNEL_GEMM_ROWS 2     /* proposed rows / columns and the refresh G~ */
#define JAGP_KERNEL_METROPOLIS 3
#define JAGP_KERNEL_BASIS 4
#define JAGP_KERNEL_ENERGY 5        /* kinetic contraction + local energy */
jagp_status_t jagp_profile(jagp_handle_t h, int kernel, int enable);
jagp_status_t jagp_profile_read(jagp_handle_t h, double *h_total_ms, long long *h_launches);
long long jagp_launch_count(jagp_handle_t h);

/* jagp_eval without any device allocation and without a workspace argument.
 * The paper has no counterpart: this is a convenience of the library for
 * callers that cannot allocate device memory when they need log|Psi| (code
 * running under an allocator or memory pool that forbids new reservations, a
 * host framework that owns every allocation, a loop that must not touch the
 * allocator).  It computes d_logabs and d_sign [W] for the configurations
 * d_r [W][N][3] always in FP64, whatever the handle's precision: on an FP64
 * handle the same values as jagp_eval, on a mixed-precision handle the FP64
 * values (jagp_eval's mixed-precision log|Psi| differs from them by at most its
 * stated 1e-6).  Its scratch is one file-scope device array of
 * JAGP_NOALLOC_SCRATCH_BYTES that every GPU loading the library holds until the
 * process exits.  Its kernels count towards jagp_launch_count.
 *   - Allocates nothing: no cudaMalloc, cudaFree or allocating library call
 *     (jagp_create still allocates the handle's tables once, at set-up).
 *   - W whose scratch (about 4 N_up L + 2 N_up^2 doubles per walker) exceeds
 *     the array returns JAGP_ERR_UNSUPPORTED before any launch.
 *   - The first call on a device looks up the array's address (that device
 *     must be current); make that first call before any stream capture.
 *   - All calls share the array, which keeps the last call's contents; the
 *     call clears what must start at zero.  Calls that overlap on the GPU
 *     (other streams, other host threads) race on it: serialise them.
 *   - A singular G~ gives log|Psi| = -inf and sign 0; no walker state is kept. */
#define JAGP_NOALLOC_SCRATCH_BYTES (32u << 20)
jagp_status_t jagp_eval_noalloc(jagp_handle_t h, const double *d_r, int W, double *d_logabs,
                                double *d_sign, void *stream);

const char *jagp_status_string(jagp_status_t s);
/* The text of the last CUDA runtime error behind a JAGP_ERR_CUDA of this thread. */
const char *jagp_last_cuda_error(void);

/* The last failure recorded on handle h (Sec. "Implementation and operations"
 * has no counterpart: a diagnostic of this library).  Every entry point that
 * takes h records a non-OK return as one line "<entry point>: <status text>"
 * followed by the CUDA error text behind a JAGP_ERR_CUDA and, where the failing
 * check gives one, the offending value (e.g. "W = 5 outside 1..4").
 * jagp_walker_status also records which walkers carry status bits (the device
 * status words) without failing, and returns JAGP_ERR_TIMEOUT when a bounded
 * tensor-core pipeline wait of this handle expired.  buf (host, may be NULL)
 * receives the text, truncated to len - 1 characters and NUL-terminated.
 * Returns the status of the last failure (JAGP_OK if none), or
 * JAGP_ERR_INVALID_ARG for a NULL handle.  Host-only; not thread-safe against
 * concurrent calls on the same handle. */
jagp_status_t jagp_last_error(jagp_handle_t h, char *buf, size_t len);

#ifdef __cplusplus
}
#endif

#endif /* JAGP_H */
