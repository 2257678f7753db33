/*
 * jagp_oracle.c -- plain, slow FP64 CPU oracle for the JAGP variational Monte
 * Carlo hot path of TurboRVB (arXiv 2002.07401).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the bench's
 * CPU-baseline leg load this file; the CUDA library never does, and the two
 * share no code.  Every function follows the paper's definitions directly
 * (no blocking, no fusion, no incremental updates) so that it can be checked
 * against the paper by eye:
 *
 *   wave function      Psi = Phi_AS * exp(J)                     Sec. 3, Eq. (Psi = Phi_AS x exp J)
 *   AGP determinant    Phi_AGP = det(G~), G~ = [G_ud | Phi]       Sec. AGP, Eqs. wfAGPs, wfAGPunpaired
 *   pairing function   g(r_i, r_j) = sum_{mu,nu} A_{mu,nu} psi_mu(r_i) psi_nu(r_j)
 *                                                                 Eq. agp_expansion (A is lambda here)
 *   atomic orbitals    |r-R|^l e^{-zeta|r-R|^2} Re[Y_lm] (Gaussian), e^{-zeta|r-R|} (Slater)
 *                                                                 Eqs. gaussian, slater
 *   one-body Jastrow   -sum (2Z)^{3/4} u((2Z)^{1/4}|r-R|), u = (1-e^{-b r})/(2b)
 *                                                                 Eqs. onebody_J_hom, onebody_u
 *   two-body Jastrow   sum_{i<j} v(r_ij), v = r/(4(1+b r)) parallel, r/(2(1+b r)) antiparallel
 *                                                                 Eqs. twobody_jastrow, twobody_v
 *   local energy       e_L = H Psi / Psi                          Sec. VMC, Eq. 1
 *   VMC                Metropolis sampling of Psi^2, E = mean e_L Sec. VMC, Eq. 2
 *   log-derivatives    O_k = d ln Psi / d alpha_k                 Sec. "Derivatives", Eq. eq_general_force
 *
 * Counter-based random numbers: Philox4x32-10 (Salmon, Moraes, Dror, Shaw,
 * "Parallel random numbers: as easy as 1, 2, 3", SC'11), written from that
 * paper's definition.
 *
 * Parity status: pinned (see tests/test_oracle_pins.py) for the basis, the
 * determinant (symmetric and non-symmetric lambda), the Jastrow, the local
 * energy, the sampler, log|Psi| gradients and the finite-difference references
 * for d e_L / d R_a, d e_L / d r_i (closed forms of the He product and of an
 * off-centre Slater orbital between two nuclei; the translation sum rule) and
 * d e_L / d lambda (closed form of a two-orbital geminal; Euler's identity).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef struct {
  int n_atoms;
  const double *R;          /* [n_atoms][3] */
  const double *Z;          /* [n_atoms]    */
  int n_shells;
  const int *shell_atom;    /* [n_shells] */
  const int *shell_l;       /* [n_shells] 0,1,2 */
  const int *shell_radial;  /* [n_shells] 0 Gaussian, 1 Slater */
  const double *shell_zeta; /* [n_shells] */
  int L;                    /* number of atomic orbitals */
  const double *lam;        /* [L][L] pairing coefficients lambda_{mu,nu} */
  int n_up, n_dn;           /* n_up >= n_dn */
  const double *unpaired;   /* [n_up-n_dn][L] unpaired orbital coefficients */
  double b_ea, b_para, b_anti;
  int use_j1, use_j2, j2_spin_independent;
  /* three/four-body Jastrow (Eq. threebody_jastrow): its own atomic basis chi
   * (shells as above, LJ functions) and the coupling matrices for parallel and
   * antiparallel pairs, [LJ][LJ] each, symmetric */
  int n_jshells;
  const int *jshell_atom, *jshell_l, *jshell_radial;
  const double *jshell_zeta;
  int LJ;
  const double *j3_para, *j3_anti;
  int use_j3;
} orc_system;

/* ------------------------------------------------------------------------ */
/* Philox4x32-10 (Salmon et al. 2011)                                        */
/* ------------------------------------------------------------------------ */
void orc_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4]) {
  uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
  uint32_t k0 = key_in[0], k1 = key_in[1];
  for (int round = 0; round < 10; ++round) {
    if (round > 0) { k0 += 0x9E3779B9u; k1 += 0xBB67AE85u; }
    uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)c0;
    uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
    uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    uint32_t n0 = hi1 ^ c1 ^ k0, n1 = lo1, n2 = hi0 ^ c3 ^ k1, n3 = lo0;
    c0 = n0; c1 = n1; c2 = n2; c3 = n3;
  }
  out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* ------------------------------------------------------------------------ */
/* Atomic orbitals (Eqs. gaussian, slater).  No normalisation constant: the   */
/* pairing coefficients absorb it.  Cartesian forms of Re[Y_lm]:              */
/*   l=0: 1   l=1: x, y, z   l=2: xy, yz, zx, x^2-y^2, 3z^2-r^2               */
/* (all harmonic, so their own Laplacian vanishes).                          */
/* ------------------------------------------------------------------------ */
static int ncomp(int l) { return 2 * l + 1; }

int orc_nfuncs(const orc_system *s) {
  int L = 0;
  for (int k = 0; k < s->n_shells; ++k) L += ncomp(s->shell_l[k]);
  return L;
}

/* angular polynomial P and its gradient for component c of angular momentum l */
static void angular(int l, int c, const double d[3], double *P, double gP[3]) {
  double x = d[0], y = d[1], z = d[2];
  gP[0] = gP[1] = gP[2] = 0.0;
  if (l == 0) { *P = 1.0; return; }
  if (l == 1) { *P = d[c]; gP[c] = 1.0; return; }
  switch (c) {
    case 0: *P = x * y; gP[0] = y; gP[1] = x; break;
    case 1: *P = y * z; gP[1] = z; gP[2] = y; break;
    case 2: *P = z * x; gP[0] = z; gP[2] = x; break;
    case 3: *P = x * x - y * y; gP[0] = 2 * x; gP[1] = -2 * y; break;
    default: *P = 3 * z * z - (x * x + y * y + z * z);
             gP[0] = -2 * x; gP[1] = -2 * y; gP[2] = 4 * z; break;
  }
}

/* Hessian of the angular polynomial (constant for l <= 2) */
static void angular_hess(int l, int c, double H[3][3]) {
  memset(H, 0, 9 * sizeof(double));
  if (l < 2) return;
  switch (c) {
    case 0: H[0][1] = H[1][0] = 1; break;
    case 1: H[1][2] = H[2][1] = 1; break;
    case 2: H[0][2] = H[2][0] = 1; break;
    case 3: H[0][0] = 2; H[1][1] = -2; break;
    default: H[0][0] = -2; H[1][1] = -2; H[2][2] = 4; break;
  }
}

/*
 * Radial factor g(|d|) with gradient, Hessian and the gradient of its
 * Laplacian (the last two are needed only by the force code).
 *   Gaussian: g = e^{-zeta r^2};  Slater: g = e^{-zeta r}.
 */
static void radial(int type, double zeta, const double d[3], double *g, double gg[3],
                   double Hg[3][3], double *lapg, double glap[3]) {
  double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
  if (type == 0) {
    double e = exp(-zeta * r2);
    *g = e;
    for (int a = 0; a < 3; ++a) gg[a] = -2.0 * zeta * d[a] * e;
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 3; ++b)
        Hg[a][b] = (4.0 * zeta * zeta * d[a] * d[b] - (a == b ? 2.0 * zeta : 0.0)) * e;
    *lapg = (4.0 * zeta * zeta * r2 - 6.0 * zeta) * e;
    /* d/dx_a [(4 z^2 r^2 - 6 z) e] = 8 z^2 d_a e + (4 z^2 r^2 - 6 z)(-2 z d_a) e */
    for (int a = 0; a < 3; ++a)
      glap[a] = (8.0 * zeta * zeta - 2.0 * zeta * (4.0 * zeta * zeta * r2 - 6.0 * zeta)) * d[a] * e;
  } else {
    double r = sqrt(r2);
    double e = exp(-zeta * r);
    *g = e;
    for (int a = 0; a < 3; ++a) gg[a] = -zeta * d[a] / r * e;
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 3; ++b)
        Hg[a][b] = (zeta * zeta * d[a] * d[b] / r2 + zeta * d[a] * d[b] / (r2 * r) -
                    (a == b ? zeta / r : 0.0)) * e;
    *lapg = (zeta * zeta - 2.0 * zeta / r) * e;
    /* d/dx_a [(z^2 - 2z/r) e] = (2 z d_a / r^3) e + (z^2 - 2 z / r)(-z d_a / r) e */
    for (int a = 0; a < 3; ++a)
      glap[a] = (2.0 * zeta / (r2 * r) - zeta * (zeta * zeta - 2.0 * zeta / r) / r) * d[a] * e;
  }
}

/*
 * Values, gradients and Laplacians of all L orbitals at point r.
 * grad is [L][3], lap is [L]; either may be NULL.
 * glap (the gradient of the Laplacian, [L][3]) and hess ([L][3][3]) are only
 * used by the force code; either may be NULL.
 */
void orc_ao_full(const orc_system *s, const double r[3], double *val, double *grad, double *lap,
                 double *hess, double *glap) {
  int mu = 0;
  for (int k = 0; k < s->n_shells; ++k) {
    int a = s->shell_atom[k], l = s->shell_l[k];
    double d[3] = {r[0] - s->R[3 * a], r[1] - s->R[3 * a + 1], r[2] - s->R[3 * a + 2]};
    double g, gg[3], Hg[3][3], lapg, glg[3];
    radial(s->shell_radial[k], s->shell_zeta[k], d, &g, gg, Hg, &lapg, glg);
    for (int c = 0; c < ncomp(l); ++c, ++mu) {
      double P, gP[3], HP[3][3];
      angular(l, c, d, &P, gP);
      angular_hess(l, c, HP);
      val[mu] = P * g;
      if (grad)
        for (int q = 0; q < 3; ++q) grad[3 * mu + q] = gP[q] * g + P * gg[q];
      if (lap) lap[mu] = 2.0 * (gP[0] * gg[0] + gP[1] * gg[1] + gP[2] * gg[2]) + P * lapg;
      if (hess)
        for (int p = 0; p < 3; ++p)
          for (int q = 0; q < 3; ++q)
            hess[9 * mu + 3 * p + q] = HP[p][q] * g + gP[p] * gg[q] + gP[q] * gg[p] + P * Hg[p][q];
      if (glap) {
        /* grad of (2 gP.gg + P lapg); the angular part is harmonic */
        for (int q = 0; q < 3; ++q) {
          double t = 0.0;
          for (int p = 0; p < 3; ++p) t += HP[q][p] * gg[p] + gP[p] * Hg[q][p];
          glap[3 * mu + q] = 2.0 * t + gP[q] * lapg + P * glg[q];
        }
      }
    }
  }
}

void orc_ao(const orc_system *s, const double r[3], double *val, double *grad, double *lap) {
  orc_ao_full(s, r, val, grad, lap, NULL, NULL);
}

/* ------------------------------------------------------------------------ */
/* LU factorisation with partial pivoting (Golub & Van Loan, Alg. 3.4.1)     */
/* ------------------------------------------------------------------------ */
/* a: n x n row-major, overwritten by L\U; piv[k] = row swapped with k.
 * Returns 0 if a zero pivot is met (singular), 1 otherwise. */
static int lu_factor(int n, double *a, int *piv, double *logabs, double *sign) {
  double la = 0.0, sg = 1.0;
  for (int k = 0; k < n; ++k) {
    int p = k;
    double best = fabs(a[k * n + k]);
    for (int i = k + 1; i < n; ++i)
      if (fabs(a[i * n + k]) > best) { best = fabs(a[i * n + k]); p = i; }
    piv[k] = p;
    if (best == 0.0) { *logabs = -INFINITY; *sign = 0.0; return 0; }
    if (p != k) {
      for (int j = 0; j < n; ++j) { double t = a[k * n + j]; a[k * n + j] = a[p * n + j]; a[p * n + j] = t; }
      sg = -sg;
    }
    double ukk = a[k * n + k];
    la += log(fabs(ukk));
    if (ukk < 0) sg = -sg;
    for (int i = k + 1; i < n; ++i) {
      double m = a[i * n + k] / ukk;
      a[i * n + k] = m;
      for (int j = k + 1; j < n; ++j) a[i * n + j] -= m * a[k * n + j];
    }
  }
  *logabs = la;
  *sign = sg;
  return 1;
}

/* inverse from the LU factors: solve A X = I column by column */
static void lu_inverse(int n, const double *lu, const int *piv, double *inv) {
  double *col = (double *)malloc(sizeof(double) * n);
  for (int c = 0; c < n; ++c) {
    for (int i = 0; i < n; ++i) col[i] = (i == c) ? 1.0 : 0.0;
    for (int k = 0; k < n; ++k) { double t = col[k]; col[k] = col[piv[k]]; col[piv[k]] = t; }
    for (int i = 0; i < n; ++i) {           /* forward: L y = P b */
      double s = col[i];
      for (int j = 0; j < i; ++j) s -= lu[i * n + j] * col[j];
      col[i] = s;
    }
    for (int i = n - 1; i >= 0; --i) {      /* backward: U x = y */
      double s = col[i];
      for (int j = i + 1; j < n; ++j) s -= lu[i * n + j] * col[j];
      col[i] = s / lu[i * n + i];
    }
    for (int i = 0; i < n; ++i) inv[i * n + c] = col[i];
  }
  free(col);
}

/* log|det|, sign and (optionally) the inverse of an n x n matrix */
int orc_det_inverse(int n, const double *A, double *logabs, double *sign, double *inv) {
  double *lu = (double *)malloc(sizeof(double) * (n > 0 ? n * n : 1));
  int *piv = (int *)malloc(sizeof(int) * (n > 0 ? n : 1));
  memcpy(lu, A, sizeof(double) * n * n);
  int ok = lu_factor(n, lu, piv, logabs, sign);
  if (ok && inv) lu_inverse(n, lu, piv, inv);
  free(lu);
  free(piv);
  return ok;
}

/* ------------------------------------------------------------------------ */
/* Geminal matrix G~ (n_up x n_up), Eqs. agp_expansion and wfAGPunpaired:     */
/*   G[i][j]        = sum_{mu,nu} phi_mu(r_i^up) lambda_{mu,nu} phi_nu(r_j^dn) */
/*   G[i][n_dn + l] = sum_mu phi_mu(r_i^up) c^{(l)}_mu   (unpaired orbitals)   */
/* phi is [N][L] (up electrons first).                                        */
/* ------------------------------------------------------------------------ */
static double pair_fn(const orc_system *s, const double *pu, const double *pd) {
  /* sum_{mu,nu} pu_mu lambda_{mu nu} pd_nu, done as (pu^T lambda) . pd */
  int L = s->L;
  double tot = 0.0;
  for (int nu = 0; nu < L; ++nu) {
    double t = 0.0;
    for (int mu = 0; mu < L; ++mu) t += pu[mu] * s->lam[mu * L + nu];
    tot += t * pd[nu];
  }
  return tot;
}

static double unpaired_fn(const orc_system *s, int l, const double *pu) {
  double t = 0.0;
  for (int mu = 0; mu < s->L; ++mu) t += s->unpaired[l * s->L + mu] * pu[mu];
  return t;
}

/* row vector a = p^T lambda and column vector b = lambda p (length L) */
static void lam_left(const orc_system *s, const double *p, double *a) {
  int L = s->L;
  for (int nu = 0; nu < L; ++nu) {
    double t = 0.0;
    for (int mu = 0; mu < L; ++mu) t += p[mu] * s->lam[mu * L + nu];
    a[nu] = t;
  }
}
static void lam_right(const orc_system *s, const double *p, double *b) {
  int L = s->L;
  for (int mu = 0; mu < L; ++mu) {
    double t = 0.0;
    for (int nu = 0; nu < L; ++nu) t += s->lam[mu * L + nu] * p[nu];
    b[mu] = t;
  }
}
static double dot(int n, const double *a, const double *b) {
  double t = 0.0;
  for (int i = 0; i < n; ++i) t += a[i] * b[i];
  return t;
}

void orc_geminal(const orc_system *s, const double *phi, double *G) {
  int nu = s->n_up, nd = s->n_dn, L = s->L;
  double *a = (double *)malloc(sizeof(double) * L);
  for (int i = 0; i < nu; ++i) {
    lam_left(s, phi + (size_t)i * L, a);
    for (int j = 0; j < nd; ++j) G[i * nu + j] = dot(L, a, phi + (size_t)(nu + j) * L);
    for (int l = 0; l < nu - nd; ++l) G[i * nu + nd + l] = unpaired_fn(s, l, phi + (size_t)i * L);
  }
  free(a);
}

/* ------------------------------------------------------------------------ */
/* Jastrow factor J = J1 + J2 (Eqs. onebody_J_hom, onebody_u, twobody_v)     */
/* ------------------------------------------------------------------------ */
/* one atom's J1 term f(r) = -c^3 u(c r), c = (2Z)^{1/4}, with f', f'' in r */
static void j1_term(double Z, double b, double r, double *f, double *fp, double *fpp) {
  double c = pow(2.0 * Z, 0.25);
  double s = c * r;
  double u, up, upp;
  if (b == 0.0) { u = 0.5 * s; up = 0.5; upp = 0.0; }  /* the b -> 0 limit */
  else {
    double e = exp(-b * s);
    u = (1.0 - e) / (2.0 * b);
    up = 0.5 * e;
    upp = -0.5 * b * e;
  }
  *f = -c * c * c * u;
  *fp = -c * c * c * c * up;
  *fpp = -c * c * c * c * c * upp;
}

/* derivative of the J1 term with respect to b */
static double j1_term_db(double Z, double b, double r) {
  double c = pow(2.0 * Z, 0.25), s = c * r;
  if (b == 0.0) return -c * c * c * (-s * s / 4.0);
  double e = exp(-b * s);
  double du = s * e / (2.0 * b) - (1.0 - e) / (2.0 * b * b);
  return -c * c * c * du;
}

/* pair term v(r) = r / (k (1 + b r)), k = 4 parallel, 2 antiparallel */
static void j2_term(const orc_system *s, int same_spin, double r, double *v, double *vp, double *vpp,
                    double *vdb) {
  double k = (same_spin && !s->j2_spin_independent) ? 4.0 : 2.0;
  double b = (same_spin && !s->j2_spin_independent) ? s->b_para : s->b_anti;
  double q = 1.0 + b * r;
  *v = r / (k * q);
  *vp = 1.0 / (k * q * q);
  *vpp = -2.0 * b / (k * q * q * q);
  if (vdb) *vdb = -r * r / (k * q * q);
}

static int is_up(const orc_system *s, int i) { return i < s->n_up; }

/* the Jastrow basis chi at r (values, gradients [LJ][3], Laplacians; the last
 * two may be NULL), evaluated by orc_ao on the Jastrow shells */
static void jastrow_basis(const orc_system *s, const double r[3], double *val, double *grad, double *lap) {
  orc_system t = *s;
  t.n_shells = s->n_jshells;
  t.shell_atom = s->jshell_atom;
  t.shell_l = s->jshell_l;
  t.shell_radial = s->jshell_radial;
  t.shell_zeta = s->jshell_zeta;
  t.L = s->LJ;
  orc_ao(&t, r, val, grad, lap);
}

/* J3 = sum_{i<j} sum_{mu,nu} M^{s_i s_j}_{mu,nu} chi_mu(r_i) chi_nu(r_j), M = j3_para for
 * equal spins and j3_anti otherwise (Eq. threebody_jastrow), as the pair sum itself */
static double jastrow3(const orc_system *s, const double *x) {
  int N = s->n_up + s->n_dn, LJ = s->LJ;
  double *chi = (double *)malloc(sizeof(double) * (size_t)N * LJ);
  for (int i = 0; i < N; ++i) jastrow_basis(s, x + 3 * i, chi + (size_t)i * LJ, NULL, NULL);
  double J = 0.0;
  for (int i = 0; i < N; ++i)
    for (int j = i + 1; j < N; ++j) {
      const double *M = is_up(s, i) == is_up(s, j) ? s->j3_para : s->j3_anti;
      for (int mu = 0; mu < LJ; ++mu)
        for (int nu = 0; nu < LJ; ++nu)
          J += M[mu * LJ + nu] * chi[(size_t)i * LJ + mu] * chi[(size_t)j * LJ + nu];
    }
  free(chi);
  return J;
}

double orc_jastrow(const orc_system *s, const double *x) {
  int N = s->n_up + s->n_dn;
  double J = 0.0, f, fp, fpp, vdb;
  if (s->use_j1)
    for (int i = 0; i < N; ++i)
      for (int a = 0; a < s->n_atoms; ++a) {
        double d0 = x[3 * i] - s->R[3 * a], d1 = x[3 * i + 1] - s->R[3 * a + 1], d2 = x[3 * i + 2] - s->R[3 * a + 2];
        j1_term(s->Z[a], s->b_ea, sqrt(d0 * d0 + d1 * d1 + d2 * d2), &f, &fp, &fpp);
        J += f;
      }
  if (s->use_j2)
    for (int i = 0; i < N; ++i)
      for (int j = i + 1; j < N; ++j) {
        double d0 = x[3 * i] - x[3 * j], d1 = x[3 * i + 1] - x[3 * j + 1], d2 = x[3 * i + 2] - x[3 * j + 2];
        j2_term(s, is_up(s, i) == is_up(s, j), sqrt(d0 * d0 + d1 * d1 + d2 * d2), &f, &fp, &fpp, &vdb);
        J += f;
      }
  if (s->use_j3) J += jastrow3(s, x);
  return J;
}

/* gradient [N][3] and Laplacian [N] of J with respect to each electron */
void orc_jastrow_derivs(const orc_system *s, const double *x, double *gJ, double *lJ) {
  int N = s->n_up + s->n_dn;
  memset(gJ, 0, sizeof(double) * 3 * N);
  memset(lJ, 0, sizeof(double) * N);
  double f, fp, fpp;
  if (s->use_j1)
    for (int i = 0; i < N; ++i)
      for (int a = 0; a < s->n_atoms; ++a) {
        double d[3];
        for (int q = 0; q < 3; ++q) d[q] = x[3 * i + q] - s->R[3 * a + q];
        double r = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
        j1_term(s->Z[a], s->b_ea, r, &f, &fp, &fpp);
        for (int q = 0; q < 3; ++q) gJ[3 * i + q] += fp * d[q] / r;
        lJ[i] += fpp + 2.0 * fp / r;
      }
  if (s->use_j2)
    for (int i = 0; i < N; ++i)
      for (int j = 0; j < N; ++j) {
        if (j == i) continue;
        double d[3];
        for (int q = 0; q < 3; ++q) d[q] = x[3 * i + q] - x[3 * j + q];
        double r = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
        j2_term(s, is_up(s, i) == is_up(s, j), r, &f, &fp, &fpp, NULL);
        for (int q = 0; q < 3; ++q) gJ[3 * i + q] += fp * d[q] / r;
        lJ[i] += fpp + 2.0 * fp / r;
      }
  if (s->use_j3) {
    /* d/dr_i of sum_{j != i} chi(r_i)^T M^{s_i s_j} chi(r_j) (M symmetric) */
    int LJ = s->LJ;
    double *chi = (double *)malloc(sizeof(double) * (size_t)N * LJ);
    double *gch = (double *)malloc(sizeof(double) * (size_t)N * LJ * 3);
    double *lch = (double *)malloc(sizeof(double) * (size_t)N * LJ);
    for (int i = 0; i < N; ++i)
      jastrow_basis(s, x + 3 * i, chi + (size_t)i * LJ, gch + (size_t)i * LJ * 3, lch + (size_t)i * LJ);
    for (int i = 0; i < N; ++i)
      for (int j = 0; j < N; ++j) {
        if (j == i) continue;
        const double *M = is_up(s, i) == is_up(s, j) ? s->j3_para : s->j3_anti;
        for (int mu = 0; mu < LJ; ++mu)
          for (int nu = 0; nu < LJ; ++nu) {
            double m = M[mu * LJ + nu] * chi[(size_t)j * LJ + nu];
            for (int q = 0; q < 3; ++q) gJ[3 * i + q] += m * gch[((size_t)i * LJ + mu) * 3 + q];
            lJ[i] += m * lch[(size_t)i * LJ + mu];
          }
      }
    free(chi);
    free(gch);
    free(lch);
  }
}

/* ------------------------------------------------------------------------ */
/* log|Psi| and its sign                                                      */
/* out: [0] log|Psi|, [1] sign(Psi), [2] log|det G~|, [3] J                   */
/* ------------------------------------------------------------------------ */
int orc_logpsi(const orc_system *s, const double *x, double *out) {
  int N = s->n_up + s->n_dn, L = s->L, nu = s->n_up;
  double *phi = (double *)malloc(sizeof(double) * (size_t)N * L);
  double *G = (double *)malloc(sizeof(double) * nu * nu);
  for (int i = 0; i < N; ++i) orc_ao(s, x + 3 * i, phi + (size_t)i * L, NULL, NULL);
  orc_geminal(s, phi, G);
  double la, sg;
  int ok = orc_det_inverse(nu, G, &la, &sg, NULL);
  double J = orc_jastrow(s, x);
  out[0] = la + J;
  out[1] = sg;
  out[2] = la;
  out[3] = J;
  free(phi);
  free(G);
  return ok;
}

/* ------------------------------------------------------------------------ */
/* Local energy e_L = (H Psi)/Psi in Hartree atomic units (Sec. VMC).         */
/*   H = -1/2 sum_i lap_i - sum_{i,a} Z_a/|r_i-R_a| + sum_{i<j} 1/r_ij          */
/*       + sum_{a<b} Z_a Z_b/R_ab                                              */
/* For Psi = D e^J:  lap_i Psi / Psi = lap_i D/D + 2 grad_i D/D . grad_i J     */
/*                                     + lap_i J + |grad_i J|^2                */
/* D = det G~ is linear in each row (up electron) and each column (down        */
/* electron), so grad_i D / D = sum_j Ginv[j][i] grad_i G[i][j] for an up     */
/* electron, the column analogue for a down electron, and the same with the    */
/* Laplacian (Jacobi's formula; no term is second order in one row).          */
/* out: [0] e_L, [1] kinetic, [2] V_ee, [3] V_ei, [4] V_ii                    */
/* gD (optional, [N][3]) receives grad_i D / D, lD ([N]) lap_i D / D.          */
/* ------------------------------------------------------------------------ */
static int det_derivs(const orc_system *s, const double *x, const double *phi, const double *gphi,
                      const double *lphi, const double *Ginv, double *gD, double *lD) {
  int N = s->n_up + s->n_dn, L = s->L, nu = s->n_up, nd = s->n_dn;
  /* Bcol[j] = d G[i][j] / d phi(r_i): lambda phi(r_j^dn) for j < n_dn, c^{(j-n_dn)} otherwise.
     Arow[i] = d G[i][j] / d phi(r_j^dn): phi(r_i^up)^T lambda. */
  double *Bcol = (double *)malloc(sizeof(double) * (size_t)nu * L);
  double *Arow = (double *)malloc(sizeof(double) * (size_t)nu * L);
  (void)x;
  for (int j = 0; j < nu; ++j) {
    if (j < nd) lam_right(s, phi + (size_t)(nu + j) * L, Bcol + (size_t)j * L);
    else memcpy(Bcol + (size_t)j * L, s->unpaired + (size_t)(j - nd) * L, sizeof(double) * L);
  }
  for (int i = 0; i < nu; ++i) lam_left(s, phi + (size_t)i * L, Arow + (size_t)i * L);
  for (int i = 0; i < N; ++i) {
    gD[3 * i] = gD[3 * i + 1] = gD[3 * i + 2] = 0.0;
    lD[i] = 0.0;
  }
  /* up electron i, entries G[i][j]: the derivative acts on phi(r_i) */
  for (int i = 0; i < nu; ++i)
    for (int j = 0; j < nu; ++j) {
      double w = Ginv[j * nu + i];
      const double *col = Bcol + (size_t)j * L;
      for (int mu = 0; mu < L; ++mu) {
        for (int q = 0; q < 3; ++q) gD[3 * i + q] += w * gphi[((size_t)i * L + mu) * 3 + q] * col[mu];
        lD[i] += w * lphi[(size_t)i * L + mu] * col[mu];
      }
    }
  /* down electron j, entries G[i][j]: the derivative acts on phi(r_j) */
  for (int j = 0; j < nd; ++j) {
    int e = nu + j;
    for (int i = 0; i < nu; ++i) {
      double w = Ginv[j * nu + i];
      const double *a = Arow + (size_t)i * L;
      for (int m = 0; m < L; ++m) {
        for (int q = 0; q < 3; ++q) gD[3 * e + q] += w * a[m] * gphi[((size_t)e * L + m) * 3 + q];
        lD[e] += w * a[m] * lphi[(size_t)e * L + m];
      }
    }
  }
  free(Bcol);
  free(Arow);
  return 1;
}

static void potentials(const orc_system *s, const double *x, double *vee, double *vei, double *vii) {
  int N = s->n_up + s->n_dn;
  double ee = 0, ei = 0, ii = 0;
  for (int i = 0; i < N; ++i)
    for (int j = i + 1; j < N; ++j) {
      double d0 = x[3 * i] - x[3 * j], d1 = x[3 * i + 1] - x[3 * j + 1], d2 = x[3 * i + 2] - x[3 * j + 2];
      ee += 1.0 / sqrt(d0 * d0 + d1 * d1 + d2 * d2);
    }
  for (int i = 0; i < N; ++i)
    for (int a = 0; a < s->n_atoms; ++a) {
      double d0 = x[3 * i] - s->R[3 * a], d1 = x[3 * i + 1] - s->R[3 * a + 1], d2 = x[3 * i + 2] - s->R[3 * a + 2];
      ei -= s->Z[a] / sqrt(d0 * d0 + d1 * d1 + d2 * d2);
    }
  for (int a = 0; a < s->n_atoms; ++a)
    for (int b = a + 1; b < s->n_atoms; ++b) {
      double d0 = s->R[3 * a] - s->R[3 * b], d1 = s->R[3 * a + 1] - s->R[3 * b + 1], d2 = s->R[3 * a + 2] - s->R[3 * b + 2];
      ii += s->Z[a] * s->Z[b] / sqrt(d0 * d0 + d1 * d1 + d2 * d2);
    }
  *vee = ee;
  *vei = ei;
  *vii = ii;
}

int orc_local_energy_ex(const orc_system *s, const double *x, double *out, double *gD_out, double *lD_out) {
  int N = s->n_up + s->n_dn, L = s->L, nu = s->n_up;
  double *phi = (double *)malloc(sizeof(double) * (size_t)N * L);
  double *gphi = (double *)malloc(sizeof(double) * (size_t)N * L * 3);
  double *lphi = (double *)malloc(sizeof(double) * (size_t)N * L);
  double *G = (double *)malloc(sizeof(double) * nu * nu);
  double *Ginv = (double *)malloc(sizeof(double) * nu * nu);
  double *gD = (double *)malloc(sizeof(double) * 3 * N);
  double *lD = (double *)malloc(sizeof(double) * N);
  double *gJ = (double *)malloc(sizeof(double) * 3 * N);
  double *lJ = (double *)malloc(sizeof(double) * N);
  for (int i = 0; i < N; ++i)
    orc_ao(s, x + 3 * i, phi + (size_t)i * L, gphi + (size_t)i * L * 3, lphi + (size_t)i * L);
  orc_geminal(s, phi, G);
  double la, sg;
  int ok = orc_det_inverse(nu, G, &la, &sg, Ginv);
  if (ok) {
    det_derivs(s, x, phi, gphi, lphi, Ginv, gD, lD);
    orc_jastrow_derivs(s, x, gJ, lJ);
    double kin = 0.0;
    for (int i = 0; i < N; ++i) {
      double t = lD[i] + lJ[i];
      for (int q = 0; q < 3; ++q) t += 2.0 * gD[3 * i + q] * gJ[3 * i + q] + gJ[3 * i + q] * gJ[3 * i + q];
      kin += -0.5 * t;
    }
    double vee, vei, vii;
    potentials(s, x, &vee, &vei, &vii);
    out[0] = kin + vee + vei + vii;
    out[1] = kin;
    out[2] = vee;
    out[3] = vei;
    out[4] = vii;
    if (gD_out) memcpy(gD_out, gD, sizeof(double) * 3 * N);
    if (lD_out) memcpy(lD_out, lD, sizeof(double) * N);
  } else {
    for (int q = 0; q < 5; ++q) out[q] = NAN;
  }
  free(phi); free(gphi); free(lphi); free(G); free(Ginv);
  free(gD); free(lD); free(gJ); free(lJ);
  return ok;
}

int orc_local_energy(const orc_system *s, const double *x, double *out) {
  return orc_local_energy_ex(s, x, out, NULL, NULL);
}

/* batched helpers over W configurations [W][N][3] */
int orc_local_energy_batch(const orc_system *s, const double *x, int W, double *eL) {
  int N = s->n_up + s->n_dn, bad = 0;
#pragma omp parallel for schedule(dynamic) reduction(+ : bad)
  for (int w = 0; w < W; ++w) {
    double out[5];
    if (!orc_local_energy(s, x + (size_t)w * N * 3, out)) bad++;
    eL[w] = out[0];
  }
  return bad == 0;
}

int orc_logpsi_batch(const orc_system *s, const double *x, int W, double *logabs, double *sign) {
  int N = s->n_up + s->n_dn, bad = 0;
#pragma omp parallel for schedule(dynamic) reduction(+ : bad)
  for (int w = 0; w < W; ++w) {
    double out[4];
    if (!orc_logpsi(s, x + (size_t)w * N * 3, out)) bad++;
    logabs[w] = out[0];
    sign[w] = out[1];
  }
  return bad == 0;
}

/* ------------------------------------------------------------------------ */
/* Sherman-Morrison row/column replacement (used only by the pin tests that  */
/* check it against full determinant recomputation).                          */
/* ------------------------------------------------------------------------ */
/* ratio det(G')/det(G) when row i of G becomes newrow: sum_j newrow_j Ginv[j][i] */
double orc_sm_ratio_row(int n, const double *Ginv, int i, const double *newrow) {
  double t = 0.0;
  for (int j = 0; j < n; ++j) t += newrow[j] * Ginv[j * n + i];
  return t;
}
/* Ginv' = Ginv - (Ginv e_i)(newrow^T Ginv - e_i^T) / ratio */
void orc_sm_update_row(int n, double *Ginv, int i, const double *newrow) {
  double *v = (double *)malloc(sizeof(double) * n), *c = (double *)malloc(sizeof(double) * n);
  for (int k = 0; k < n; ++k) {
    double t = 0.0;
    for (int j = 0; j < n; ++j) t += newrow[j] * Ginv[j * n + k];
    v[k] = t;
  }
  double R = v[i];
  for (int j = 0; j < n; ++j) c[j] = Ginv[j * n + i];
  for (int j = 0; j < n; ++j)
    for (int k = 0; k < n; ++k) Ginv[j * n + k] -= c[j] * (v[k] - (k == i ? 1.0 : 0.0)) / R;
  free(v);
  free(c);
}

/* ------------------------------------------------------------------------ */
/* Variational Monte Carlo (Sec. VMC), single-electron Metropolis.            */
/* The move of electron e in sweep t of walker w draws one Philox4x32-10      */
/* block: counter = (w, t, e, 1), key = (seed low 32 bits, seed high 32).     */
/* x0..x2 give the proposal r' = r + delta (2u - 1), u = (x + 1/2) 2^-32,     */
/* computed as fma(delta, (x + 1/2) 2^-31 - 1, r); x3 gives the acceptance    */
/* draw u_acc = x3 2^-32, and the move is accepted iff                       */
/* u_acc < |Psi(x')/Psi(x)|^2.  Electrons move in the order 0..N-1 (up first). */
/* The determinant ratio is taken from a full LU of the updated matrix        */
/* (definition; no Sherman-Morrison) and the Jastrow difference from a full   */
/* recomputation of J.                                                        */
/* ------------------------------------------------------------------------ */
void orc_move_draws(uint64_t seed, uint32_t walker, uint32_t sweep, uint32_t electron, double delta,
                    const double r[3], double rp[3], double *u_acc) {
  uint32_t ctr[4] = {walker, sweep, electron, 1u};
  uint32_t key[2] = {(uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32)};
  uint32_t o[4];
  orc_philox4x32_10(ctr, key, o);
  for (int k = 0; k < 3; ++k) {
    double t = ((double)o[k] + 0.5) * 0x1p-31 - 1.0;
    rp[k] = fma(delta, t, r[k]);
  }
  *u_acc = (double)o[3] * 0x1p-32;
}

/* ------------------------------------------------------------------------ */
/* Guiding function (Sec. "Atomic forces", Eqs. guiding_function, R_r,        */
/* regularization, reweighting): from G~ and its inverse,                    */
/*   R = (S sum_{ij} |G~^{-1}_ij|^2)^{-theta},  S = min_i sum_j |G~_ij|^2,   */
/* Psi_G = (R^eps / R) Psi_T with R^eps = max(R, eps), and the weight       */
/* W = (Psi_T / Psi_G)^2 = (R / max(R, eps))^2.                            */
/* ------------------------------------------------------------------------ */
static double guiding_R(int n, const double *G, const double *Ginv, double theta) {
  double f = 0.0, S = INFINITY;
  for (int i = 0; i < n; ++i) {
    double rs = 0.0;
    for (int j = 0; j < n; ++j) {
      rs += G[i * n + j] * G[i * n + j];
      f += Ginv[i * n + j] * Ginv[i * n + j];
    }
    if (rs < S) S = rs;
  }
  return pow(S * f, -theta);
}

static double guiding_W(double R, double eps) {
  double q = R / (R > eps ? R : eps);
  return q * q;
}

/* R of one configuration (0 if G~ is singular) */
double orc_guiding_R(const orc_system *s, const double *x, double theta) {
  int N = s->n_up + s->n_dn, L = s->L, nu = s->n_up;
  double *phi = (double *)malloc(sizeof(double) * (size_t)N * L);
  double *G = (double *)malloc(sizeof(double) * nu * nu), *Gi = (double *)malloc(sizeof(double) * nu * nu);
  for (int i = 0; i < N; ++i) orc_ao(s, x + 3 * i, phi + (size_t)i * L, NULL, NULL);
  orc_geminal(s, phi, G);
  double la, sg, R = 0.0;
  if (orc_det_inverse(nu, G, &la, &sg, Gi)) R = guiding_R(nu, G, Gi, theta);
  free(phi); free(G); free(Gi);
  return R;
}

static int vmc_walker(const orc_system *s, double *x, uint32_t wid, uint64_t seed, uint32_t sweep0,
                      int nsweeps, double delta, double *eL_out, int W_stride, int w,
                      double *logpsi_out, long long *n_acc_out, double theta, double eps, double *R_out) {
  int N = s->n_up + s->n_dn, L = s->L, nu = s->n_up, nd = s->n_dn;
  double *phi = (double *)malloc(sizeof(double) * (size_t)N * L);
  double *G = (double *)malloc(sizeof(double) * nu * nu);
  double *Gp = (double *)malloc(sizeof(double) * nu * nu);
  double *pnew = (double *)malloc(sizeof(double) * L);
  double *vec = (double *)malloc(sizeof(double) * L);
  double *xp = (double *)malloc(sizeof(double) * 3 * N);
  /* guided sampling (eps > 0): inverses for R of the current and the proposed configuration */
  const int guided = eps > 0.0;
  double *Gi = (double *)malloc(sizeof(double) * nu * nu), *Gpi = (double *)malloc(sizeof(double) * nu * nu);
  for (int i = 0; i < N; ++i) orc_ao(s, x + 3 * i, phi + (size_t)i * L, NULL, NULL);
  orc_geminal(s, phi, G);
  double logdet, sgn;
  int ok = orc_det_inverse(nu, G, &logdet, &sgn, Gi);
  double J = orc_jastrow(s, x);
  double Wcur = ok && guided ? guiding_W(guiding_R(nu, G, Gi, theta), eps) : 1.0;
  long long nacc = 0;
  for (int t = 0; t < nsweeps && ok; ++t) {
    uint32_t sweep = sweep0 + (uint32_t)t;
    for (int e = 0; e < N; ++e) {
      double rp[3], uacc;
      orc_move_draws(seed, wid, sweep, (uint32_t)e, delta, x + 3 * e, rp, &uacc);
      orc_ao(s, rp, pnew, NULL, NULL);
      memcpy(Gp, G, sizeof(double) * nu * nu);
      if (e < nu) {                       /* new row e of G~ */
        lam_left(s, pnew, vec);
        for (int j = 0; j < nd; ++j) Gp[e * nu + j] = dot(L, vec, phi + (size_t)(nu + j) * L);
        for (int l = 0; l < nu - nd; ++l) Gp[e * nu + nd + l] = unpaired_fn(s, l, pnew);
      } else {                            /* new column (e - n_up) of G~ */
        int j = e - nu;
        lam_right(s, pnew, vec);
        for (int i = 0; i < nu; ++i) Gp[i * nu + j] = dot(L, phi + (size_t)i * L, vec);
      }
      double logdet_p, sgn_p;
      int okp = orc_det_inverse(nu, Gp, &logdet_p, &sgn_p, guided ? Gpi : NULL);
      memcpy(xp, x, sizeof(double) * 3 * N);
      xp[3 * e] = rp[0]; xp[3 * e + 1] = rp[1]; xp[3 * e + 2] = rp[2];
      double Jp = orc_jastrow(s, xp);
      double p = okp ? exp(2.0 * (logdet_p - logdet) + 2.0 * (Jp - J)) : 0.0;
      /* |Psi_G(x')/Psi_G(x)|^2 = |Psi_T(x')/Psi_T(x)|^2 W(x) / W(x') */
      double Wp = 1.0;
      if (guided && okp) {
        Wp = guiding_W(guiding_R(nu, Gp, Gpi, theta), eps);
        p *= Wcur / Wp;
      }
      if (uacc < p) {
        memcpy(x + 3 * e, rp, sizeof(double) * 3);
        memcpy(phi + (size_t)e * L, pnew, sizeof(double) * L);
        memcpy(G, Gp, sizeof(double) * nu * nu);
        logdet = logdet_p;
        sgn = sgn_p;
        J = Jp;
        Wcur = Wp;
        nacc++;
      }
    }
    if (eL_out) {
      double out[5];
      orc_local_energy(s, x, out);
      eL_out[(size_t)t * W_stride + w] = out[0];
    }
  }
  if (logpsi_out) logpsi_out[w] = logdet + J;
  if (n_acc_out) n_acc_out[w] = nacc;
  if (R_out) R_out[w] = ok ? orc_guiding_R(s, x, theta > 0.0 ? theta : 0.375) : 0.0;
  (void)sgn;
  free(phi); free(G); free(Gp); free(pnew); free(vec); free(xp); free(Gi); free(Gpi);
  return ok;
}

/* x: [W][N][3] in/out.  eL_out: [nsweeps][W] or NULL (local energy after each
 * sweep).  logpsi_out: [W] or NULL.  n_acc: [W] or NULL.  Walker w uses the
 * Philox walker index walker0 + w.  nthreads <= 0 uses the OpenMP default. */
int orc_vmc(const orc_system *s, double *x, int W, long long walker0, uint64_t seed, long long sweep0,
            int nsweeps, double delta, double *eL_out, double *logpsi_out, long long *n_acc, int nthreads) {
  int N = s->n_up + s->n_dn, bad = 0;
#ifdef _OPENMP
  if (nthreads > 0) omp_set_num_threads(nthreads);
#else
  (void)nthreads;
#endif
#pragma omp parallel for schedule(dynamic) reduction(+ : bad)
  for (int w = 0; w < W; ++w)
    if (!vmc_walker(s, x + (size_t)w * N * 3, (uint32_t)(walker0 + w), seed, (uint32_t)sweep0, nsweeps,
                    delta, eL_out, W, w, logpsi_out, n_acc, 0.0, 0.0, NULL))
      bad++;
  return bad == 0;
}

/* orc_vmc sampling the guiding function Psi_G = (max(R, eps) / R) Psi_T
 * (Eq. guiding_function) instead of Psi_T: the acceptance probability is
 * |Psi_T(x')/Psi_T(x)|^2 W(x) / W(x').  R_out [W] (may be NULL) receives R of
 * each walker's final configuration. */
int orc_vmc_guided(const orc_system *s, double *x, int W, long long walker0, uint64_t seed, long long sweep0,
                   int nsweeps, double delta, double theta, double eps, double *eL_out, double *logpsi_out,
                   long long *n_acc, double *R_out, int nthreads) {
  int N = s->n_up + s->n_dn, bad = 0;
#ifdef _OPENMP
  if (nthreads > 0) omp_set_num_threads(nthreads);
#else
  (void)nthreads;
#endif
#pragma omp parallel for schedule(dynamic) reduction(+ : bad)
  for (int w = 0; w < W; ++w)
    if (!vmc_walker(s, x + (size_t)w * N * 3, (uint32_t)(walker0 + w), seed, (uint32_t)sweep0, nsweeps,
                    delta, eL_out, W, w, logpsi_out, n_acc, theta, eps, R_out))
      bad++;
  return bad == 0;
}

int orc_max_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

/* ------------------------------------------------------------------------ */
/* Log-derivatives O_k = d ln|Psi| / d alpha_k (Sec. "Derivatives of energy")  */
/*   d/d lambda_{mu,nu}: sum_{i, j<n_dn} Ginv[j][i] phi_mu(r_i) phi_nu(r_j)     */
/*                       (every entry of lambda taken as independent)          */
/*   d/d b_ea, b_para, b_anti: Jastrow parameter derivatives                   */
/*   d/d R_a: orbitals on atom a depend on r - R_a (d/dR_a = -d/dr), plus J1   */
/*   d/d r_i: grad_i D / D + grad_i J                                          */
/* dlam: [L][L] (may be NULL), djas: [3], dR: [n_atoms][3], dr: [N][3] (NULL ok) */
/* ------------------------------------------------------------------------ */
int orc_grad_logpsi(const orc_system *s, const double *x, double *dlam, double *djas, double *dR,
                    double *dr) {
  int N = s->n_up + s->n_dn, L = s->L, nu = s->n_up, nd = s->n_dn;
  double *phi = (double *)malloc(sizeof(double) * (size_t)N * L);
  double *gphi = (double *)malloc(sizeof(double) * (size_t)N * L * 3);
  double *lphi = (double *)malloc(sizeof(double) * (size_t)N * L);
  double *G = (double *)malloc(sizeof(double) * nu * nu);
  double *Ginv = (double *)malloc(sizeof(double) * nu * nu);
  double *a = (double *)malloc(sizeof(double) * L);
  double *col = (double *)malloc(sizeof(double) * L);
  int *owner = (int *)malloc(sizeof(int) * L);
  for (int k = 0, mu = 0; k < s->n_shells; ++k)
    for (int c = 0; c < ncomp(s->shell_l[k]); ++c) owner[mu++] = s->shell_atom[k];
  for (int i = 0; i < N; ++i)
    orc_ao(s, x + 3 * i, phi + (size_t)i * L, gphi + (size_t)i * L * 3, lphi + (size_t)i * L);
  orc_geminal(s, phi, G);
  double la, sg;
  int ok = orc_det_inverse(nu, G, &la, &sg, Ginv);
  if (!ok) goto done;
  if (dlam) {
    for (int mu = 0; mu < L; ++mu)
      for (int n2 = 0; n2 < L; ++n2) {
        double t = 0.0;
        for (int i = 0; i < nu; ++i)
          for (int j = 0; j < nd; ++j) t += Ginv[j * nu + i] * phi[(size_t)i * L + mu] * phi[(size_t)(nu + j) * L + n2];
        dlam[mu * L + n2] = t;
      }
  }
  if (djas) {
    djas[0] = djas[1] = djas[2] = 0.0;
    if (s->use_j1)
      for (int i = 0; i < N; ++i)
        for (int at = 0; at < s->n_atoms; ++at) {
          double d0 = x[3 * i] - s->R[3 * at], d1 = x[3 * i + 1] - s->R[3 * at + 1], d2 = x[3 * i + 2] - s->R[3 * at + 2];
          djas[0] += j1_term_db(s->Z[at], s->b_ea, sqrt(d0 * d0 + d1 * d1 + d2 * d2));
        }
    if (s->use_j2)
      for (int i = 0; i < N; ++i)
        for (int j = i + 1; j < N; ++j) {
          double d0 = x[3 * i] - x[3 * j], d1 = x[3 * i + 1] - x[3 * j + 1], d2 = x[3 * i + 2] - x[3 * j + 2];
          double v, vp, vpp, vdb;
          int same = is_up(s, i) == is_up(s, j);
          j2_term(s, same, sqrt(d0 * d0 + d1 * d1 + d2 * d2), &v, &vp, &vpp, &vdb);
          if (same && !s->j2_spin_independent) djas[1] += vdb;
          else djas[2] += vdb;
        }
  }
  if (dR) {
    memset(dR, 0, sizeof(double) * 3 * s->n_atoms);
    /* determinant part: sum_{i,j} Ginv[j][i] dG[i][j]/dR_a, where an orbital
       on atom a depends on r - R_a so that d/dR_a = -d/dr */
    double *Bcol = (double *)malloc(sizeof(double) * (size_t)nu * L);
    double *Arow = (double *)malloc(sizeof(double) * (size_t)nu * L);
    for (int j = 0; j < nu; ++j) {
      if (j < nd) lam_right(s, phi + (size_t)(nu + j) * L, Bcol + (size_t)j * L);
      else memcpy(Bcol + (size_t)j * L, s->unpaired + (size_t)(j - nd) * L, sizeof(double) * L);
    }
    for (int i = 0; i < nu; ++i) lam_left(s, phi + (size_t)i * L, Arow + (size_t)i * L);
    for (int i = 0; i < nu; ++i)
      for (int j = 0; j < nu; ++j) {
        double w = Ginv[j * nu + i];
        for (int mu = 0; mu < L; ++mu)
          for (int q = 0; q < 3; ++q) {
            dR[3 * owner[mu] + q] -= w * gphi[((size_t)i * L + mu) * 3 + q] * Bcol[(size_t)j * L + mu];
            if (j < nd)
              dR[3 * owner[mu] + q] -= w * Arow[(size_t)i * L + mu] * gphi[((size_t)(nu + j) * L + mu) * 3 + q];
          }
      }
    free(Bcol);
    free(Arow);
    if (s->use_j1)
      for (int i = 0; i < N; ++i)
        for (int at = 0; at < s->n_atoms; ++at) {
          double d[3], f, fp, fpp;
          for (int q = 0; q < 3; ++q) d[q] = x[3 * i + q] - s->R[3 * at + q];
          double r = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
          j1_term(s->Z[at], s->b_ea, r, &f, &fp, &fpp);
          for (int q = 0; q < 3; ++q) dR[3 * at + q] -= fp * d[q] / r;
        }
    if (s->use_j3) {
      /* chi_mu on atom a depends on r - R_a: d/dR_a = -d/dr on its functions */
      int LJ = s->LJ;
      int *jowner = (int *)malloc(sizeof(int) * LJ);
      for (int k = 0, mu = 0; k < s->n_jshells; ++k)
        for (int c = 0; c < ncomp(s->jshell_l[k]); ++c) jowner[mu++] = s->jshell_atom[k];
      double *chi = (double *)malloc(sizeof(double) * (size_t)N * LJ);
      double *gch = (double *)malloc(sizeof(double) * (size_t)N * LJ * 3);
      for (int i = 0; i < N; ++i) jastrow_basis(s, x + 3 * i, chi + (size_t)i * LJ, gch + (size_t)i * LJ * 3, NULL);
      for (int i = 0; i < N; ++i)
        for (int j = 0; j < N; ++j) {
          if (j == i) continue;
          const double *M = is_up(s, i) == is_up(s, j) ? s->j3_para : s->j3_anti;
          for (int mu = 0; mu < LJ; ++mu)
            for (int nu = 0; nu < LJ; ++nu) {
              double m = M[mu * LJ + nu] * chi[(size_t)j * LJ + nu];
              for (int q = 0; q < 3; ++q) dR[3 * jowner[mu] + q] -= m * gch[((size_t)i * LJ + mu) * 3 + q];
            }
        }
      free(jowner);
      free(chi);
      free(gch);
    }
  }
  if (dr) {
    double *gD = (double *)malloc(sizeof(double) * 3 * N), *lD = (double *)malloc(sizeof(double) * N);
    double *gJ = (double *)malloc(sizeof(double) * 3 * N), *lJ = (double *)malloc(sizeof(double) * N);
    det_derivs(s, x, phi, gphi, lphi, Ginv, gD, lD);
    orc_jastrow_derivs(s, x, gJ, lJ);
    for (int q = 0; q < 3 * N; ++q) dr[q] = gD[q] + gJ[q];
    free(gD); free(lD); free(gJ); free(lJ);
  }
done:
  free(phi); free(gphi); free(lphi); free(G); free(Ginv); free(a); free(col); free(owner);
  return ok;
}

/* ------------------------------------------------------------------------ */
/* Reference derivatives of the local energy with respect to the nuclear     */
/* positions R_a and the electron positions r_i (the ingredients of the      */
/* Hellmann-Feynman + Pulay force of Eq. forces:aad without the space warp): */
/* central differences of orc_local_energy, Richardson-extrapolated          */
/*   D(h) = (e(+h) - e(-h)) / 2h,  D = (4 D(h/2) - D(h)) / 3   (error O(h^4)) */
/* dR: [n_atoms][3] (may be NULL), dr: [N][3] (may be NULL).                 */
/* ------------------------------------------------------------------------ */
static double el_at(const orc_system *s, const double *x) {
  double out[5];
  orc_local_energy(s, x, out);
  return out[0];
}

int orc_elocal_grad_fd(const orc_system *s, const double *x, double h, double *dR, double *dr) {
  int N = s->n_up + s->n_dn;
  double *xx = (double *)malloc(sizeof(double) * 3 * N);
  double *RR = (double *)malloc(sizeof(double) * 3 * s->n_atoms);
  orc_system t = *s;
  t.R = RR;
  memcpy(xx, x, sizeof(double) * 3 * N);
  memcpy(RR, s->R, sizeof(double) * 3 * s->n_atoms);
  const double hs[2] = {h, 0.5 * h};
  if (dr)
    for (int q = 0; q < 3 * N; ++q) {
      double D[2];
      for (int k = 0; k < 2; ++k) {
        xx[q] = x[q] + hs[k];
        double ep = el_at(s, xx);
        xx[q] = x[q] - hs[k];
        double em = el_at(s, xx);
        xx[q] = x[q];
        D[k] = (ep - em) / (2.0 * hs[k]);
      }
      dr[q] = (4.0 * D[1] - D[0]) / 3.0;
    }
  if (dR)
    for (int q = 0; q < 3 * s->n_atoms; ++q) {
      double D[2];
      for (int k = 0; k < 2; ++k) {
        RR[q] = s->R[q] + hs[k];
        double ep = el_at(&t, x);
        RR[q] = s->R[q] - hs[k];
        double em = el_at(&t, x);
        RR[q] = s->R[q];
        D[k] = (ep - em) / (2.0 * hs[k]);
      }
      dR[q] = (4.0 * D[1] - D[0]) / 3.0;
    }
  free(xx);
  free(RR);
  return 1;
}

/* the same for one entry lambda_{mu,nu} (every entry independent) */
double orc_elocal_dlambda_fd(const orc_system *s, const double *x, int mu, int nu, double h) {
  int L = s->L;
  double *lam = (double *)malloc(sizeof(double) * (size_t)L * L);
  memcpy(lam, s->lam, sizeof(double) * (size_t)L * L);
  orc_system t = *s;
  t.lam = lam;
  const double hs[2] = {h, 0.5 * h};
  double D[2];
  for (int k = 0; k < 2; ++k) {
    lam[(size_t)mu * L + nu] = s->lam[(size_t)mu * L + nu] + hs[k];
    double ep = el_at(&t, x);
    lam[(size_t)mu * L + nu] = s->lam[(size_t)mu * L + nu] - hs[k];
    double em = el_at(&t, x);
    lam[(size_t)mu * L + nu] = s->lam[(size_t)mu * L + nu];
    D[k] = (ep - em) / (2.0 * hs[k]);
  }
  free(lam);
  return (4.0 * D[1] - D[0]) / 3.0;
}

/* Selected components of the same central differences, one component per  */
/* thread, each on its own copies of x, R and lambda (so that full-size      */
/* systems can be checked at a few components): kind[c] = 0 for             */
/* d e_L / d R (index[c] = 3 a + q), 1 for d e_L / d r (index[c] = 3 i + q), */
/* 2 for d e_L / d lambda (index[c] = mu L + nu).  out[c] is the value      */
/* orc_elocal_grad_fd or orc_elocal_dlambda_fd gives for that component     */
/* (the same steps in the same order).  Returns 0 for a bad kind or index.  */
int orc_elocal_fd_select(const orc_system *s, const double *x, double h, int n, const int *kind,
                         const long long *index, double *out) {
  const int N = s->n_up + s->n_dn, L = s->L;
  for (int c = 0; c < n; ++c) {
    const long long lim = kind[c] == 0 ? 3LL * s->n_atoms : kind[c] == 1 ? 3LL * N : (long long)L * L;
    if (kind[c] < 0 || kind[c] > 2 || index[c] < 0 || index[c] >= lim) return 0;
  }
#pragma omp parallel for schedule(dynamic)
  for (int c = 0; c < n; ++c) {
    orc_system t = *s;
    double *xx = (double *)malloc(sizeof(double) * 3 * N);
    double *RR = (double *)malloc(sizeof(double) * 3 * s->n_atoms);
    double *lam = kind[c] == 2 ? (double *)malloc(sizeof(double) * (size_t)L * L) : NULL;
    memcpy(xx, x, sizeof(double) * 3 * N);
    memcpy(RR, s->R, sizeof(double) * 3 * s->n_atoms);
    t.R = RR;
    if (lam) {
      memcpy(lam, s->lam, sizeof(double) * (size_t)L * L);
      t.lam = lam;
    }
    double *v = kind[c] == 0 ? RR : kind[c] == 1 ? xx : lam;
    const double v0 = v[index[c]];
    const double hs[2] = {h, 0.5 * h};
    double D[2];
    for (int k = 0; k < 2; ++k) {
      v[index[c]] = v0 + hs[k];
      const double ep = el_at(&t, xx);
      v[index[c]] = v0 - hs[k];
      const double em = el_at(&t, xx);
      v[index[c]] = v0;
      D[k] = (ep - em) / (2.0 * hs[k]);
    }
    out[c] = (4.0 * D[1] - D[0]) / 3.0;
    free(xx);
    free(RR);
    free(lam);
  }
  return 1;
}

/* ------------------------------------------------------------------------ */
/* Error bar of the VMC mean from correlated samples by reblocking (Sec.    */
/* VMC: blocks of growing size until the estimate of the error plateaus).   */
/* eL: [T][W] local energies of W walkers over T sweeps.  The series is the  */
/* walker mean per sweep, m_t = (1/W) sum_w eL[t][w].  Level k groups it in  */
/* n_k = floor(T / 2^k) consecutive blocks of B = 2^k sweeps (a ragged tail  */
/* is dropped) with block means b_j; for n_k >= 2:                          */
/*   sigma_k = sqrt( sum_j (b_j - bbar)^2 / (n_k (n_k - 1)) ),              */
/*   err_k   = sigma_k / sqrt(2 (n_k - 1))    (error of sigma_k for          */
/*                                             independent Gaussian blocks). */
/* levels: [nlev][4] = (B, n_k, sigma_k, err_k), nlev = levels with n_k >= 2. */
/* stats[4] = (mean of all T W values, chosen sigma, chosen level, plateau): */
/* the chosen level is the smallest k whose next level has n_{k+1} >= 8     */
/* blocks and |sigma_{k+1} - sigma_k| <= err_k (plateau = 1); without such a */
/* k, the last level with n_k >= 8 (plateau = 0).  Returns nlev.            */
/* ------------------------------------------------------------------------ */
int orc_reblock_levels(int T) {
  int n = 0;
  for (long B = 1; T / B >= 2; B *= 2) n++;
  return n;
}

int orc_reblock(const double *eL, int T, int W, double *levels, double *stats) {
  double *m = (double *)malloc(sizeof(double) * (T > 0 ? T : 1));
  double tot = 0.0;
  for (int t = 0; t < T; ++t) {
    double s = 0.0;
    for (int w = 0; w < W; ++w) s += eL[(size_t)t * W + w];
    m[t] = s / W;
    tot += s;
  }
  int nlev = orc_reblock_levels(T);
  for (int k = 0; k < nlev; ++k) {
    long B = 1L << k;
    long nb = T / B;
    double bbar = 0.0;
    for (long j = 0; j < nb; ++j) {
      double b = 0.0;
      for (long t = 0; t < B; ++t) b += m[j * B + t];
      bbar += b / B;
    }
    bbar /= nb;
    double ss = 0.0;
    for (long j = 0; j < nb; ++j) {
      double b = 0.0;
      for (long t = 0; t < B; ++t) b += m[j * B + t];
      double d = b / B - bbar;
      ss += d * d;
    }
    double sig = sqrt(ss / ((double)nb * (double)(nb - 1)));
    levels[4 * k + 0] = (double)B;
    levels[4 * k + 1] = (double)nb;
    levels[4 * k + 2] = sig;
    levels[4 * k + 3] = sig / sqrt(2.0 * (double)(nb - 1));
  }
  int chosen = -1, plateau = 0;
  for (int k = 0; k + 1 < nlev; ++k) {
    if (levels[4 * (k + 1) + 1] < 8.0) break;
    if (fabs(levels[4 * (k + 1) + 2] - levels[4 * k + 2]) <= levels[4 * k + 3]) {
      chosen = k;
      plateau = 1;
      break;
    }
  }
  if (chosen < 0)
    for (int k = 0; k < nlev; ++k)
      if (levels[4 * k + 1] >= 8.0) chosen = k;
  if (chosen < 0) chosen = 0;
  stats[0] = T > 0 && W > 0 ? tot / ((double)T * W) : 0.0;
  stats[1] = nlev > 0 ? levels[4 * chosen + 2] : 0.0;
  stats[2] = (double)chosen;
  stats[3] = (double)plateau;
  free(m);
  return nlev;
}

/* ------------------------------------------------------------------------ */
/* Stochastic reconfiguration (Sec. "Stochastic reconfiguration", Eqs.      */
/* SRupdate, sr and the diagonal shift of the regularised matrix): from M   */
/* samples with log-derivatives O [M][P] (O_k(x_i) = d ln|Psi(x_i)| / d     */
/* alpha_k, Sec. "Derivatives with respect to variational parameters") and  */
/* local energies e [M]:                                                    */
/*   Obar_k = (1/M) sum_i O_ik                                              */
/*   S_kl   = (1/M) sum_i (O_ik - Obar_k)(O_il - Obar_l)                    */
/*   f_k    = -2 (1/M) sum_i e_i (O_ik - Obar_k)     (Eq. eq_general_force)  */
/*   S'_kk  = S_kk (1 + eps), S'_kl = S_kl for k != l                       */
/*   dalpha = Delta S'^{-1} f   (solved by LU with partial pivoting)        */
/* Outputs (each may be NULL except f): Obar [P], S [P][P], f [P],          */
/* dalpha [P].  Returns 0 if S' is singular.                                */
/* ------------------------------------------------------------------------ */
int orc_sr(const double *O, const double *e, int M, int P, double eps, double delta, double *Obar_out,
           double *S_out, double *f, double *dalpha) {
  double *Ob = (double *)malloc(sizeof(double) * P);
  double *S = (double *)malloc(sizeof(double) * (size_t)P * P);
  for (int k = 0; k < P; ++k) {
    double s = 0.0;
    for (int i = 0; i < M; ++i) s += O[(size_t)i * P + k];
    Ob[k] = s / M;
  }
  for (int k = 0; k < P; ++k)
    for (int l = 0; l < P; ++l) {
      double s = 0.0;
      for (int i = 0; i < M; ++i) s += (O[(size_t)i * P + k] - Ob[k]) * (O[(size_t)i * P + l] - Ob[l]);
      S[(size_t)k * P + l] = s / M;
    }
  for (int k = 0; k < P; ++k) {
    double s = 0.0;
    for (int i = 0; i < M; ++i) s += e[i] * (O[(size_t)i * P + k] - Ob[k]);
    f[k] = -2.0 * s / M;
  }
  if (Obar_out) memcpy(Obar_out, Ob, sizeof(double) * P);
  if (S_out) memcpy(S_out, S, sizeof(double) * (size_t)P * P);
  int ok = 1;
  if (dalpha) {
    double *Sp = (double *)malloc(sizeof(double) * (size_t)P * P);
    double *inv = (double *)malloc(sizeof(double) * (size_t)P * P);
    memcpy(Sp, S, sizeof(double) * (size_t)P * P);
    for (int k = 0; k < P; ++k) Sp[(size_t)k * P + k] *= 1.0 + eps;
    double la, sg;
    ok = orc_det_inverse(P, Sp, &la, &sg, inv);
    if (ok)
      for (int k = 0; k < P; ++k) {
        double s = 0.0;
        for (int l = 0; l < P; ++l) s += inv[(size_t)k * P + l] * f[l];
        dalpha[k] = delta * s;
      }
    free(Sp);
    free(inv);
  }
  free(Ob);
  free(S);
  return ok;
}

/* ------------------------------------------------------------------------ */
/* Space-warp coordinate transformation for forces (Sec. "Atomic forces"):  */
/* an electron at r moves with nucleus a by Delta R_a omega_a(r),           */
/*   omega_a(r) = kappa(|r - R_a|) / sum_b kappa(|r - R_b|), kappa(d) = 1/d^4 */
/* omega: [n_atoms], domega: [n_atoms][3] (the gradient of omega_a at r).   */
/* ------------------------------------------------------------------------ */
void orc_swct_omega(const orc_system *s, const double r[3], double *omega, double *domega) {
  int na = s->n_atoms;
  double *k = (double *)malloc(sizeof(double) * na), *gk = (double *)malloc(sizeof(double) * 3 * na);
  double sk = 0.0, sg[3] = {0.0, 0.0, 0.0};
  for (int a = 0; a < na; ++a) {
    double d[3], d2 = 0.0;
    for (int q = 0; q < 3; ++q) {
      d[q] = r[q] - s->R[3 * a + q];
      d2 += d[q] * d[q];
    }
    k[a] = 1.0 / (d2 * d2);                                       /* |d|^-4 */
    for (int q = 0; q < 3; ++q) gk[3 * a + q] = -4.0 * d[q] / (d2 * d2 * d2);  /* grad |d|^-4 */
    sk += k[a];
    for (int q = 0; q < 3; ++q) sg[q] += gk[3 * a + q];
  }
  for (int a = 0; a < na; ++a) {
    omega[a] = k[a] / sk;
    if (domega)
      for (int q = 0; q < 3; ++q) domega[3 * a + q] = (gk[3 * a + q] * sk - k[a] * sg[q]) / (sk * sk);
  }
  free(k);
  free(gk);
}

/* The total derivatives of Eq. forces:aad with the space warp, for one      */
/* configuration x:                                                         */
/*   dEL[a] = d e_L / d R_a = de_L/dR_a + sum_i omega_a(r_i) de_L/dr_i      */
/*   dLJ[a] = d ln(J^{1/2} Psi) / d R_a                                     */
/*          = d ln|Psi|/dR_a + sum_i [omega_a(r_i) d ln|Psi|/dr_i + grad omega_a(r_i) / 2] */
/* with the partial derivatives of e_L from orc_elocal_grad_fd (step h) and  */
/* those of ln|Psi| from orc_grad_logpsi.  dEL, dLJ: [n_atoms][3].          */
int orc_swct_derivs(const orc_system *s, const double *x, double h, double *dEL, double *dLJ) {
  int N = s->n_up + s->n_dn, na = s->n_atoms;
  double *eR = (double *)malloc(sizeof(double) * 3 * na), *er = (double *)malloc(sizeof(double) * 3 * N);
  double *lR = (double *)malloc(sizeof(double) * 3 * na), *lr = (double *)malloc(sizeof(double) * 3 * N);
  double *om = (double *)malloc(sizeof(double) * na), *dom = (double *)malloc(sizeof(double) * 3 * na);
  double djas[3];
  orc_elocal_grad_fd(s, x, h, eR, er);
  int ok = orc_grad_logpsi(s, x, NULL, djas, lR, lr);
  if (ok) {
    memcpy(dEL, eR, sizeof(double) * 3 * na);
    memcpy(dLJ, lR, sizeof(double) * 3 * na);
    for (int i = 0; i < N; ++i) {
      orc_swct_omega(s, x + 3 * i, om, dom);
      for (int a = 0; a < na; ++a)
        for (int q = 0; q < 3; ++q) {
          dEL[3 * a + q] += om[a] * er[3 * i + q];
          dLJ[3 * a + q] += om[a] * lr[3 * i + q] + 0.5 * dom[3 * a + q];
        }
    }
  }
  free(eR); free(er); free(lR); free(lr); free(om); free(dom);
  return ok;
}

/* ======================================================================== */
/* Lattice-regularised diffusion Monte Carlo (Sec. "Lattice regularized     */
/* Monte Carlo"), guiding function Psi_G = Psi_T, continuous time.          */
/* ======================================================================== */
/* Hops of one configuration.  Hop k = 6 i + 2 d + s moves electron i by     */
/* +a (s = 0) or -a (s = 1) along axis d.  rho_k = Psi_G(x'_k) / Psi_G(x),    */
/* from log|det G~|, its sign and J recomputed at x'_k (definition; 0 if     */
/* G~ is singular there).  The discretised kinetic energy has the element    */
/* -1/(2 a^2) for every hop; the fixed-node Hamiltonian keeps it where       */
/* s_{x',x} = rho_k H_{x',x} < 0 (rho_k > 0) and multiplies it by -gamma     */
/* where s_{x',x} > 0 (rho_k < 0, a hop across the node), moving (1 + gamma) */
/* V_sf to the diagonal.  The importance-sampled Green's function then      */
/* leaves x for x'_k with the rate                                           */
/*   t_k = (rho_k > 0 ? rho_k : gamma |rho_k|) / (2 a^2),                    */
/* Gamma = sum_k t_k (k = 0 .. 6N-1 in order).  With the regularised         */
/* potential V^a (Eq. lrdmc_potential) sum_x' H^FN_{x',x} Psi_G(x')/Psi_G(x)  */
/* is the continuous local energy e_L(x) for every gamma (the V_sf terms     */
/* cancel), which is what weights the walker.                                */
int orc_lrdmc_hops(const orc_system *s, const double *x, double a, double gamma, double *rho, double *t,
                   double *Gamma, double *eL) {
  const int N = s->n_up + s->n_dn;
  double o0[4], o1[4], e[5];
  if (!orc_logpsi(s, x, o0)) return 0;
  double *xp = (double *)malloc(sizeof(double) * 3 * N);
  const double c = 1.0 / (2.0 * a * a);
  double G = 0.0;
  for (int k = 0; k < 6 * N; ++k) {
    const int i = k / 6, d = (k % 6) / 2, sg = k % 2;
    memcpy(xp, x, sizeof(double) * 3 * N);
    xp[3 * i + d] = sg ? x[3 * i + d] - a : x[3 * i + d] + a;
    double r = 0.0;
    if (orc_logpsi(s, xp, o1)) r = o1[1] * o0[1] * exp(o1[0] - o0[0]);
    rho[k] = r;
    t[k] = (r > 0.0 ? r : -gamma * r) * c;
    G += t[k];
  }
  free(xp);
  *Gamma = G;
  orc_local_energy(s, x, e);
  *eL = e[0];
  return 1;
}

/* One projection of length tau for each of W walkers (continuous time): at  */
/* x the walker waits tau_xi = -ln(1 - xi) / Gamma(x) and its log-weight     */
/* falls by tau_xi (e_L(x) - e_ref); once the wait reaches the time left it  */
/* falls by the time left times (e_L(x) - e_ref) instead and the projection  */
/* ends; otherwise the walker hops to x'_k with probability t_k / Gamma.     */
/* e_ref only shifts every log-weight by the same tau e_ref.  Hop h of       */
/* walker w in generation g draws one Philox4x32-10 block, counter          */
/* (w, g, h, 2) and the VMC key: xi = (x0 + 1/2) 2^-32, and hop k is the     */
/* first whose running sum of t (k = 0, 1, ...) exceeds (x1 + 1/2) 2^-32     */
/* Gamma (the last hop with t > 0 if rounding leaves none).  A walker that   */
/* has made max_hops hops stays where it is for the rest of the time and    */
/* gets flag bit 1; a singular G~ gives flag bit 2, a non-finite Gamma or   */
/* e_L flag bit 4, and either ends its projection.                           */
/* weight[w] *= exp(sum of its log-weight changes); eL_out[w] = e_L at the  */
/* final configuration; hops_out[w] = hops made.                             */
static void lrdmc_walker(const orc_system *s, double *x, uint32_t wid, uint64_t seed, uint32_t gen, double a,
                         double gamma, double tau, double e_ref, int max_hops, double *weight, double *eL_out,
                         int *hops_out, int *flags_out) {
  const int N = s->n_up + s->n_dn;
  double *rho = (double *)malloc(sizeof(double) * 6 * N), *t = (double *)malloc(sizeof(double) * 6 * N);
  const uint32_t key[2] = {(uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32)};
  double left = tau, lw = 0.0, Gamma = 0.0, eL = 0.0;
  int h = 0, flags = 0;
  for (;;) {
    if (!orc_lrdmc_hops(s, x, a, gamma, rho, t, &Gamma, &eL)) {
      flags |= 2;
      break;
    }
    if (!isfinite(Gamma) || !isfinite(eL)) {
      flags |= 4;
      break;
    }
    if (h >= max_hops) {
      flags |= 1;
      lw -= left * (eL - e_ref);
      break;
    }
    const uint32_t ctr[4] = {wid, gen, (uint32_t)h, 2u};
    uint32_t o[4];
    orc_philox4x32_10(ctr, key, o);
    const double xi = ((double)o[0] + 0.5) * 0x1p-32;
    const double wait = Gamma > 0.0 ? -log(1.0 - xi) / Gamma : INFINITY;
    if (wait >= left) {
      lw -= left * (eL - e_ref);
      break;
    }
    lw -= wait * (eL - e_ref);
    left -= wait;
    const double thr = ((double)o[1] + 0.5) * 0x1p-32 * Gamma;
    double run = 0.0;
    int k = -1;
    for (int q = 0; q < 6 * N; ++q) {
      run += t[q];
      if (t[q] > 0.0) k = q;
      if (run > thr) break;
    }
    const int i = k / 6, d = (k % 6) / 2;
    x[3 * i + d] = (k % 2) ? x[3 * i + d] - a : x[3 * i + d] + a;
    h++;
  }
  *weight *= exp(lw);
  *eL_out = eL;
  *hops_out = h;
  *flags_out = flags;
  free(rho);
  free(t);
}

int orc_lrdmc_project(const orc_system *s, double *x, int W, long long walker0, uint64_t seed, long long gen,
                      double a, double gamma, double tau, double e_ref, int max_hops, double *weight, double *eL_out,
                      int *hops_out, int *flags_out, int nthreads) {
  const int N = s->n_up + s->n_dn;
  int bad = 0;
#ifdef _OPENMP
  if (nthreads > 0) omp_set_num_threads(nthreads);
#else
  (void)nthreads;
#endif
#pragma omp parallel for schedule(dynamic) reduction(+ : bad)
  for (int w = 0; w < W; ++w) {
    lrdmc_walker(s, x + (size_t)w * N * 3, (uint32_t)(walker0 + w), seed, (uint32_t)gen, a, gamma, tau, e_ref,
                 max_hops, weight + w, eL_out + w, hops_out + w, flags_out + w);
    if (flags_out[w] & 2) bad++;
  }
  return bad == 0;
}

/* Reconfiguration after a projection (Eqs. branching-1, branching-2): W new */
/* walkers drawn from the old ones with probabilities w_a / sum_b w_b, by   */
/* systematic resampling with one uniform per generation (Philox4x32-10,     */
/* counter (0, g, 0, 3), the VMC key, z = (x0 + 1/2) 2^-32): new walker j    */
/* takes the first old walker a whose running weight sum (a = 0, 1, ... in   */
/* order) exceeds (j + z) sum w / W (the last walker with w > 0 if rounding  */
/* leaves none).  wbar = sum w / W; ebar = sum w e_L / sum w (the mean local */
/* energy before the reconfiguration); the new weights are all 1.            */
void orc_lrdmc_branch(int W, uint64_t seed, long long gen, const double *w, const double *eL, int *parent,
                      double *wbar, double *ebar) {
  const uint32_t key[2] = {(uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32)};
  const uint32_t ctr[4] = {0u, (uint32_t)gen, 0u, 3u};
  uint32_t o[4];
  if (W <= 0) return;
  orc_philox4x32_10(ctr, key, o);
  const double z = ((double)o[0] + 0.5) * 0x1p-32;
  double S = 0.0, Se = 0.0;
  int last = 0;
  for (int b = 0; b < W; ++b) {
    S += w[b];
    Se += w[b] * eL[b];
    if (w[b] > 0.0) last = b;
  }
  int b = 0;
  double run = w[0];
  for (int j = 0; j < W; ++j) {
    const double thr = ((double)j + z) * S / W;
    while (b < W && !(run > thr)) {
      b++;
      if (b < W) run += w[b];
    }
    parent[j] = b < W ? b : last;
  }
  *wbar = S / W;
  *ebar = Se / S;
}

/* Energy with the correcting factor (Eq. many-walker-weight and the         */
/* estimator after it): E = sum_{n=p}^{T-1} G_n ebar_n / sum_{n=p}^{T-1} G_n,  */
/* G_n = prod_{j=1..p} wbar_{n-j}, the products taken as exponentials of     */
/* sums of logarithms less their largest (the same ratio without overflow).  */
double orc_lrdmc_energy(int T, const double *wbar, const double *ebar, int p) {
  if (p < 0 || p >= T) return NAN;
  double *lg = (double *)malloc(sizeof(double) * T);
  double mx = -INFINITY;
  for (int n = p; n < T; ++n) {
    double l = 0.0;
    for (int j = 1; j <= p; ++j) l += log(wbar[n - j]);
    lg[n] = l;
    if (l > mx) mx = l;
  }
  double num = 0.0, den = 0.0;
  for (int n = p; n < T; ++n) {
    const double g = exp(lg[n] - mx);
    num += g * ebar[n];
    den += g;
  }
  free(lg);
  return num / den;
}
