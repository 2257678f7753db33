// k_lrdmc.cu -- lattice-regularised diffusion Monte Carlo (Sec. "Lattice
// regularized Monte Carlo"), FP64 path, guiding function Psi_G = Psi_T,
// continuous time.
//
// Hop k = 6 i + 2 d + s moves electron i by +a (s = 0) or -a (s = 1) along
// axis d.  Its ratio Psi_G(x') / Psi_G(x) needs no determinant: the new row
// (up electron) or column (down electron) of G~ is linear in phi(r'), so the
// determinant ratio is phi(r') . M_i with the kinetic contraction vectors
// M_i = sum_j G~^{-1}[j][i] Bt_j (up) or sum_j G~^{-1}[i'][j] A_up_j (down)
// that the local energy of the current configuration has already formed;
// the Jastrow factor contributes exp(dJ1 + dJ2).  The fixed-node,
// importance-sampled Green's function leaves x for x'_k at the rate
// t_k = (rho_k > 0 ? rho_k : gamma |rho_k|) / (2 a^2), and weights the
// walker by exp(-(e_L(x) - e_ref) dt) while it stays (the regularised
// potential of Eq. lrdmc_potential makes the column sum of the fixed-node
// Hamiltonian the continuous local energy).
//
// A projection runs in rounds: every walker with time left takes one hop
// (or ends) per round, one thread deciding for each walker; then the moved
// electrons' orbital rows and their lambda products, and, on a compact copy
// of the moved walkers' state, a refresh of G~^{-1} and the local energy of
// the new configurations (jagp_api.cu) prepare the next round.  Decisions read the Philox4x32-10 stream (walker, generation, hop, 2).
#include "jagp_launch.h"

namespace jagp {

namespace {

constexpr int kRatioThreads = 128;

// warp-wide double-word sum; dw_add is commutative, so every lane of the
// butterfly ends with the same value
__device__ __forceinline__ fdw warp_sum_dw(fdw v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const fdw u{__shfl_xor_sync(0xffffffffu, v.hi, o), __shfl_xor_sync(0xffffffffu, v.lo, o)};
    v = dw_add(v, u);
  }
  return v;
}

__device__ __forceinline__ fdw dw_dist(const fdw *p, const fdw *q) {
  const fdw dx = dw_add(p[0], dw_neg(q[0])), dy = dw_add(p[1], dw_neg(q[1])), dz = dw_add(p[2], dw_neg(q[2]));
  return dw_sqrt(dw_add(dw_add(dw_mul(dx, dx), dw_mul(dy, dy)), dw_mul(dz, dz)));
}

// one-body term of one atom, -c^3 u(c r), u(s) = (1 - e^{-b s}) / (2b) (s / 2 at b = 0)
__device__ __forceinline__ fdw j1_term_dw(fdw c, fdw mc3, fdw b, fdw inv2b, bool b0, fdw r) {
  const fdw sc = dw_mul(c, r);
  const fdw u = b0 ? dw_mul_f(sc, 0.5f) : dw_mul(dw_add_f(dw_neg(dw_exp_neg(dw_neg(dw_mul(b, sc)))), 1.0f), inv2b);
  return dw_mul(mc3, u);
}

// pair term r / (k (1 + b r)), 1/k = kinv (a power of two)
__device__ __forceinline__ fdw j2_term_dw(fdw b, float kinv, fdw r) {
  return dw_mul_f(dw_mul(r, dw_recip(dw_add_f(dw_mul(b, r), 1.0f))), kinv);
}

// rho[w][k] for every hop of every walker still active: one CTA per walker, a
// warp per electron and its six hops (lanes over shells, atoms and electrons),
// in double-word FP32 arithmetic (relative error a few units of 2^-46; FP64
// instructions only to convert M, the positions and the atoms): GB300 issues
// FP32 at ~64x its FP64 rate, and the 6N orbital evaluations per walker and
// round are the bulk of the ratio work.
__global__ void __launch_bounds__(kRatioThreads) k_lrdmc_ratios(DevSystem s, const double *__restrict__ r,
                                                                 const double *__restrict__ mbuf,
                                                                 const int *__restrict__ active, double a,
                                                                 double *__restrict__ rho) {
  extern __shared__ double xs[];                         // the walker's positions [N][3]
  fdw *xd = reinterpret_cast<fdw *>(xs + 3 * s.N);       // the same as double-words
  const int w = blockIdx.x, N = s.N, L = s.L;
  if (!active[w]) return;
  for (int t = threadIdx.x; t < 3 * N; t += kRatioThreads) {
    const double v = r[(size_t)w * N * 3 + t];
    xs[t] = v;
    xd[t] = dw_of(v);
  }
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const bool b0 = s.b_ea == 0.0;
  const fdw bea = dw_of(s.b_ea), inv2b = dw_of(b0 ? 0.0 : 0.5 / s.b_ea);
  for (int i = warp; i < N; i += kRatioThreads / 32) {
    const double *o = xs + 3 * i;
    const fdw *od = xd + 3 * i;
    fdw pd[6][3];
#pragma unroll
    for (int k = 0; k < 6; ++k) {
      const int d = k / 2;
#pragma unroll
      for (int q = 0; q < 3; ++q) pd[k][q] = q == d ? dw_of((k & 1) ? o[d] - a : o[d] + a) : od[q];
    }
    fdw dot[6], dj[6];
#pragma unroll
    for (int k = 0; k < 6; ++k) dot[k] = dj[k] = fdw{0.0f, 0.0f};
    const double *Mi = mbuf + ((size_t)w * N + i) * L;
    for (int sh = lane; sh < s.n_shells; sh += 32) {
      const float4 gh = s.shell_dw[2 * sh], gl = s.shell_dw[2 * sh + 1];
      const int info = s.shell_info[sh], off = shell_off(info), nc = 2 * shell_l(info) + 1;
      fdw m[5];
#pragma unroll
      for (int c = 0; c < 5; ++c) m[c] = c < nc ? dw_of(Mi[off + c]) : fdw{0.0f, 0.0f};
      const fdw zeta{gh.w, gl.w};
#pragma unroll
      for (int k = 0; k < 6; ++k) {
        const DwDisp dd = dw_displacement(pd[k], gh, gl);
        float v[5], vl[5];
        shell_values_dw(info, zeta, dd, v, vl);
#pragma unroll
        for (int c = 0; c < 5; ++c)
          if (c < nc) dot[k] = dw_add(dot[k], dw_mul(fdw{v[c], vl[c]}, m[c]));
      }
    }
    if (s.use_j1) {
      for (int at = lane; at < s.n_atoms; at += 32) {
        const fdw R[3] = {dw_of(s.R[3 * at]), dw_of(s.R[3 * at + 1]), dw_of(s.R[3 * at + 2])};
        const double c = s.c1[at];
        const fdw cd = dw_of(c), mc3 = dw_of(-c * c * c);
        const fdw f0 = j1_term_dw(cd, mc3, bea, inv2b, b0, dw_dist(od, R));
#pragma unroll
        for (int k = 0; k < 6; ++k)
          dj[k] = dw_add(dj[k], dw_add(j1_term_dw(cd, mc3, bea, inv2b, b0, dw_dist(pd[k], R)), dw_neg(f0)));
      }
    }
    if (s.use_j2) {
      const bool up = i < s.n_up;
      for (int q = lane; q < N; q += 32) {
        if (q == i) continue;
        double kk, bb;
        j2_params(s, (q < s.n_up) == up, &kk, &bb);
        const fdw b = dw_of(bb);
        const float kinv = kk == 4.0 ? 0.25f : 0.5f;
        const fdw f0 = j2_term_dw(b, kinv, dw_dist(od, xd + 3 * q));
#pragma unroll
        for (int k = 0; k < 6; ++k)
          dj[k] = dw_add(dj[k], dw_add(j2_term_dw(b, kinv, dw_dist(pd[k], xd + 3 * q)), dw_neg(f0)));
      }
    }
#pragma unroll
    for (int k = 0; k < 6; ++k) {
      const fdw dk = warp_sum_dw(dot[k]), jk = warp_sum_dw(dj[k]);
      if (lane == k)
        rho[(size_t)w * 6 * N + 6 * i + k] =
            (static_cast<double>(dk.hi) + static_cast<double>(dk.lo)) *
            exp(static_cast<double>(jk.hi) + static_cast<double>(jk.lo));
    }
  }
}

// Start of a projection: time left tau, log-weight 0, no hops; walkers whose
// G~ is singular (or positions non-finite) do not take part (flag 2).
__global__ void k_lrdmc_start(const int *__restrict__ status, int W, double tau, double *__restrict__ left,
                              double *__restrict__ lw, int *__restrict__ hops, int *__restrict__ flags,
                              int *__restrict__ active) {
  const int w = blockIdx.x * blockDim.x + threadIdx.x;
  if (w >= W) return;
  const bool bad = (status[w] & (JAGP_WS_SINGULAR | JAGP_WS_NONFINITE)) != 0;
  left[w] = tau;
  lw[w] = 0.0;
  hops[w] = 0;
  flags[w] = bad ? 2 : 0;
  active[w] = bad ? 0 : 1;
}

// One round's decision per walker (one thread each, in the order the oracle
// takes the steps): the rates and Gamma from rho in hop order, the wait
// tau_xi = -ln(1 - xi) / Gamma; the walker ends (log-weight less the time
// left times e_L - e_ref) or hops to the first k whose running rate sum
// exceeds u Gamma (a non-finite Gamma or e_L ends the walker with flag 4).
// A moved electron's row goes to the up or down list
// (w n_up + row) for the lambda products, the walker to list_w; cnt[2]
// counts the walkers that moved (those still active).
__global__ void k_lrdmc_decide(DevSystem s, double *__restrict__ r, const double *__restrict__ rho,
                               const double *__restrict__ eL, const int *__restrict__ status, int W, uint32_t walker0,
                               uint32_t gen, double a, double gamma, double e_ref, int max_hops,
                               double *__restrict__ left, double *__restrict__ lw, int *__restrict__ hops,
                               int *__restrict__ flags, int *__restrict__ active, int *__restrict__ moved,
                               int *__restrict__ list_up, int *__restrict__ list_dn, int *__restrict__ list_w,
                               int *__restrict__ cnt) {
  const int w = blockIdx.x * blockDim.x + threadIdx.x;
  if (w >= W) return;
  moved[w] = -1;
  if (!active[w]) return;
  if (status[w] & (JAGP_WS_SINGULAR | JAGP_WS_NONFINITE)) {
    flags[w] |= 2;
    active[w] = 0;
    return;
  }
  const int N = s.N, n = s.n_up;
  const double *q = rho + (size_t)w * 6 * N;
  const double c = 1.0 / (2.0 * a * a);
  double G = 0.0;
  for (int k = 0; k < 6 * N; ++k) G += (q[k] > 0.0 ? q[k] : -gamma * q[k]) * c;
  const double e = eL[w];
  if (!isfinite(G) || !isfinite(e)) {
    flags[w] |= 4;
    active[w] = 0;
    return;
  }
  const int h = hops[w];
  if (h >= max_hops) {
    flags[w] |= 1;
    lw[w] -= left[w] * (e - e_ref);
    active[w] = 0;
    return;
  }
  uint32_t o[4] = {walker0 + (uint32_t)w, gen, (uint32_t)h, 2u};
  philox4x32_10(o, s.key0, s.key1);
  const double xi = ((double)o[0] + 0.5) * 0x1p-32;
  const double wait = G > 0.0 ? -log(1.0 - xi) / G : INFINITY;
  if (wait >= left[w]) {
    lw[w] -= left[w] * (e - e_ref);
    active[w] = 0;
    return;
  }
  lw[w] -= wait * (e - e_ref);
  left[w] -= wait;
  const double thr = ((double)o[1] + 0.5) * 0x1p-32 * G;
  double run = 0.0;
  int k = -1;
  for (int j = 0; j < 6 * N; ++j) {
    const double t = (q[j] > 0.0 ? q[j] : -gamma * q[j]) * c;
    run += t;
    if (t > 0.0) k = j;
    if (run > thr) break;
  }
  const int i = k / 6, d = (k % 6) / 2;
  double *x = r + ((size_t)w * N + i) * 3 + d;
  *x = (k & 1) ? *x - a : *x + a;
  hops[w] = h + 1;
  moved[w] = i;
  if (i < n)
    list_up[atomicAdd(cnt, 1)] = w * n + i;
  else
    list_dn[atomicAdd(cnt + 1, 1)] = w * n + (i - n);
  list_w[atomicAdd(cnt + 2, 1)] = w;
}

// Per-walker arrays between the state and the compact state of this round's
// moved walkers: gather dst[j] = src[list[j]], scatter dst[list[j]] = src[j],
// in 4-byte words (every per-walker size is a multiple of 4 bytes).
__global__ void __launch_bounds__(256) k_walker_copy(WalkerCopies cp, const int *__restrict__ list, int scatter) {
  const int j = blockIdx.x, w = list[j];
  for (int a = 0; a < cp.n; ++a) {
    const size_t words = cp.c[a].bytes / 4;
    const uint32_t *s = reinterpret_cast<const uint32_t *>(cp.c[a].src) + (size_t)(scatter ? j : w) * words;
    uint32_t *d = reinterpret_cast<uint32_t *>(cp.c[a].dst) + (size_t)(scatter ? w : j) * words;
    for (size_t t = threadIdx.x; t < words; t += blockDim.x) d[t] = s[t];
  }
}

// Orbital values of each moved electron at its new position into the
// proposal table (row w n_up + row of its spin) and, for an up electron, into
// the current table phi_up.
__global__ void __launch_bounds__(128) k_lrdmc_rows(DevSystem s, const double *__restrict__ r,
                                                     const int *__restrict__ moved, double *__restrict__ pprop,
                                                     double *__restrict__ phi_up) {
  const int w = blockIdx.x, i = moved[w];
  if (i < 0) return;
  const int n = s.n_up, L = s.L;
  const double *p = r + ((size_t)w * s.N + i) * 3;
  const bool up = i < n;
  const size_t row = (size_t)w * n + (up ? i : i - n);
  for (int sh = threadIdx.x; sh < s.n_shells; sh += blockDim.x) {
    const double4 g = s.shell_geo[sh];
    const int info = s.shell_info[sh], off = shell_off(info);
    double v[5];
    const int nc = shell_values(info, g.w, p[0] - g.x, p[1] - g.y, p[2] - g.z, v);
    for (int c = 0; c < nc; ++c) {
      pprop[row * L + off + c] = v[c];
      if (up) phi_up[row * L + off + c] = v[c];
    }
  }
}

// End of a projection: weight *= exp(log-weight), e_L of the final configuration.
__global__ void k_lrdmc_finish(int W, const double *__restrict__ lw, const double *__restrict__ eL_cur,
                               double *__restrict__ weight, double *__restrict__ eL_out) {
  const int w = blockIdx.x * blockDim.x + threadIdx.x;
  if (w >= W) return;
  weight[w] *= exp(lw[w]);
  if (eL_out) eL_out[w] = eL_cur[w];
}

// Reconfiguration (Eqs. branching-1, branching-2) by systematic resampling,
// one thread, every sum in walker order: z from Philox (0, g, 0, 3); new
// walker j takes the first old walker whose running weight sum exceeds
// (j + z) S / W; stats = (wbar, ebar).  Weights reset to 1.
__global__ void k_lrdmc_select(int W, uint32_t gen, uint32_t key0, uint32_t key1, double *__restrict__ weight,
                               const double *__restrict__ eL, int *__restrict__ parent, double *__restrict__ stats) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  uint32_t o[4] = {0u, gen, 0u, 3u};
  philox4x32_10(o, key0, key1);
  const double z = ((double)o[0] + 0.5) * 0x1p-32;
  double S = 0.0, Se = 0.0;
  int last = 0;
  for (int b = 0; b < W; ++b) {
    S += weight[b];
    Se += weight[b] * eL[b];
    if (weight[b] > 0.0) last = b;
  }
  int b = 0;
  double run = weight[0];
  for (int j = 0; j < W; ++j) {
    const double thr = ((double)j + z) * S / W;
    while (b < W && !(run > thr)) {
      b++;
      if (b < W) run += weight[b];
    }
    parent[j] = b < W ? b : last;
  }
  stats[0] = S / W;
  stats[1] = Se / S;
  for (int j = 0; j < W; ++j) weight[j] = 1.0;
}

// r_new[j] = r_old[parent[j]] (positions of the new population)
__global__ void k_lrdmc_gather(const double *__restrict__ r_old, const int *__restrict__ parent, int W, int N3,
                               double *__restrict__ r_new) {
  const long t = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long)W * N3) return;
  const int j = (int)(t / N3), c = (int)(t % N3);
  r_new[t] = r_old[(size_t)parent[j] * N3 + c];
}

// E = sum_{n >= p} G_n ebar_n / sum G_n, G_n = prod_{j=1..p} wbar_{n-j}, as
// exponentials of log sums less their largest (one thread, in order)
__global__ void k_lrdmc_energy(const double *__restrict__ wbar, const double *__restrict__ ebar, int T, int p,
                               double *__restrict__ E) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double mx = -INFINITY;
  for (int n = p; n < T; ++n) {
    double l = 0.0;
    for (int j = 1; j <= p; ++j) l += log(wbar[n - j]);
    mx = fmax(mx, l);
  }
  double num = 0.0, den = 0.0;
  for (int n = p; n < T; ++n) {
    double l = 0.0;
    for (int j = 1; j <= p; ++j) l += log(wbar[n - j]);
    const double g = exp(l - mx);
    num += g * ebar[n];
    den += g;
  }
  E[0] = num / den;
}

}  // namespace

cudaError_t launch_lrdmc_ratios(const DevSystem &s, const double *r, const double *mbuf, const int *active, double a,
                                double *rho, int W, cudaStream_t st) {
  if (W <= 0) return cudaSuccess;
  const size_t smem = (size_t)s.N * 3 * (sizeof(double) + sizeof(fdw));
  if (smem > 48 * 1024) return cudaErrorInvalidValue;
  k_lrdmc_ratios<<<W, kRatioThreads, smem, st>>>(s, r, mbuf, active, a, rho);
  return cudaGetLastError();
}

cudaError_t launch_lrdmc_start(const int *status, int W, double tau, LrdmcWork &lw, cudaStream_t st) {
  if (W <= 0) return cudaSuccess;
  k_lrdmc_start<<<(W + 127) / 128, 128, 0, st>>>(status, W, tau, lw.left, lw.lw, lw.hops, lw.flags, lw.active);
  return cudaGetLastError();
}

cudaError_t launch_lrdmc_decide(const DevSystem &s, double *r, const double *eL, const int *status, int W,
                                uint32_t walker0, uint32_t gen, double a, double gamma, double e_ref, int max_hops,
                                LrdmcWork &lw, cudaStream_t st) {
  if (W <= 0) return cudaSuccess;
  k_lrdmc_decide<<<(W + 127) / 128, 128, 0, st>>>(s, r, lw.rho, eL, status, W, walker0, gen, a, gamma, e_ref,
                                                   max_hops, lw.left, lw.lw, lw.hops, lw.flags, lw.active, lw.moved,
                                                   lw.list_up, lw.list_dn, lw.list_w, lw.cnt);
  return cudaGetLastError();
}

cudaError_t launch_lrdmc_rows(const DevSystem &s, const double *r, const int *moved, double *pprop, double *phi_up,
                              int W, cudaStream_t st) {
  if (W <= 0) return cudaSuccess;
  k_lrdmc_rows<<<W, 128, 0, st>>>(s, r, moved, pprop, phi_up);
  return cudaGetLastError();
}

cudaError_t launch_walker_copy(const WalkerCopies &cp, const int *list, int Wc, bool scatter, cudaStream_t st) {
  if (Wc <= 0) return cudaSuccess;
  for (int a = 0; a < cp.n; ++a)
    if (cp.c[a].bytes % 4) return cudaErrorInvalidValue;
  k_walker_copy<<<Wc, 256, 0, st>>>(cp, list, scatter ? 1 : 0);
  return cudaGetLastError();
}

cudaError_t launch_lrdmc_finish(int W, const double *lw, const double *eL_cur, double *weight, double *eL_out,
                                cudaStream_t st) {
  if (W <= 0) return cudaSuccess;
  k_lrdmc_finish<<<(W + 127) / 128, 128, 0, st>>>(W, lw, eL_cur, weight, eL_out);
  return cudaGetLastError();
}

cudaError_t launch_lrdmc_branch(int W, int N, uint32_t gen, uint32_t key0, uint32_t key1, double *weight,
                                const double *eL, int *parent, double *stats, const double *r_old, double *r_new,
                                cudaStream_t st) {
  if (W <= 0) return cudaSuccess;
  k_lrdmc_select<<<1, 32, 0, st>>>(W, gen, key0, key1, weight, eL, parent, stats);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const long tot = (long)W * N * 3;
  k_lrdmc_gather<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(r_old, parent, W, 3 * N, r_new);
  return cudaGetLastError();
}

cudaError_t launch_lrdmc_energy(const double *wbar, const double *ebar, int T, int p, double *E, cudaStream_t st) {
  k_lrdmc_energy<<<1, 32, 0, st>>>(wbar, ebar, T, p, E);
  return cudaGetLastError();
}

}  // namespace jagp
