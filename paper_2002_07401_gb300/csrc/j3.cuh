// j3.cuh -- the three/four-body Jastrow factor (Eq. threebody_jastrow) on the
// GPU, FP64 path:
//   J3 = sum_{i<j} chi(r_i)^T M^{s_i s_j} chi(r_j),
// M = M_p for equal spins, M_a otherwise (both symmetric), chi the Jastrow's
// own atomic basis.  With the spin sums U_s = sum_{i in s} chi(r_i) kept per
// walker together with M_p U_s and M_a U_s (the "j3 vectors", [6][LJ]:
// U_up, U_dn, M_p U_up, M_p U_dn, M_a U_up, M_a U_dn), electron i of spin s
// sees Q_i = M_p (U_s - chi_i) + M_a U_{s'}, and
//   J3 = 1/2 sum_i chi_i^T Q_i,  grad_i J3 = (grad chi_i)^T Q_i,  lap_i J3 = (lap chi_i)^T Q_i,
// and moving electron i by d chi changes J3 by d chi^T Q_i.
#pragma once

#include "jagp_common.cuh"

namespace jagp {

constexpr int kMaxLJ = 512;  // Jastrow basis functions (a thread keeps chi of one point)

// chi at a point into out[0 .. LJ)
__device__ __forceinline__ void j3_basis(const DevSystem &s, double px, double py, double pz, double *out) {
  for (int k = 0; k < s.n_jshells; ++k) {
    const double4 g = s.jshell_geo[k];
    const int info = s.jshell_info[k];
    double v[5];
    const int nc = shell_values(info, g.w, px - g.x, py - g.y, pz - g.z, v);
    for (int c = 0; c < nc; ++c) out[shell_off(info) + c] = v[c];
  }
}

// J3 pieces of one electron of spin `up` at (px, py, pz): adds 1/2 chi^T Q to
// *val, (grad chi)^T Q to g and (lap chi)^T Q to *lap.  V: the walker's j3 vectors.
__device__ inline void j3_electron(const DevSystem &s, const double *V, bool up, double px, double py, double pz,
                                   double *val, double g[3], double *lap) {
  const int LJ = s.LJ;
  double chi[kMaxLJ];
  j3_basis(s, px, py, pz, chi);
  const double *Vs = V + (up ? 2 : 3) * LJ, *Va = V + (up ? 5 : 4) * LJ;
  for (int k = 0; k < s.n_jshells; ++k) {
    const double4 gg = s.jshell_geo[k];
    const int info = s.jshell_info[k], off = shell_off(info);
    double d[5][5];
    const int nc = shell_derivs(info, gg.w, px - gg.x, py - gg.y, pz - gg.z, d);
    for (int c = 0; c < nc; ++c) {
      const int mu = off + c;
      const double *Mrow = s.j3p + (size_t)mu * LJ;
      double mc = 0.0;
      for (int nu = 0; nu < LJ; ++nu) mc = fma(Mrow[nu], chi[nu], mc);
      const double q = Vs[mu] + Va[mu] - mc;
      *val = fma(0.5 * d[c][0], q, *val);
      g[0] = fma(d[c][1], q, g[0]);
      g[1] = fma(d[c][2], q, g[1]);
      g[2] = fma(d[c][3], q, g[2]);
      *lap = fma(d[c][4], q, *lap);
    }
  }
}

}  // namespace jagp
