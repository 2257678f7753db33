// k_j3.cu -- the per-walker vectors of the three/four-body Jastrow (see j3.cuh).
#include "j3.cuh"
#include "jagp_group.cuh"
#include "jagp_launch.h"

namespace jagp {

namespace {

// One CTA per walker: U_s[mu] = sum_{i in s} chi_mu(r_i) (each thread owns whole
// shells and sums over the electrons in order), then M_p U_s and M_a U_s.
struct J3Prep {
  static __device__ __forceinline__ void run(DevSystem s, const double *__restrict__ r, double *__restrict__ buf,
                                             const uint3 bid, const uint3 gdim) {
    const int w = bid.x, N = s.N, LJ = s.LJ, tid = threadIdx.x;
    double *V = buf + (size_t)w * 6 * LJ;
    const double *x = r + (size_t)w * N * 3;
    for (int k = tid; k < s.n_jshells; k += blockDim.x) {
      const double4 g = s.jshell_geo[k];
      const int info = s.jshell_info[k], off = shell_off(info);
      double uu[5] = {0.0, 0.0, 0.0, 0.0, 0.0}, ud[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
      int nc = 1;
      for (int i = 0; i < N; ++i) {
        double v[5];
        nc = shell_values(info, g.w, x[3 * i] - g.x, x[3 * i + 1] - g.y, x[3 * i + 2] - g.z, v);
        for (int c = 0; c < nc; ++c) {
          if (i < s.n_up)
            uu[c] += v[c];
          else
            ud[c] += v[c];
        }
      }
      for (int c = 0; c < nc; ++c) {
        V[off + c] = uu[c];
        V[LJ + off + c] = ud[c];
      }
    }
    __syncthreads();
    for (int mu = tid; mu < LJ; mu += blockDim.x) {
      double pu = 0.0, pd = 0.0, au = 0.0, ad = 0.0;
      for (int nu = 0; nu < LJ; ++nu) {
        const double mp = s.j3p[(size_t)mu * LJ + nu], ma = s.j3a[(size_t)mu * LJ + nu];
        pu = fma(mp, V[nu], pu);
        pd = fma(mp, V[LJ + nu], pd);
        au = fma(ma, V[nu], au);
        ad = fma(ma, V[LJ + nu], ad);
      }
      V[2 * LJ + mu] = pu;
      V[3 * LJ + mu] = pd;
      V[4 * LJ + mu] = au;
      V[5 * LJ + mu] = ad;
    }
}
};
__global__ void __launch_bounds__(128) k_j3_prep(DevSystem s, const double *__restrict__ r, double *__restrict__ buf) {
  J3Prep::run(s, r, buf, blockIdx, gridDim);
}

}  // namespace

cudaError_t launch_j3_prep(const DevSystem &s, const double *r, double *buf, int W, cudaStream_t st) {
  if (W <= 0 || !s.use_j3) return cudaSuccess;
  return launch_or_record<J3Prep, 128>(k_j3_prep, dim3(W), dim3(128), 0, st, s, r, buf);
}

}  // namespace jagp
