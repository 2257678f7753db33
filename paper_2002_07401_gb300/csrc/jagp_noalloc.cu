// jagp_noalloc.cu -- jagp_eval_noalloc: log|Psi| and sign of W configurations
// without any device allocation and without a caller-provided workspace.
//
// Some callers cannot allocate device memory at the point where they need a
// wave-function value: code running inside a memory pool or allocator that
// forbids new reservations, a framework hook that owns every allocation of
// the process, or a latency-critical loop that must not touch the allocator.
// For them this entry point keeps its scratch (orbital tables, lambda
// products, G~, its inverse, per-walker scalars) in one file-scope device
// array of fixed size instead of the walker-state buffer that jagp_eval takes.
//
// Limits and rules (also stated in include/jagp.h):
//   * The array holds kNoAllocScratchBytes (32 MiB) on every GPU that loads
//     this library, until the process exits.  W is limited by it: a call whose
//     scratch would not fit returns JAGP_ERR_UNSUPPORTED before any launch.
//   * All calls share the one array and it keeps the last call's contents.
//     Everything a call reads is either written earlier in the same call or,
//     for the per-walker status and counters, cleared at its start.  Calls
//     whose work overlaps on the GPU (several streams, several host threads)
//     race on the array and give wrong results; serialise them.
//   * The first call on a device looks up the array's device address with
//     cudaGetSymbolAddress (with that device current) and caches it; make that
//     first call before any stream capture.
//   * jagp_create (which copies the system to the device) still allocates
//     once, at set-up; this entry point itself calls no cudaMalloc, cudaFree or
//     allocating library routine.
//   * It always evaluates in FP64 (FP64 orbitals, lambda products, G~ and its
//     elimination), whatever the handle's precision: on a mixed-precision
//     handle its log|Psi| is the FP64 value, which differs from jagp_eval's
//     mixed-precision one by that path's stated error (<= 1e-6).
//   * Its kernels count towards jagp_launch_count; a failure is recorded for
//     jagp_last_error like that of any other entry point.
#include <mutex>

#include "jagp_ctx.h"

using namespace jagp;

namespace {

constexpr size_t kNoAllocScratchBytes = JAGP_NOALLOC_SCRATCH_BYTES;
constexpr int kMaxDevices = 64;

// In host code this name is only a host-side stand-in for the device array:
// kernels must get the address from cudaGetSymbolAddress (below), never the
// symbol itself.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

std::mutex g_noalloc_mu;
void *g_noalloc_ptr[kMaxDevices] = {};

// the sub-arrays of the scratch that the evaluation touches
struct EvalScratch {
  size_t phi_up, a_up, bt, pprop, ginv, gprop, scal, status, total;
};

EvalScratch eval_scratch_layout(size_t W, size_t n, size_t L) {
  EvalScratch s;
  size_t o = 0;
  auto take = [&](size_t bytes) { size_t r = o; o = align256(o + bytes); return r; };
  s.phi_up = take(W * n * L * 8);
  s.a_up = take(W * n * L * 8);
  s.bt = take(W * n * L * 8);
  s.pprop = take(W * n * L * 8);
  s.ginv = take(W * n * n * 8);
  s.gprop = take(W * n * n * 8);
  s.scal = take(W * S_STRIDE * 8);
  s.status = take(W * 4);
  s.total = o;
  return s;
}

// device address of the scratch array on the current device (set-up on first use)
jagp_status_t scratch_address(int device, void **out) {
  if (device < 0 || device >= kMaxDevices) return JAGP_ERR_UNSUPPORTED;
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (!g_noalloc_ptr[device]) {
    void *p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) {
      jagp_set_cuda_error(e);
      return JAGP_ERR_CUDA;
    }
    g_noalloc_ptr[device] = p;
  }
  *out = g_noalloc_ptr[device];
  return JAGP_OK;
}

#define NA_CU(call)                      \
  do {                                   \
    const cudaError_t e_ = (call);       \
    ++h->launches;                       \
    if (e_ != cudaSuccess) {             \
      jagp_set_cuda_error(e_);           \
      return JAGP_ERR_CUDA;              \
    }                                    \
  } while (0)

jagp_status_t eval_noalloc(jagp_handle_t h, const double *d_r, int W, double *d_logabs, double *d_sign,
                           void *stream) {
  if (!h || !d_r || W <= 0 || W > h->max_walkers) return JAGP_ERR_INVALID_ARG;
  if (h->ds.use_j3) {
    jagp_set_detail("the fixed scratch holds no three-body Jastrow vectors");
    return JAGP_ERR_UNSUPPORTED;
  }
  const DevSystem &d = h->ds;
  const int n = d.n_up, Lb = d.L;
  const EvalScratch S = eval_scratch_layout((size_t)W, (size_t)n, (size_t)Lb);
  if (S.total > kNoAllocScratchBytes) {
    jagp_set_detail("W = %d needs %zu bytes of scratch, more than the %zu of the fixed array", W, S.total,
                    kNoAllocScratchBytes);
    return JAGP_ERR_UNSUPPORTED;
  }
  int device = -1;
  if (cudaGetDevice(&device) != cudaSuccess) return JAGP_ERR_CUDA;
  if (device != h->device) {
    jagp_set_detail("current device %d is not the handle's device %d", device, h->device);
    return JAGP_ERR_INVALID_ARG;
  }
  void *base = nullptr;
  jagp_status_t rc = scratch_address(device, &base);
  if (rc != JAGP_OK) return rc;
  char *b = static_cast<char *>(base);
  double *phi_up = reinterpret_cast<double *>(b + S.phi_up), *a_up = reinterpret_cast<double *>(b + S.a_up);
  double *bt = reinterpret_cast<double *>(b + S.bt), *pprop = reinterpret_cast<double *>(b + S.pprop);
  double *ginv = reinterpret_cast<double *>(b + S.ginv), *gprop = reinterpret_cast<double *>(b + S.gprop);
  double *scal = reinterpret_cast<double *>(b + S.scal);
  int *status = reinterpret_cast<int *>(b + S.status);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  // the same sequence as jagp_eval, on the static scratch
  NA_CU(launch_walker_init(scal, status, W, st, d_r, d.N));
  NA_CU(launch_basis_points(d, false, d_r, W, 0, n, phi_up, nullptr, nullptr, 0, 0, st));
  NA_CU(launch_basis_points(d, false, d_r, W, n, d.n_dn, pprop, nullptr, nullptr, 0, 0, st));
  NA_CU(launch_lambda_rows(phi_up, d.lam, a_up, nullptr, nullptr, W * n, n, n, Lb, W * n, st));
  if (d.n_dn > 0)
    NA_CU(launch_lambda_rows(pprop, d.lamT, bt, nullptr, nullptr, W * d.n_dn, d.n_dn, n, Lb, W * d.n_dn, st));
  NA_CU(launch_fill_unpaired(d, bt, W, st));
  NA_CU(launch_gemm_rows(phi_up, (size_t)n * Lb, bt, (size_t)n * Lb, n, n, Lb, gprop, (size_t)n * n, n, W, st));
  NA_CU(launch_refresh_inverse(gprop, ginv, scal, status, n, W, 0, h->drift_tol, st));
  NA_CU(launch_jastrow_full(d, d_r, scal, W, st));
  NA_CU(launch_logpsi_out(scal, W, d_logabs, d_sign, st));
  return JAGP_OK;
}

}  // namespace

extern "C" jagp_status_t jagp_eval_noalloc(jagp_handle_t h, const double *d_r, int W, double *d_logabs,
                                          double *d_sign, void *stream) {
  return jagp_note(h, "jagp_eval_noalloc", eval_noalloc(h, d_r, W, d_logabs, d_sign, stream));
}
