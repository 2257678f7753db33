// jagp_ctx.h -- the handle behind jagp_handle_t (internal to libjagp).
#pragma once

#include <utility>
#include <vector>

#include "jagp_launch.h"

struct jagp_ctx {
  int device = 0;
  jagp::DevSystem ds{};
  int precision = JAGP_PREC_FP64;
  int max_walkers = 0;
  double drift_tol = 1e-8;
  int refresh_moves = 0;  // see jagp_options_t
  // lambda products on the tensor cores: the mixed path, or FP64 with
  // fp64_tensor_cores (slices per element and bits per slice)
  bool tc_lambda = false;
  int tc_slices = 0, tc_bits = 8;
  void *d_mem = nullptr;
  long long launches = 0;
  int prof_kernel = 0;
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> prof_events;
  // mixed path: lambda as fixed-point slices (kFixedSlices exact 8-bit integer
  // terms per element, BF16) with one exponent per output column, for the tensor cores
  int kp = 0;                            // L padded to a multiple of 64
  const uint16_t *split_lamT = nullptr;  // [L][5 kp]: row n slices lambda[:, n]  (A_up = phi^T lambda)
  const uint16_t *split_lam = nullptr;   // [L][5 kp]: row n slices lambda[n, :]  (Bt = lambda phi)
  const int *exp_lamT = nullptr;         // [L] exponents of those rows
  const int *exp_lam = nullptr;          // [L]
  int *d_err = nullptr;                  // tensor-core pipeline timeout flag
  // tile choices of jagp_autotune (0 / -1: the shape heuristics)
  int tune_bn_left = 0, tune_bn_right = 0;  // tensor-core tile width of the lambda products
  int tune_st_left = 0, tune_st_right = 0;  // and pipeline depth (0: as many stages as fit)
  int tune_tile_prop = -1;                  // per-walker proposal products (gemm_rows tile)
  int tune_tile_refresh = -1;               // per-walker refresh product G~ = Phi_up Bt^T
  // guided sampling (jagp_set_guiding): eps > 0 samples Psi_G instead of Psi_T
  double guide_theta = 0.375, guide_eps = 0.0;
  // text of the last failed call on this handle (jagp_last_error)
  jagp_status_t last_status = JAGP_OK;
  char last_error[512] = "no error";
};

// Error reporting shared by the translation units of libjagp (jagp_api.cu):
// jagp_note records a failed entry point's status, its name, the CUDA error
// text behind a JAGP_ERR_CUDA and the detail set by the failing check, in the
// handle (jagp_last_error) and returns the status unchanged.
jagp_status_t jagp_note(jagp_ctx *h, const char *fn, jagp_status_t s);
// the CUDA error text behind the next JAGP_ERR_CUDA of this thread
void jagp_set_cuda_error(cudaError_t e);
// a one-line detail of the next failure of this thread (e.g. which argument)
void jagp_set_detail(const char *fmt, ...);
