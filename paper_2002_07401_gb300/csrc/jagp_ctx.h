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
  void *d_mem = nullptr;
  long long launches = 0;
  int prof_kernel = 0;
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> prof_events;
};
