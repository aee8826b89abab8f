// DIC-preconditioned CG of the pressure system (see dic.cu).  Internal.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include "cfd_internal.h"

namespace cfd {

struct DicArgs {
  GridDims g;
  double* x;          // solution (in: x0 unless zero_x0; out)
  double* b;          // right-hand side (mean removed in place when remove_mean)
  double* r;          // work vectors, each g.count() doubles
  double* z;
  double* p;
  double* q;
  double* t;          // forward-sweep scratch
  double* d;          // reciprocal DIC pivots 1 / d_c (computed when setup = 1)
  double* scratch;    // >= dic_scratch_bytes() bytes
  int setup;          // 1: compute the pivots first
  int zero_x0;
  int remove_mean;
  int gauge;          // 1: shift x to mean gauge_value after the solve
  double gauge_value;
  double rtol;
  int max_iters;
  int max_restarts;
};

struct DicResult {
  int iters;
  int restarts;
  int status;         // kOk, kErrNotConverged, kErrBreakdown
  double rel_resid;   // true ||b - A x|| / ||b||
  double b_norm;
};

size_t dic_scratch_bytes();
cudaError_t launch_dic_setup(GridDims g, double* inv_d, cudaStream_t s, int64_t* launches);
cudaError_t launch_dic_apply(GridDims g, const double* inv_d, const double* r, double* t, double* z, cudaStream_t s,
                             int64_t* launches);
// x += target - mean(x): the gauge of the projection's pressure.
cudaError_t launch_gauge(GridDims g, double* x, double target, double* scratch, cudaStream_t s, int64_t* launches);
// Runs the whole solve (synchronises the stream once per iteration).
cudaError_t run_dic_pcg(const DicArgs& a, cudaStream_t s, int64_t* launches, DicResult* res);

}  // namespace cfd
