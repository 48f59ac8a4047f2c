// Arguments of the device-controlled step kernels (kernels_loop.cu).
#pragma once

#include <cuda_runtime.h>

#include "ctl.h"

namespace sbci {

struct StepArgs {
  CtlState *ctl;
  double *x, *X, *y, *Y, *w;
  const double *diag;
  const double *xc;          // [k][n] stored states x_c^i
  long long n;
  int sector, na, nb;
  double *partials;          // [S_COUNT][grid] block partials
  unsigned int *counter;     // last-block counters: [0] update, [1] project
  unsigned long long cond;   // graph while-loop condition handle, 0 if none
};

int step_grid(long long n, int nsm);
cudaError_t launch_update_ctl(const StepArgs &a, int grid, cudaStream_t s);
cudaError_t launch_project_ctl(const StepArgs &a, int grid, cudaStream_t s);

}  // namespace sbci
