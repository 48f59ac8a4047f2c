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
  const double *pinv;        // [n] 1 / guarded(D - E_c^0), valid while ctl->pinv_ready
  long long n;
  int sector, na, nb;
  double *partials;          // [S_COUNT][grid] block partials
  unsigned int *counter;     // last-block counters: [0] update, [1] project
  unsigned long long cond;   // graph while-loop condition handle, 0 if none
};

int step_grid(long long n, int nsm);
cudaError_t launch_update_ctl(const StepArgs &a, int grid, cudaStream_t s);
cudaError_t launch_project_ctl(const StepArgs &a, int grid, cudaStream_t s);
// out[i] = 1 / guarded(diag[i] - E): the preconditioner of the excited states,
// whose shift E_c^0 is fixed for the whole state (the same arithmetic as the
// update sweep's, so the sweep may read it instead).
cudaError_t launch_pinv(const double *diag, double E, double guard, long long n, double *out, cudaStream_t s);

// The restart that follows an FP64 re-sync (end of the low-precision stage or
// of a refinement window), on the device: with xx = x.x and xX = x.X of the
// exact H-image (dots[0], dots[1]), the controller restarts from x/|x| with
// E = xX/xx on the first-step path of stage 1, exactly the fields the host's
// restart sets (same IEEE divisions and square root).
struct RestartArgs {
  double *z0, *Z0, *z1, *Z1;  // the ping-pong buffers in their start order
  float *zf;                  // FP32 copy of z for the low-precision sigma, or nullptr
  int prec;                   // sigma precision of the next stage
  int iter_cap;
  int ground;                 // 1: the preconditioner shift follows E (state 0)
  double Epre_fixed;          // the shift of an excited state (E_c^0)
};
cudaError_t launch_restart_resync(CtlState *ctl, const double *dots, const RestartArgs &r, cudaStream_t s);

}  // namespace sbci
