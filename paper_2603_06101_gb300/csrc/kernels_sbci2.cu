// The SBCI2 pair controller on the GPU (pair_ctl.h): one thread per kernel,
// between the pair step's streaming kernels, so that a pair loop runs as one
// CUDA-graph while-loop with no host round trip per step.  Compiled with
// -fmad=false: the controller's arithmetic is the host pair step's, operation
// for operation.
#include <cuda_runtime.h>

#include "pair_ctl.h"

namespace sbci {

namespace {

__global__ void k_pair_proj_coef(PairCtl *ctl, const double *res) {
  if (threadIdx.x == 0 && blockIdx.x == 0) pair_proj_coef(*ctl, res);
}

__global__ void k_pair_after_dots(PairCtl *ctl, const double *res) {
  if (threadIdx.x == 0 && blockIdx.x == 0) pair_after_dots(*ctl, res);
}

__global__ void k_pair_decide(PairCtl *ctl, const double *res, unsigned long long cond) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  PairCtl &s = *ctl;
  if (s.halt == PH_RUN) pair_decide(s, res);
  // the H-product cap halts a pair within trace_cap steps; should it not, the
  // loop still ends here
  if (++s.bodies > s.trace_cap && s.halt == PH_RUN) s.halt = PH_BOUND;
  // (a step that restarts and reaches the cap is rescaled before the host
  // takes over, as in the host-driven loop)
  if (s.halt != PH_RUN && cond) cudaGraphSetConditional((cudaGraphConditionalHandle)cond, 0u);
}

}  // namespace

cudaError_t launch_pair_proj_coef(PairCtl *ctl, const double *res, cudaStream_t s) {
  k_pair_proj_coef<<<1, 32, 0, s>>>(ctl, res);
  return cudaGetLastError();
}

cudaError_t launch_pair_after_dots(PairCtl *ctl, const double *res, cudaStream_t s) {
  k_pair_after_dots<<<1, 32, 0, s>>>(ctl, res);
  return cudaGetLastError();
}

cudaError_t launch_pair_decide(PairCtl *ctl, const double *res, unsigned long long cond, cudaStream_t s) {
  k_pair_decide<<<1, 32, 0, s>>>(ctl, res, cond);
  return cudaGetLastError();
}

}  // namespace sbci
