// Device-controlled SBCI1 step: the fused symplectic-Euler update sweep
// (Eqs. 10-11 with the H-image recurrences S56-S59, the residual S60 and the
// preconditioner of Eqs. 6-7) and the projection against stored states
// (Eq. S31).  Scalars come from the device controller state (ctl.h); the last
// block of the update sweep finishes its dot products and runs the
// convergence / restart test, so consecutive steps need no host round trip.
//
// Every kernel returns at once when the controller has halted, and then
// clears the loop condition of the enclosing graph (if any), so a graph
// while-loop over these kernels always ends.
#include <cuda_runtime.h>

#include "ctl.h"
#include "devreduce.cuh"
#include "sbci_internal.h"
#include "step.h"

namespace sbci {

constexpr int kStepThreads = 256;

__device__ __forceinline__ double guarded(double d, double g) {
  if (fabs(d) < g) return d < 0.0 ? -g : g;
  return d;
}

// 1/d from an FP32 estimate refined by two Newton steps in FP64 (relative
// error ~2^-46 after one, at FP64 rounding after two): four FP64 FMAs instead
// of the FP64 division sequence, which matters on GB300's narrow FP64 pipe.
__device__ __forceinline__ double recip(double d) {
  double r = (double)__frcp_rn((float)d);
  r = r * fma(-d, r, 2.0);
  r = r * fma(-d, r, 2.0);
  return r;
}

__device__ __forceinline__ void halt_loop(unsigned long long cond) {
  if (cond && blockIdx.x == 0 && threadIdx.x == 0)
    cudaGraphSetConditional((cudaGraphConditionalHandle)cond, 0u);
}

__global__ void __launch_bounds__(kStepThreads) k_update_ctl(StepArgs a) {
  CtlState *s = a.ctl;
  if (s->halt) {
    halt_loop(a.cond);
    return;
  }
  const UpdParams u = s->up;
  const int alpha = s->alpha;
  const bool proj = (alpha > 0) || (a.sector != 0);
  const int nxc = proj ? alpha : 0;
  const double *z = s->zc, *Z = s->Zc;
  double *wout = proj ? a.w : s->zn;
  const double guard = s->p.guard;
  constexpr int NV = 10 + kMaxStates;
  double acc[NV];
#pragma unroll
  for (int j = 0; j < NV; ++j) acc[j] = 0.0;
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < a.n; i += stride) {
    const double y = u.sy * a.y[i] - u.c * z[i];
    const double Y = u.sy * a.Y[i] - u.c * Z[i];
    const double x = u.sx * a.x[i] + u.b * y;
    const double X = u.sx * a.X[i] + u.b * Y;
    a.y[i] = y;
    a.Y[i] = Y;
    a.x[i] = x;
    a.X[i] = X;
    const double zp = (X - u.E * x) * u.kinv;
    const double w = zp * recip(guarded(a.diag[i] - u.Epre, guard));
    wout[i] = w;
    acc[0] += x * x;
    acc[1] += x * y;
    acc[2] += y * y;
    acc[3] += x * X;
    acc[4] += x * Y;
    acc[5] += y * Y;
    acc[6] += zp * zp;
    if (!proj) {
      acc[7] += x * w;
      acc[8] += y * w;
      acc[9] += w * w;
    }
#pragma unroll
    for (int j = 0; j < kMaxStates; ++j)
      if (j < nxc) acc[10 + j] += a.xc[(size_t)j * a.n + i] * w;
  }
  int slots[NV];
#pragma unroll
  for (int j = 0; j < 7; ++j) slots[j] = S_NXX + j;
#pragma unroll
  for (int j = 7; j < 10; ++j) slots[j] = proj ? -1 : (S_NXZ + j - 7);
#pragma unroll
  for (int j = 0; j < kMaxStates; ++j) slots[10 + j] = (j < nxc) ? S_XCW0 + j : -1;
  block_partials<NV, kStepThreads>(acc, slots, a.partials, gridDim.x);
  if (!last_block(a.counter + 0)) return;
  int act[NV];
  int na = 0;
  for (int j = 0; j < NV; ++j)
    if (slots[j] >= 0) act[na++] = slots[j];
  finish_slots(a.partials, gridDim.x, act, na, s->dots, a.counter + 0);
  if (threadIdx.x == 0) {
    s->iters += 1;
    if (s->iters > s->iter_cap) s->halt = H_CAP;
    ctl_check(*s);
    if (s->halt && a.cond) cudaGraphSetConditional((cudaGraphConditionalHandle)a.cond, 0u);
  }
}

// z_next = sym(w) - sum_i (x_c^i . w) x_c^i ; dots x.z, y.z, z.z.
__global__ void __launch_bounds__(kStepThreads) k_project_ctl(StepArgs a) {
  CtlState *s = a.ctl;
  if (s->halt) {
    halt_loop(a.cond);
    return;
  }
  const int alpha = s->alpha;
  if (!(alpha > 0 || a.sector)) return;  // the update wrote z directly
  double coef[kMaxStates];
#pragma unroll
  for (int j = 0; j < kMaxStates; ++j) coef[j] = (j < alpha) ? s->dots[S_XCW0 + j] : 0.0;
  double *z = s->zn;
  double acc[3] = {0.0, 0.0, 0.0};
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < a.n; i += stride) {
    double v = a.w[i];
    if (a.sector) {
      const int ia = (int)(i / a.nb), ib = (int)(i - (long long)ia * a.nb);
      v = 0.5 * (v + a.w[(size_t)ib * a.nb + ia]);
    }
#pragma unroll
    for (int j = 0; j < kMaxStates; ++j)
      if (j < alpha) v -= coef[j] * a.xc[(size_t)j * a.n + i];
    z[i] = v;
    acc[0] += a.x[i] * v;
    acc[1] += a.y[i] * v;
    acc[2] += v * v;
  }
  const int slots[3] = {S_NXZ, S_NYZ, S_NZZ};
  block_partials<3, kStepThreads>(acc, slots, a.partials, gridDim.x);
  if (!last_block(a.counter + 1)) return;
  finish_slots(a.partials, gridDim.x, slots, 3, s->dots, a.counter + 1);
}

int step_grid(long long n, int nsm) {
  long long g = (n + 4 * kStepThreads - 1) / (4 * kStepThreads);  // ~4 elements per thread
  if (g > 2LL * nsm) g = 2LL * nsm;
  if (g < 1) g = 1;
  return (int)g;
}

cudaError_t launch_update_ctl(const StepArgs &a, int grid, cudaStream_t s) {
  k_update_ctl<<<grid, kStepThreads, 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_project_ctl(const StepArgs &a, int grid, cudaStream_t s) {
  k_project_ctl<<<grid, kStepThreads, 0, s>>>(a);
  return cudaGetLastError();
}

}  // namespace sbci
