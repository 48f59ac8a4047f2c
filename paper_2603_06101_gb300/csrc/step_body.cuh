// Bodies of the device-controlled step kernels, shared by the one-solve
// kernels and the persistent batched kernels (kernels_loop.cu, the only
// translation unit that includes this header, compiled without implicit
// multiply-add contraction: the fused operations below are explicit fma(), so
// both kinds of kernel round identically).
// A body processes virtual block vb of nvb for one solve;
// the solve's last virtual block finishes the dot products and runs the
// controller.  Returns true when this call ran the last block and the solve's
// controller is halted afterwards.
#pragma once

#include <cuda_runtime.h>

#include <type_traits>

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

// Symplectic-Euler update sweep (Eqs. 10-11, S56-S59), residual (Eq. S60) and
// preconditioner (Eqs. 6-7); the last block runs the convergence / restart
// test of the controller (Eq. S61, S62).
__device__ __forceinline__ bool update_body(const StepArgs &a, int vb, int nvb) {
  CtlState *s = a.ctl;
  if (s->halt) return false;
  const UpdParams u = s->up;
  const int alpha = s->alpha;
  const bool proj = (alpha > 0) || (a.sector != 0);
  const int nxc = proj ? alpha : 0;
  const double *z = s->zc, *Z = s->Zc;
  double *wout = proj ? a.w : s->zn;
  float *zf = proj ? nullptr : s->zf;
  const double guard = s->p.guard;
  const double *pinv = s->pinv_ready ? a.pinv : nullptr;
  constexpr int NV = 11 + kMaxStates;  // 10 step dots, x_c . w, y . (D y)
  double acc[NV];
#pragma unroll
  for (int j = 0; j < NV; ++j) acc[j] = 0.0;
  const long long stride = (long long)nvb * blockDim.x;
  // Unit: sx = sy = 1 (every step but the first of a cycle and the lazily
  // scaled restart); then sx * x and sy * y are x and y exactly and their
  // products are skipped (two fewer FP64 operations per recurrence).
  auto sweep = [&](auto unit_tag) {
    constexpr bool Unit = decltype(unit_tag)::value;
    for (long long i = (long long)vb * blockDim.x + threadIdx.x; i < a.n; i += stride) {
      const double y = fma(-u.c, z[i], Unit ? a.y[i] : u.sy * a.y[i]);
      const double Y = fma(-u.c, Z[i], Unit ? a.Y[i] : u.sy * a.Y[i]);
      const double x = fma(u.b, y, Unit ? a.x[i] : u.sx * a.x[i]);
      const double X = fma(u.b, Y, Unit ? a.X[i] : u.sx * a.X[i]);
      a.y[i] = y;
      a.Y[i] = Y;
      a.x[i] = x;
      a.X[i] = X;
      const double zp = fma(-u.E, x, X) * u.kinv;
      const double w = zp * (pinv ? pinv[i] : recip(guarded(a.diag[i] - u.Epre, guard)));
      wout[i] = w;
      if (zf) zf[i] = (float)w;
      acc[0] = fma(x, x, acc[0]);
      acc[1] = fma(x, y, acc[1]);
      acc[2] = fma(y, y, acc[2]);
      acc[3] = fma(x, X, acc[3]);
      acc[4] = fma(x, Y, acc[4]);
      acc[5] = fma(y, Y, acc[5]);
      acc[6] = fma(zp, zp, acc[6]);
      if (!proj) {
        acc[7] = fma(x, w, acc[7]);
        acc[8] = fma(y, w, acc[8]);
        acc[9] = fma(w, w, acc[9]);
      }
#pragma unroll
      for (int j = 0; j < kMaxStates; ++j)
        if (j < nxc) acc[10 + j] = fma(a.xc[(size_t)j * a.n + i], w, acc[10 + j]);
      acc[NV - 1] = fma(y * a.diag[i], y, acc[NV - 1]);  // kinetic term of Section S4 (M = D - E)
    }
  };
  if (u.sx == 1.0 && u.sy == 1.0) sweep(std::true_type{});
  else sweep(std::false_type{});
  int slots[NV];
#pragma unroll
  for (int j = 0; j < 7; ++j) slots[j] = S_NXX + j;
#pragma unroll
  for (int j = 7; j < 10; ++j) slots[j] = proj ? -1 : (S_NXZ + j - 7);
#pragma unroll
  for (int j = 0; j < kMaxStates; ++j) slots[10 + j] = (j < nxc) ? S_XCW0 + j : -1;
  slots[NV - 1] = S_YDY;
  block_partials<NV, kStepThreads>(acc, slots, a.partials, nvb, vb);
  if (!last_block(a.counter + 0, nvb)) return false;
  int act[NV];
  int na = 0;
  for (int j = 0; j < NV; ++j)
    if (slots[j] >= 0) act[na++] = slots[j];
  finish_slots(a.partials, nvb, act, na, s->dots, a.counter + 0);
  return ctl_run_shadowed(s, [](CtlHead &h) {
           h.iters += 1;
           if (h.iters > h.iter_cap) h.halt = H_CAP;
           ctl_check(h);
         }) != 0;
}

// Projection against the stored states (Eq. S31) with the c = c^T
// symmetrisation of the singlet sector; dots x.z, y.z, z.z.
__device__ __forceinline__ void project_body(const StepArgs &a, int vb, int nvb) {
  CtlState *s = a.ctl;
  if (s->halt) return;
  const int alpha = s->alpha;
  if (!(alpha > 0 || a.sector)) return;  // the update wrote z directly
  double coef[kMaxStates];
#pragma unroll
  for (int j = 0; j < kMaxStates; ++j) coef[j] = (j < alpha) ? s->dots[S_XCW0 + j] : 0.0;
  double *z = s->zn;
  float *zf = s->zf;
  double acc[3] = {0.0, 0.0, 0.0};
  const long long stride = (long long)nvb * blockDim.x;
  for (long long i = (long long)vb * blockDim.x + threadIdx.x; i < a.n; i += stride) {
    double v = a.w[i];
    if (a.sector) {
      int ia, ib;
      split_det(i, a.nb, ia, ib);
      v = 0.5 * (v + a.w[(size_t)ib * a.nb + ia]);
    }
#pragma unroll
    for (int j = 0; j < kMaxStates; ++j)
      if (j < alpha) v = fma(-coef[j], a.xc[(size_t)j * a.n + i], v);
    z[i] = v;
    if (zf) zf[i] = (float)v;
    acc[0] = fma(a.x[i], v, acc[0]);
    acc[1] = fma(a.y[i], v, acc[1]);
    acc[2] = fma(v, v, acc[2]);
  }
  const int slots[3] = {S_NXZ, S_NYZ, S_NZZ};
  block_partials<3, kStepThreads>(acc, slots, a.partials, nvb, vb);
  if (!last_block(a.counter + 1, nvb)) return;
  finish_slots(a.partials, nvb, slots, 3, s->dots, a.counter + 1);
}

}  // namespace sbci
