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

// 1/d to ~2^-46 relative (one Newton step): the preconditioner values of the
// sector sweep, where an error of 1e-14 in a component of z moves the step's
// coefficients far less than the FP64 rounding of the dot products does.
__device__ __forceinline__ double recip46(double d) {
  const double r = (double)__frcp_rn((float)d);
  return r * fma(-d, r, 2.0);
}

// Symplectic-Euler update sweep (Eqs. 10-11, S56-S59), residual (Eq. S60) and
// preconditioner (Eqs. 6-7); the last block runs the convergence / restart
// test of the controller (Eq. S61, S62).
constexpr int kUpdNV = 11 + kMaxStates;  // 10 step dots, x_c . w, y . (D y)

__device__ __forceinline__ bool update_body(const StepArgs &a, int vb, int nvb, unsigned char *smem) {
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
  constexpr int NV = kUpdNV;
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
  block_partials_in<NV, kStepThreads>(acc, slots, a.partials, nvb, vb,
                                      reinterpret_cast<double (*)[NV][33]>(smem));
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

// The update sweep of a singlet-sector solve (c = c^T, n_alpha = n_beta):
// every vector of the step is symmetric as a matrix, so the sweep takes each
// symmetric pair of elements (i, j), (j, i) once.  Work unit: a pair of 16 x 16
// tiles, (ti, tj) read coalesced and its transpose (tj, ti) written through
// shared memory (on a diagonal tile the elements with row >= column).  Per
// pair: the recurrences and the residual once; the preconditioner at both
// diagonal elements D_ij and D_ji (reciprocals to 2^-46), and the symmetrised
// w = (w_ij + w_ji) / 2
// of reading R10 (formerly the projection's first step); the dot products
// weighted by the pair's two elements.  For the ground state (no stored
// state to project against) it writes z itself, with its FP32 copy and the
// dots x.z, y.z, z.z, and the projection pass has nothing left to do.
constexpr int kSymT = 16;  // 256 threads: one element of the tile each
struct SymSmem {
  double v[5][kSymT][kSymT + 1];  // y, Y, x, X, w of tile (ti, tj), stored transposed
  float f[kSymT][kSymT + 1];      // FP32 copy of z, transposed
  double dT[kSymT][kSymT + 1];    // D of tile (tj, ti)
  double pT[kSymT][kSymT + 1];    // 1 / guarded(D - E_c^0) of tile (tj, ti) (excited states)
};
// Shared memory of an update kernel: the tile buffers of the symmetric sweep
// or the block reduction's buffer (used one after the other).
constexpr size_t kUpdSmemBytes = sizeof(SymSmem) > block_partials_bytes<kUpdNV, kStepThreads>()
                                     ? sizeof(SymSmem)
                                     : block_partials_bytes<kUpdNV, kStepThreads>();

__device__ __forceinline__ bool update_body_sym(const StepArgs &a, int vb, int nvb, unsigned char *smem) {
  SymSmem &sm = *reinterpret_cast<SymSmem *>(smem);
  CtlState *s = a.ctl;
  if (s->halt) return false;
  const UpdParams u = s->up;
  const int alpha = s->alpha;
  const bool direct = (alpha == 0);  // z itself, no projection pass
  const int nxc = alpha;
  const double *z = s->zc, *Z = s->Zc;
  double *wout = direct ? s->zn : a.w;
  float *zf = direct ? s->zf : nullptr;
  const double guard = s->p.guard;
  const double *pinv = s->pinv_ready ? a.pinv : nullptr;
  const bool unit = (u.sx == 1.0 && u.sy == 1.0);
  constexpr int NV = kUpdNV;
  // half-weighted sums: a pair of elements adds its value once, a diagonal
  // element half of it; the sums are doubled (exactly) at the end
  double acc[NV];
#pragma unroll
  for (int j = 0; j < NV; ++j) acc[j] = 0.0;
  const int n = a.na;
  const int T = (n + kSymT - 1) / kSymT, units = T * (T + 1) / 2;
  const int tid = threadIdx.x, c = tid & (kSymT - 1), r0 = tid / kSymT;
  constexpr int kRows = kStepThreads / kSymT;  // rows of a tile per pass
  for (int un = vb; un < units; un += nvb) {
    int ti, tj;
    tri_unit(un, &ti, &tj);
    __syncthreads();  // the previous unit's readers of the shared buffers are done
    for (int r = r0; r < kSymT; r += kRows) {  // D (and the excited-state preconditioner) of tile (tj, ti)
      const int i2 = tj * kSymT + r, j2 = ti * kSymT + c;
      const bool in = i2 < n && j2 < n;
      sm.dT[r][c] = in ? a.diag[(size_t)i2 * n + j2] : 0.0;
      if (pinv) sm.pT[r][c] = in ? pinv[(size_t)i2 * n + j2] : 0.0;
    }
    __syncthreads();
    for (int r = r0; r < kSymT; r += kRows) {
      const int i = ti * kSymT + r, j = tj * kSymT + c;
      if (i >= n || j >= n || (ti == tj && r < c)) continue;
      const bool on_diag = (i == j);
      const size_t I = (size_t)i * n + j;
      const double y = fma(-u.c, z[I], unit ? a.y[I] : u.sy * a.y[I]);
      const double Y = fma(-u.c, Z[I], unit ? a.Y[I] : u.sy * a.Y[I]);
      const double x = fma(u.b, y, unit ? a.x[I] : u.sx * a.x[I]);
      const double X = fma(u.b, Y, unit ? a.X[I] : u.sx * a.X[I]);
      const double zp = fma(-u.E, x, X) * u.kinv;
      const double dA = a.diag[I], dB = sm.dT[c][r];
      const double pa = pinv ? pinv[I] : recip46(guarded(dA - u.Epre, guard));
      const double pb = on_diag ? pa : (pinv ? sm.pT[c][r] : recip46(guarded(dB - u.Epre, guard)));
      const double w = 0.5 * (zp * pa + zp * pb);
      a.y[I] = y;
      a.Y[I] = Y;
      a.x[I] = x;
      a.X[I] = X;
      wout[I] = w;
      if (zf) zf[I] = (float)w;
      sm.v[0][c][r] = y;
      sm.v[1][c][r] = Y;
      sm.v[2][c][r] = x;
      sm.v[3][c][r] = X;
      sm.v[4][c][r] = w;
      if (zf) sm.f[c][r] = (float)w;
      // the dots in half weight: the first factor halved on the diagonal
      auto dots = [&](auto diag_tag) {
        constexpr bool Dg = decltype(diag_tag)::value;
        const double xh = Dg ? 0.5 * x : x, yh = Dg ? 0.5 * y : y;
        const double zh = Dg ? 0.5 * zp : zp, wh = Dg ? 0.5 * w : w;
        acc[0] = fma(xh, x, acc[0]);
        acc[1] = fma(xh, y, acc[1]);
        acc[2] = fma(yh, y, acc[2]);
        acc[3] = fma(xh, X, acc[3]);
        acc[4] = fma(xh, Y, acc[4]);
        acc[5] = fma(yh, Y, acc[5]);
        acc[6] = fma(zh, zp, acc[6]);
        if (direct) {
          acc[7] = fma(xh, w, acc[7]);
          acc[8] = fma(yh, w, acc[8]);
          acc[9] = fma(wh, w, acc[9]);
        }
#pragma unroll
        for (int q = 0; q < kMaxStates; ++q)
          if (q < nxc) acc[10 + q] = fma(a.xc[(size_t)q * a.n + I], wh, acc[10 + q]);
        // y^T D y in full weight: y^2 (D_ij + D_ji) for a pair, y^2 D_ii on the diagonal
        acc[NV - 1] = fma(yh * y, dA + dB, acc[NV - 1]);
      };
      if (on_diag) dots(std::true_type{});
      else dots(std::false_type{});
    }
    __syncthreads();
    // tile (tj, ti): element (r, c) is the transpose of (c, r) of tile (ti, tj)
    for (int r = r0; r < kSymT; r += kRows) {
      const int i2 = tj * kSymT + r, j2 = ti * kSymT + c;
      if (i2 >= n || j2 >= n || (ti == tj && r >= c)) continue;
      const size_t I2 = (size_t)i2 * n + j2;
      a.y[I2] = sm.v[0][r][c];
      a.Y[I2] = sm.v[1][r][c];
      a.x[I2] = sm.v[2][r][c];
      a.X[I2] = sm.v[3][r][c];
      wout[I2] = sm.v[4][r][c];
      if (zf) zf[I2] = sm.f[r][c];
    }
  }
  // the half-weighted sums count twice (the y^T D y sum is in full weight):
  // doubled once per block, in the reduction's last stage
  double wgt[NV];
#pragma unroll
  for (int j = 0; j < NV; ++j) wgt[j] = (j < NV - 1) ? 2.0 : 1.0;
  __syncthreads();  // the tile buffers become the reduction's
  int slots[NV];
#pragma unroll
  for (int j = 0; j < 7; ++j) slots[j] = S_NXX + j;
#pragma unroll
  for (int j = 7; j < 10; ++j) slots[j] = direct ? (S_NXZ + j - 7) : -1;
#pragma unroll
  for (int j = 0; j < kMaxStates; ++j) slots[10 + j] = (j < nxc) ? S_XCW0 + j : -1;
  slots[NV - 1] = S_YDY;
  block_partials_in<NV, kStepThreads>(acc, slots, a.partials, nvb, vb,
                                      reinterpret_cast<double (*)[NV][33]>(smem), wgt);
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

// Projection against the stored states (Eq. S31); dots x.z, y.z, z.z.
__device__ __forceinline__ void project_body(const StepArgs &a, int vb, int nvb) {
  CtlState *s = a.ctl;
  if (s->halt) return;
  const int alpha = s->alpha;
  if (alpha == 0) return;  // the update wrote z directly (symmetrised in the sector)
  double coef[kMaxStates];
#pragma unroll
  for (int j = 0; j < kMaxStates; ++j) coef[j] = (j < alpha) ? s->dots[S_XCW0 + j] : 0.0;
  double *z = s->zn;
  float *zf = s->zf;
  double acc[3] = {0.0, 0.0, 0.0};
  const long long stride = (long long)nvb * blockDim.x;
  for (long long i = (long long)vb * blockDim.x + threadIdx.x; i < a.n; i += stride) {
    double v = a.w[i];  // (symmetric in the sector: the update symmetrised it)
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
