// Device-resident controller of one SBCI1 solve (Algorithm 1, Sections
// S1.2-S1.5).  The state lives in device memory; the logic below runs on one
// GPU thread (the last block to finish a kernel) and, for the same data, on
// the host in tests.  Two entry points:
//
//   ctl_check(s)  after the update sweep of step t: convergence (Eq. S61),
//                 end of the low-precision stage, restarts (Eq. S62a-c,
//                 max_cycle), Gram-Schmidt breakdown of y, per-state cap;
//   ctl_solve(s)  after sigma of the next z: the 2x2 (Eqs. S10-S24) or 3x3
//                 (Eqs. S33-S55) subspace problem -> parameters of the next
//                 update (Eqs. S56-S60) and the second Ritz vector (S1.4).
//
// The kernels stop doing work once s.halt != 0; the host then handles the
// event (state converged, switch to FP64, cap reached, numeric failure).
#pragma once

#include <math.h>
#include <stdint.h>

#include "../../include/sbci.h"
#include "sbci_internal.h"

namespace sbci {

constexpr int kTraceCap = 2048;

enum Halt : int { H_RUN = 0, H_CONVERGED = 1, H_SWITCH = 2, H_CAP = 3, H_NUMERIC = 4 };

struct CtlParams {
  double eps0, r0, b_th, eps1, x_th1, x_th2, r1, guard, gs_tol, mixed_eps, mixed_r;
  int max_cycle, max_sigma, refine_max_sigma, user_prec;
};

// Scalars of the next update sweep.
struct UpdParams {
  double sx, sy, b, c, E, kinv, Epre;
};

struct CtlState {
  CtlParams p;
  // ping-pong z / Z: the update reads (zc, Zc), projection/sigma write (zn, Zn)
  double *zc, *Zc, *zn, *Zn;
  int alpha, t, first, pending_check, prec, halt;
  int stage;       // 0: low-precision stage (ends with H_SWITCH); 1: to Eq. S61
  int n_stage1;    // H-products spent in stage 1 of this state
  double sx_pending;
  double E;        // E_t
  double E_solve;  // E_{t+1} of the last subspace solve
  double Ec0;      // converged ground-state energy (preconditioner shift for alpha > 0)
  UpdParams up;
  double second[3], E2;  // second Ritz vector on (x_new, y_new, z_t) and its value
  int n_sigma, n_sigma_fp64, n_step, n_restart[4];
  int iters, iter_cap;  // bodies run since the host last wrote the state; hard bound
  sbci_trace_record pending;
  int ntrace;  // records committed since the host last drained them
  double dots[S_COUNT];
  sbci_trace_record trace[kTraceCap];
};

__host__ __device__ inline void ctl_eigh(int n, const double *Ain, double *w, double *V) {
  double A[9];
  for (int i = 0; i < n * n; ++i) A[i] = Ain[i];
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) V[i * n + j] = (i == j) ? 1.0 : 0.0;
  for (int sweep = 0; sweep < 32; ++sweep) {
    double off = 0.0, dg = 0.0;
    for (int i = 0; i < n; ++i) {
      dg += A[i * n + i] * A[i * n + i];
      for (int j = i + 1; j < n; ++j) off += A[i * n + j] * A[i * n + j];
    }
    if (off <= 1e-36 * (dg + 1e-300)) break;
    for (int p = 0; p < n; ++p)
      for (int q = p + 1; q < n; ++q) {
        const double apq = A[p * n + q];
        if (apq == 0.0) continue;
        const double theta = (A[q * n + q] - A[p * n + p]) / (2.0 * apq);
        const double t = (theta >= 0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
        const double c = 1.0 / sqrt(t * t + 1.0), s = t * c;
        for (int k = 0; k < n; ++k) {
          const double akp = A[k * n + p], akq = A[k * n + q];
          A[k * n + p] = c * akp - s * akq;
          A[k * n + q] = s * akp + c * akq;
        }
        for (int k = 0; k < n; ++k) {
          const double apk = A[p * n + k], aqk = A[q * n + k];
          A[p * n + k] = c * apk - s * aqk;
          A[q * n + k] = s * apk + c * aqk;
        }
        for (int k = 0; k < n; ++k) {
          const double vkp = V[k * n + p], vkq = V[k * n + q];
          V[k * n + p] = c * vkp - s * vkq;
          V[k * n + q] = s * vkp + c * vkq;
        }
      }
  }
  for (int i = 0; i < n; ++i) w[i] = A[i * n + i];
  for (int i = 0; i < n; ++i) {
    int m = i;
    for (int j = i + 1; j < n; ++j)
      if (w[j] < w[m]) m = j;
    if (m != i) {
      const double tw = w[i];
      w[i] = w[m];
      w[m] = tw;
      for (int k = 0; k < n; ++k) {
        const double tv = V[k * n + i];
        V[k * n + i] = V[k * n + m];
        V[k * n + m] = tv;
      }
    }
  }
}

struct StepOut {
  double E, b, c, k, E2;
  double r[3];
  double sx, sy;
};

// First-step path (Eqs. S10-S24) on x_0 = sx * x (|x_0| = 1).
__host__ __device__ inline void ctl_first_step(const CtlState &s, StepOut &o) {
  const double *d = s.dots;
  const double sx = s.sx_pending;
  const double Hxx = sx * sx * d[S_HXX];
  const double Nxz = sx * d[S_NXZ], Hxz = sx * d[S_HXZ];
  const double Nzz = d[S_NZZ], Hzz = d[S_HZZ];
  o.sx = sx;
  o.sy = 0.0;
  o.b = 1.0;
  const double g = Nzz - Nxz * Nxz;
  if (!(g > 0.0) || g < s.p.gs_tol * Nzz) {  // z inside span{x}: no move
    o.E = Hxx;
    o.c = 0.0;
    o.k = 1.0;
    o.E2 = Hxx;
    o.r[0] = o.r[1] = o.r[2] = 0.0;
    return;
  }
  const double Bz = 1.0 / sqrt(g);  // S12
  const double Bx = -Nxz * Bz;      // S13
  double V[4], w[2], U[4];
  V[0] = Hxx;
  V[1] = V[2] = Bx * Hxx + Bz * Hxz;
  V[3] = Bx * Bx * Hxx + Bz * Bz * Hzz + 2.0 * Bx * Bz * Hxz;
  ctl_eigh(2, V, w, U);
  const double vx = U[0], vz = U[2];
  o.E = w[0];
  o.k = 1.0 / (vx + vz * Bx);       // S23
  o.c = -vz * Bz / (vx + vz * Bx);  // S24
  const double A = U[1] + U[3] * Bx;
  o.r[0] = A;  // x_0 = x_new - y_new
  o.r[1] = -A;
  o.r[2] = U[3] * Bz;
  o.E2 = w[1];
}

// Later-step path (Eqs. S33-S55).
__host__ __device__ inline void ctl_later_step(const CtlState &s, StepOut &o) {
  const double *d = s.dots;
  const double Nxx = d[S_NXX], Nxy = d[S_NXY], Nxz = d[S_NXZ];
  const double Nyy = d[S_NYY], Nyz = d[S_NYZ], Nzz = d[S_NZZ];
  const double Hxx = d[S_HXX], Hxy = d[S_HXY], Hxz = d[S_HXZ];
  const double Hyy = d[S_HYY], Hyz = d[S_HYZ], Hzz = d[S_HZZ];
  o.sx = 1.0;
  o.sy = 1.0;
  const double Ax = 1.0 / sqrt(Nxx);                         // S34
  const double By = 1.0 / sqrt(Nyy - Nxy * Nxy / Nxx);       // S36
  const double Bx = -Nxy / Nxx * By;                         // S37
  const double P = Bx * Nxz + By * Nyz;                      // S42
  const double gz = Nzz - Nxz * Nxz / Nxx - P * P;
  if (!(gz > 0.0) || gz < s.p.gs_tol * Nzz) {                // z inside span{x, y}: c = 0
    double V[4], w[2], U[4];
    V[0] = Ax * Ax * Hxx;
    V[1] = V[2] = Ax * (Bx * Hxx + By * Hxy);
    V[3] = Bx * Bx * Hxx + By * By * Hyy + 2.0 * Bx * By * Hxy;
    ctl_eigh(2, V, w, U);
    const double vx = U[0], vy = U[2];
    o.k = 1.0 / (vx * Ax + vy * Bx);
    o.b = vy * By * o.k;
    o.c = 0.0;
    o.E = w[0];
    const double cx = U[1] * Ax + U[3] * Bx, cy = U[3] * By;
    o.r[0] = cx;
    o.r[1] = cy - cx * o.b;
    o.r[2] = 0.0;
    o.E2 = w[1];
    return;
  }
  const double Cz = 1.0 / sqrt(gz);                          // S39
  const double Cy = -P * By * Cz;                            // S40
  const double Cx = -(Nxz / Nxx + P * Bx) * Cz;              // S41
  const double hx = Cx * Hxx + Cy * Hxy + Cz * Hxz;
  const double hy = Cx * Hxy + Cy * Hyy + Cz * Hyz;
  double V[9], w[3], U[9];
  V[0] = Ax * Ax * Hxx;                                        // S44a
  V[1] = V[3] = Ax * (Bx * Hxx + By * Hxy);                    // S44b
  V[2] = V[6] = Ax * hx;                                       // S44c
  V[4] = Bx * Bx * Hxx + By * By * Hyy + 2.0 * Bx * By * Hxy;  // S44d
  V[5] = V[7] = Bx * hx + By * hy;                             // S44e
  V[8] = Cx * Cx * Hxx + Cy * Cy * Hyy + Cz * Cz * Hzz + 2.0 * Cx * Cy * Hxy +
         2.0 * Cx * Cz * Hxz + 2.0 * Cy * Cz * Hyz;            // S44f
  ctl_eigh(3, V, w, U);
  const double vx = U[0], vy = U[3], vz = U[6];
  const double den = vx * Ax + vy * Bx + vz * Cx;
  o.E = w[0];
  o.k = 1.0 / den;                                           // S53
  o.b = (vy * By + vz * Cy) / den;                           // S54
  o.c = -vz * Cz / (vy * By + vz * Cy);                      // S55
  const double cx = U[1] * Ax + U[4] * Bx + U[7] * Cx, cy = U[4] * By + U[7] * Cy, cz = U[7] * Cz;
  o.r[0] = cx;  // pre-update vectors: y_t = y_new + c z_t, x_t = x_new - b y_new
  o.r[1] = cy - cx * o.b;
  o.r[2] = cy * o.c + cz;
  o.E2 = w[1];
}

__host__ __device__ inline void ctl_commit(CtlState &s, const sbci_trace_record &r) {
  if (s.ntrace < kTraceCap) s.trace[s.ntrace] = r;
  s.ntrace += 1;
}

// After the update sweep: finish the pending record and decide.
__host__ __device__ inline void ctl_check(CtlState &s) {
  if (s.halt || !s.pending_check) return;
  s.pending_check = 0;
  const double *d = s.dots;
  sbci_trace_record r = s.pending;
  const double dz = sqrt(d[S_ZPZP]);
  const double dE = fabs(s.E_solve - s.E);
  r.dE = dE;
  r.dz = dz;
  s.E = s.E_solve;
  const bool low_stage = (s.stage == 0 && r.prec != SBCI_FP64);
  if (!isfinite(dz) || !isfinite(d[S_NXX])) {
    s.halt = H_NUMERIC;
    ctl_commit(s, r);
    return;
  }
  if (low_stage && ((dE < s.p.mixed_eps && dz < s.p.mixed_r) || s.n_sigma >= s.p.max_sigma / 2)) {
    r.event = 6;
    ctl_commit(s, r);
    s.halt = H_SWITCH;
    return;
  }
  if (!low_stage && dE < s.p.eps0 && dz < s.p.r0) {  // Eq. S61
    r.event = 1;
    ctl_commit(s, r);
    s.halt = H_CONVERGED;
    return;
  }
  int cause = 0;  // S62a, S62b, S62c, max_cycle
  if (s.alpha > 0 && fabs(r.b) < s.p.b_th && dE < s.p.eps1) cause = 1;
  else if (fabs(r.k) < s.p.x_th1 || fabs(r.k) > s.p.x_th2) cause = 2;
  else if (dz > s.p.r1 && r.t > 0) cause = 3;
  else if (r.t + 1 >= s.p.max_cycle) cause = 4;
  r.event = cause ? cause + 1 : 0;
  ctl_commit(s, r);
  if (cause) {
    s.n_restart[cause - 1] += 1;
    s.first = 1;
    s.sx_pending = 1.0 / sqrt(d[S_NXX]);
    s.t = 0;
  } else {
    s.t += 1;
    const double gy = d[S_NYY] - d[S_NXY] * d[S_NXY] / d[S_NXX];
    if (gy < s.p.gs_tol * d[S_NYY]) {  // y inside span{x}: first-step path
      s.first = 1;
      s.sx_pending = 1.0 / sqrt(d[S_NXX]);
      s.t = 0;
    }
  }
  if (s.n_sigma >= s.p.max_sigma || (s.p.user_prec != SBCI_FP64 && s.n_stage1 >= s.p.refine_max_sigma))
    s.halt = H_CAP;
}

// After sigma of the next z: subspace solve, parameters of the next update.
__host__ __device__ inline void ctl_solve(CtlState &s) {
  if (s.halt) return;
  StepOut o;
  if (s.first) ctl_first_step(s, o);
  else ctl_later_step(s, o);
  if (!isfinite(o.E) || !isfinite(o.k) || !isfinite(o.b) || !isfinite(o.c)) {
    s.halt = H_NUMERIC;
    return;
  }
  s.n_sigma += 1;
  if (s.prec == SBCI_FP64) s.n_sigma_fp64 += 1;
  if (s.stage == 1) s.n_stage1 += 1;
  s.n_step += 1;
  sbci_trace_record r;
  r.state = s.alpha;
  r.t = s.t;
  r.energy = o.E;
  r.b = o.b;
  r.c = o.c;
  r.k = o.k;
  r.dE = 0.0;
  r.dz = 0.0;
  r.event = 0;
  r.prec = s.prec;
  s.pending = r;
  s.E_solve = o.E;
  s.second[0] = o.r[0];
  s.second[1] = o.r[1];
  s.second[2] = o.r[2];
  s.E2 = o.E2;
  s.up.sx = o.sx;
  s.up.sy = o.sy;
  s.up.b = o.b;
  s.up.c = o.c;
  s.up.E = o.E;
  s.up.kinv = 1.0 / o.k;
  s.up.Epre = (s.alpha == 0) ? o.E : s.Ec0;  // newest ground-state Rayleigh quotient
  s.first = 0;
  s.pending_check = 1;
  // the next z becomes the current one
  double *tz = s.zc, *tZ = s.Zc;
  s.zc = s.zn;
  s.Zc = s.Zn;
  s.zn = tz;
  s.Zn = tZ;
}

}  // namespace sbci
