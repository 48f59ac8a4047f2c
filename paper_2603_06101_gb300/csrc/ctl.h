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

// The controller's scalar state.  The device runs its decisions on a copy of
// this header in shared memory (one L2 round trip in, one out) instead of
// chasing global-memory loads on a single thread; trace records go straight to
// the ring behind trace_ptr.
struct CtlHead {
  CtlParams p;
  // ping-pong z / Z: the update reads (zc, Zc), projection/sigma write (zn, Zn)
  double *zc, *Zc, *zn, *Zn;
  // FP32 copy of zn written by its producer (update or projection) when the
  // sigma runs in a split/FP32 mode (nullptr in FP64 mode): the low-precision
  // gather reads it instead of converting zn element by element
  float *zf;
  int alpha, t, first, pending_check, prec, halt;
  int stage;       // 0: low-precision stage (ends with H_SWITCH); 1: to Eq. S61
  int pinv_ready;  // the step arguments' pinv holds 1 / guarded(D - Ec0) for this state
  int n_stage1;    // H-products spent in stage 1 of this state
  int n_sync;      // stage-1 H-products since X was last made exact (FP64 H x)
  double sx_pending;
  double E;        // E_t
  double E_solve;  // E_{t+1} of the last subspace solve
  double Ec0;      // converged ground-state energy (preconditioner shift for alpha > 0)
  UpdParams up;
  double second[3], E2;  // second Ritz vector on (x_new, y_new, z_t) and its value
  int n_sigma, n_sigma_fp64, n_step, n_restart[4];
  long long ctl_cycles;  // device cycles spent in ctl_check + ctl_solve (this state)
  int iters, iter_cap;  // bodies run since the host last wrote the state; hard bound
  sbci_trace_record pending;
  int ntrace;  // records committed since the host last drained them
  double dots[S_COUNT];
  // y_t . (D y_t), y_t . y_t after the previous update and (b, c) of the
  // previous step: the Eq. S136 diagnostic of the next step
  double s136_yDy, s136_Nyy, s136_b, s136_c;
  sbci_trace_record *trace_ptr;  // the ring of the device state (CtlState::trace)
};

struct CtlState : CtlHead {
  sbci_trace_record trace[kTraceCap];
};

// FP64 reciprocal and reciprocal square root from an FP32 estimate refined by
// Newton steps: a handful of FP64 FMAs instead of the long FP64 division and
// square-root sequences, which the single controller thread pays serially on
// GB300's narrow FP64 pipe.
__host__ __device__ inline double f_recip(double d) {
#ifdef __CUDA_ARCH__
  double r = (double)__frcp_rn((float)d);
#else
  double r = (double)(1.0f / (float)d);
#endif
  r = r * fma(-d, r, 2.0);
  r = r * fma(-d, r, 2.0);
  return r;
}

__host__ __device__ inline double f_rsqrt(double x) {
#ifdef __CUDA_ARCH__
  double r = (double)rsqrtf((float)x);
#else
  double r = (double)(1.0f / sqrtf((float)x));
#endif
  // two Newton steps from the ~23-bit estimate: ~46, then FP64 rounding level
  for (int i = 0; i < 2; ++i) r = r * fma(-0.5 * x * r, r, 1.5);  // r <- r (3 - x r^2) / 2
  return r;
}

// Symmetric eigen-solver in FP32 (cyclic Jacobi), ascending.  n is a
// template parameter so that every loop unrolls and the arrays stay in
// registers (the controller runs on one thread; local memory would put an
// L1 round trip on its serial path).
template <int n>
__host__ __device__ inline void eigh_f32(const double *Ain, float *w, float *V) {
  float A[9];
  for (int i = 0; i < n * n; ++i) A[i] = (float)Ain[i];
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) V[i * n + j] = (i == j) ? 1.0f : 0.0f;
  for (int sweep = 0; sweep < 16; ++sweep) {
    float off = 0.0f, dg = 0.0f;
    for (int i = 0; i < n; ++i) {
      dg += A[i * n + i] * A[i * n + i];
      for (int j = i + 1; j < n; ++j) off += A[i * n + j] * A[i * n + j];
    }
    if (off <= 1e-14f * (dg + 1e-30f)) break;
    for (int p = 0; p < n; ++p)
      for (int q = p + 1; q < n; ++q) {
        const float apq = A[p * n + q];
        if (apq == 0.0f) continue;
        const float theta = (A[q * n + q] - A[p * n + p]) / (2.0f * apq);
        const float t = (theta >= 0.0f ? 1.0f : -1.0f) / (fabsf(theta) + sqrtf(theta * theta + 1.0f));
        const float c = 1.0f / sqrtf(t * t + 1.0f), s = t * c;
        for (int k = 0; k < n; ++k) {
          const float akp = A[k * n + p], akq = A[k * n + q];
          A[k * n + p] = c * akp - s * akq;
          A[k * n + q] = s * akp + c * akq;
        }
        for (int k = 0; k < n; ++k) {
          const float apk = A[p * n + k], aqk = A[q * n + k];
          A[p * n + k] = c * apk - s * aqk;
          A[q * n + k] = s * apk + c * aqk;
        }
        for (int k = 0; k < n; ++k) {
          const float vkp = V[k * n + p], vkq = V[k * n + q];
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
      const float tw = w[i];
      w[i] = w[m];
      w[m] = tw;
      for (int k = 0; k < n; ++k) {
        const float tv = V[k * n + i];
        V[k * n + i] = V[k * n + m];
        V[k * n + m] = tv;
      }
    }
  }
}

// One Rayleigh-quotient-iteration step in FP64 for a 2x2 / 3x3 symmetric V
// from an FP32 eigenpair (lam, v): v <- adj(V - lam I) v, normalised, and
// lam <- v^T V v.  Cubically convergent, so FP32 accuracy becomes FP64
// accuracy in one step for separated eigenvalues.  Returns the residual
// |V v - lam v| for the caller's acceptance test.
template <int n>
__host__ __device__ inline double rqi_refine(const double *V, double &lam, double *v) {
  double w[3];
  if (n == 2) {
    const double a = V[0] - lam, b = V[1], d = V[3] - lam;
    // adj [[a, b], [b, d]] = [[d, -b], [-b, a]]
    w[0] = d * v[0] - b * v[1];
    w[1] = -b * v[0] + a * v[1];
  } else {
    const double a = V[0] - lam, b = V[1], c = V[2], d = V[4] - lam, e = V[5], f = V[8] - lam;
    const double A00 = d * f - e * e, A01 = c * e - b * f, A02 = b * e - c * d;
    const double A11 = a * f - c * c, A12 = b * c - a * e, A22 = a * d - b * b;
    w[0] = A00 * v[0] + A01 * v[1] + A02 * v[2];
    w[1] = A01 * v[0] + A11 * v[1] + A12 * v[2];
    w[2] = A02 * v[0] + A12 * v[1] + A22 * v[2];
  }
  double nn = 0.0;
  for (int i = 0; i < n; ++i) nn = fma(w[i], w[i], nn);
  if (!(nn > 0.0)) return 1e300;
  const double inv = f_rsqrt(nn);
  // keep the sign of the starting vector
  double dot = 0.0;
  for (int i = 0; i < n; ++i) dot = fma(w[i], v[i], dot);
  const double sg = dot < 0.0 ? -inv : inv;
  for (int i = 0; i < n; ++i) v[i] = w[i] * sg;
  double Vv[3], l = 0.0;
  for (int i = 0; i < n; ++i) {
    double t = 0.0;
    for (int j = 0; j < n; ++j) t = fma(V[i * n + j], v[j], t);
    Vv[i] = t;
    l = fma(v[i], t, l);
  }
  lam = l;
  double r = 0.0;
  for (int i = 0; i < n; ++i) r = fma(Vv[i] - l * v[i], Vv[i] - l * v[i], r);
  return r;
}

template <int n>
__host__ __device__ inline void ctl_eigh(const double *Ain, double *w, double *V);

// Lowest two eigenpairs of a 2x2 / 3x3 symmetric V: FP32 Jacobi, then one
// FP64 Rayleigh-quotient-iteration step for the lowest pair (E_{t+1} and the
// step coefficients need FP64 accuracy: with FP32 coefficients, each step
// injects components of order 1e-7 along y and z that slow the last approach
// to Eq. S61).  The second pair only seeds the next state's start vector
// (S1.4), whose H-image is formed from the same coefficients, so its FP32
// accuracy is kept.  Falls back to the FP64 Jacobi solver when the refined
// residual is not at rounding level or the order is lost.
template <int n>
__host__ __device__ inline void ctl_eigh_fast(const double *V, double *w, double *U) {
  float wf[3], Uf[9];
  eigh_f32<n>(V, wf, Uf);
  double scale = 0.0;
  for (int i = 0; i < n * n; ++i) scale = fmax(scale, fabs(V[i]));
  double v[3], lam = (double)wf[0];
  for (int i = 0; i < n; ++i) v[i] = (double)Uf[i * n];
  const double r = rqi_refine<n>(V, lam, v);
  w[0] = lam;
  for (int i = 0; i < n; ++i) U[i * n] = v[i];
  w[1] = (double)wf[1];
  for (int i = 0; i < n; ++i) U[i * n + 1] = (double)Uf[i * n + 1];
  if (n == 3) {
    w[2] = (double)wf[2];
    for (int i = 0; i < n; ++i) U[i * n + 2] = (double)Uf[i * n + 2];
  }
  if (!(r <= 1e-26 * scale * scale) || !(w[0] <= w[1])) ctl_eigh<n>(V, w, U);
}

template <int n>
__host__ __device__ inline void ctl_eigh(const double *Ain, double *w, double *V) {
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
__host__ __device__ inline void ctl_first_step(const CtlHead &s, StepOut &o) {
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
  const double Bz = f_rsqrt(g);  // S12
  const double Bx = -Nxz * Bz;      // S13
  double V[4], w[2], U[4];
  V[0] = Hxx;
  V[1] = V[2] = Bx * Hxx + Bz * Hxz;
  V[3] = Bx * Bx * Hxx + Bz * Bz * Hzz + 2.0 * Bx * Bz * Hxz;
  ctl_eigh_fast<2>(V, w, U);
  const double vx = U[0], vz = U[2];
  o.E = w[0];
  const double den = f_recip(vx + vz * Bx);
  o.k = den;                        // S23
  o.c = -vz * Bz * den;             // S24
  const double A = U[1] + U[3] * Bx;
  o.r[0] = A;  // x_0 = x_new - y_new
  o.r[1] = -A;
  o.r[2] = U[3] * Bz;
  o.E2 = w[1];
}

// Later-step path (Eqs. S33-S55).
__host__ __device__ inline void ctl_later_step(const CtlHead &s, StepOut &o) {
  const double *d = s.dots;
  const double Nxx = d[S_NXX], Nxy = d[S_NXY], Nxz = d[S_NXZ];
  const double Nyy = d[S_NYY], Nyz = d[S_NYZ], Nzz = d[S_NZZ];
  const double Hxx = d[S_HXX], Hxy = d[S_HXY], Hxz = d[S_HXZ];
  const double Hyy = d[S_HYY], Hyz = d[S_HYZ], Hzz = d[S_HZZ];
  o.sx = 1.0;
  o.sy = 1.0;
  const double iNxx = f_recip(Nxx);
  const double Ax = f_rsqrt(Nxx);                            // S34
  const double By = f_rsqrt(Nyy - Nxy * Nxy * iNxx);         // S36
  const double Bx = -Nxy * iNxx * By;                        // S37
  const double P = Bx * Nxz + By * Nyz;                      // S42
  const double gz = Nzz - Nxz * Nxz * iNxx - P * P;
  if (!(gz > 0.0) || gz < s.p.gs_tol * Nzz) {                // z inside span{x, y}: c = 0
    double V[4], w[2], U[4];
    V[0] = Ax * Ax * Hxx;
    V[1] = V[2] = Ax * (Bx * Hxx + By * Hxy);
    V[3] = Bx * Bx * Hxx + By * By * Hyy + 2.0 * Bx * By * Hxy;
    ctl_eigh_fast<2>(V, w, U);
    const double vx = U[0], vy = U[2];
    o.k = f_recip(vx * Ax + vy * Bx);
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
  const double Cz = f_rsqrt(gz);                             // S39
  const double Cy = -P * By * Cz;                            // S40
  const double Cx = -(Nxz * iNxx + P * Bx) * Cz;             // S41
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
  ctl_eigh_fast<3>(V, w, U);
  const double vx = U[0], vy = U[3], vz = U[6];
  const double iden = f_recip(vx * Ax + vy * Bx + vz * Cx);
  o.E = w[0];
  o.k = iden;                                                // S53
  o.b = (vy * By + vz * Cy) * iden;                          // S54
  o.c = -vz * Cz * f_recip(vy * By + vz * Cy);               // S55
  const double cx = U[1] * Ax + U[4] * Bx + U[7] * Cx, cy = U[4] * By + U[7] * Cy, cz = U[7] * Cz;
  o.r[0] = cx;  // pre-update vectors: y_t = y_new + c z_t, x_t = x_new - b y_new
  o.r[1] = cy - cx * o.b;
  o.r[2] = cy * o.c + cz;
  o.E2 = w[1];
}

__host__ __device__ inline void ctl_commit(CtlHead &s, const sbci_trace_record &r) {
  if (s.ntrace < kTraceCap) s.trace_ptr[s.ntrace] = r;
  s.ntrace += 1;
}

// After the update sweep: finish the pending record and decide.
__host__ __device__ inline void ctl_check(CtlHead &s) {
  if (s.halt || !s.pending_check) return;
  s.pending_check = 0;
  const double *d = s.dots;
  sbci_trace_record r = s.pending;
  const double dz = d[S_ZPZP] > 0.0 ? d[S_ZPZP] * f_rsqrt(d[S_ZPZP]) : 0.0;
  const double dE = fabs(s.E_solve - s.E);
  r.dE = dE;
  r.dz = dz;
  // Section S4, Eq. S136 (indices of the update of step t, y_t -> y_{t+1}):
  // (2/c_{t-1}) Delta T = (b_{t-1}/c_{t-1}) (y_{t+1}^T M y_{t+1} - y_t^T M y_t),
  // M = D - E_{t+1}; defined on later steps (y_t is the previous update's y)
  r.s136 = (double)NAN;
  if (r.t > 0 && s.s136_c != 0.0) {
    const double Et1 = s.E_solve;
    const double dT = fma(-Et1, d[S_NYY], d[S_YDY]) - fma(-Et1, s.s136_Nyy, s.s136_yDy);
    r.s136 = s.s136_b * f_recip(s.s136_c) * dT;
  }
  s.s136_yDy = d[S_YDY];
  s.s136_Nyy = d[S_NYY];
  s.s136_b = r.b;
  s.s136_c = r.c;
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
  r.event = cause ? cause + 1 : r.event;  // (8 stays when no restart follows)
  ctl_commit(s, r);
  if (cause) {
    s.n_restart[cause - 1] += 1;
    s.first = 1;
    s.sx_pending = f_rsqrt(d[S_NXX]);
    s.t = 0;
  } else {
    s.t += 1;
    const double gy = d[S_NYY] - d[S_NXY] * d[S_NXY] * f_recip(d[S_NXX]);
    if (gy < s.p.gs_tol * d[S_NYY]) {  // y inside span{x}: first-step path
      s.first = 1;
      s.sx_pending = f_rsqrt(d[S_NXX]);
      s.t = 0;
    }
  }
  const bool low = s.p.user_prec != SBCI_FP64 && s.prec != SBCI_FP64;
  if (s.n_sigma >= s.p.max_sigma || (low && s.n_stage1 >= s.p.refine_max_sigma)) {
    s.halt = H_CAP;
  } else if (low && s.stage == 1 && s.n_sync >= s.p.max_cycle) {
    // The low-precision refinement carries X = H x by low-precision images
    // of y and z; where y or z is nearly dependent the update coefficients
    // grow (|b| up to 1e10 seen) and carry that rounding into X, so SB
    // energies can fall below the ground state and run away.  X is made
    // exact (one FP64 sigma) after every max_cycle refinement steps; after
    // two such windows without Eq. S61 the low-precision sigma is taken to
    // sit at its noise floor above the FP64 thresholds, and the state goes
    // on with FP64 sigma.
    s.halt = s.n_stage1 >= 2 * s.p.max_cycle ? H_CAP : H_SWITCH;
  }
}

// After sigma of the next z: subspace solve, parameters of the next update.
__host__ __device__ inline void ctl_solve(CtlHead &s) {
  if (s.halt) return;
  StepOut o;
  int event = 0;
  if (s.first) {
    ctl_first_step(s, o);
  } else {
    ctl_later_step(s, o);
    if (!isfinite(o.E) || !isfinite(o.k) || !isfinite(o.b) || !isfinite(o.c)) {
      // reading R15: a zero denominator in Eqs. S53-S55 leaves the later step
      // undefined; the step is taken on the first-step path from x/|x| (y
      // dropped), as a restart just before it would
      s.first = 1;
      s.sx_pending = f_rsqrt(s.dots[S_NXX]);
      s.t = 0;
      event = 8;
      ctl_first_step(s, o);
    }
  }
  if (!isfinite(o.E) || !isfinite(o.k) || !isfinite(o.b) || !isfinite(o.c)) {
    s.halt = H_NUMERIC;
    return;
  }
  s.n_sigma += 1;
  if (s.prec == SBCI_FP64) s.n_sigma_fp64 += 1;
  if (s.stage == 1) {
    s.n_stage1 += 1;
    s.n_sync += 1;
  }
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
  r.event = event;
  r.prec = s.prec;
  r.s136 = 0.0;
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
  s.up.kinv = f_recip(o.k);
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

#ifdef __CUDACC__
// Runs f on a shared-memory copy of the controller header (thread 0 of the
// calling block; all threads copy the header in and out) and returns the
// halt code.  Called by the one block that finishes a step's reductions.
template <typename F>
__device__ __forceinline__ int ctl_run_shadowed(CtlState *g, F f) {
  __shared__ __align__(16) CtlHead sh;
  static_assert(sizeof(CtlHead) % 4 == 0, "word copy");
  constexpr int nw = (int)(sizeof(CtlHead) / 4);
  uint32_t *d = reinterpret_cast<uint32_t *>(&sh);
  uint32_t *gw = reinterpret_cast<uint32_t *>(static_cast<CtlHead *>(g));
  __syncthreads();
  for (int i = threadIdx.x; i < nw; i += blockDim.x) d[i] = __ldcg(gw + i);
  __syncthreads();
  if (threadIdx.x == 0) {
    const long long t0 = clock64();
    f(sh);
    sh.ctl_cycles += clock64() - t0;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < nw; i += blockDim.x) gw[i] = d[i];
  const int h = sh.halt;
  __syncthreads();
  return h;
}
#endif

}  // namespace sbci
