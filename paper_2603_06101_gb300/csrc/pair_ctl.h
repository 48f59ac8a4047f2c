// Device-resident controller of the SBCI2 pair steps (Algorithm 2, Sections
// S2.1-S2.5): the state of one pair (alpha, alpha + 1) lives in device memory
// and the logic below runs on one GPU thread between the pair step's kernels
// (kernels_sbci2.cu), and, for the same data, on the host in tests.  Three
// entry points, in the order of one step:
//
//   pair_proj_coef   (alpha > 0) the projection of the preconditioned
//                    residuals against the stored states (Eqs. S101, S4-S7):
//                    coefficients of z^i -= sum_j (x_c^j . z^i) x_c^j;
//   pair_after_dots  the overlap S and T = B^T [H B] of the step's basis
//                    (x^a, x^b, y^a, y^b, z^a, z^b): canonical
//                    orthogonalisation, the 4x4 or 6x6 eigen-problem and the
//                    coefficients of Eqs. S93 / S112-S121 (reading Q6 falls
//                    back to the first-step path) -> the coefficients of the
//                    one combination that forms x, X (Q9), y, Y and z';
//   pair_decide      the norms |z'^a|, |z'^b|, |x^a|, |x^b| after it: trace
//                    record, convergence (Eq. S127), restart causes (Section
//                    S2.5, Q7) with the rescaling of x, X and z, the H-product
//                    cap (Q8).
//
// The arithmetic is the host pair step's, operation for operation (no fused
// multiply-adds: the file that includes this for the GPU is compiled with
// -fmad=false), so a device-driven pair loop takes the same steps as the
// host-driven one.
#pragma once

#include <math.h>

#include "../../include/sbci.h"
#include "sbci_internal.h"

namespace sbci {

enum PairHalt : int { PH_RUN = 0, PH_CONVERGED = 1, PH_CAP = 2, PH_UNDEF = 3, PH_NUMERIC = 4, PH_BOUND = 5 };

// The one combination of a step: inputs x^a, x^b, y^a, y^b, z^a, z^b and
// their H-images (12); outputs x^a, x^b, X^a, X^b, y^a, y^b, Y^a, Y^b,
// z'^a, z'^b (10).  Coefficient tables are [input][output] with row stride
// kDavMaxOut, the layout of the combination kernel.
constexpr int kPairIn = 12, kPairOut = 10;
constexpr int kPairDots = 21 + 36;  // upper triangle of S, then T in full

struct PairCoef {
  bool first;       // first-step path (Eq. S93): basis x^a, x^b, z^a, z^b
  int nb;           // basis vectors (4 or 6)
  double Vp[6][2];  // V' = P V, columns of the two lowest Ritz vectors
  double w[2];      // E_{t+1}^a, E_{t+1}^b
  double A[2][2], B[2][2], C[2][2], k[2];
};

struct PairCtl {
  // parameters of the pair (set by the host before the loop)
  double eps0, r0, b_th, eps1, x_th1, x_th2, r1;
  double Ec0;  // preconditioner shift of a later pair (Q3)
  int alpha, max_sigma, max_cycle2, trace_cap;
  // iteration state
  double E[2];  // E^a, E^b of the last step (E^a is the ground pair's shift)
  int first, t, nstep, sigma, restarts[4];
  int halt, restart, undef, ntrace;
  int bodies;  // steps begun: a backstop halts the loop past trace_cap of them
  // coefficients of the device-side combinations
  double comb[kPairIn * kDavMaxOut];
  double proj[(2 + kMaxStates) * kDavMaxOut];
  double scale[6 * kDavMaxOut];
  // the last step, for the host: Ritz values, coefficients, norms
  double w[2], k[2], B00, B11, C00, dz, nx[2];
  sbci_trace_record *trace;  // device ring of trace_cap records
};

// Symmetric eigen-problem of order n <= 6 by cyclic Jacobi, ascending
// eigenvalues, eigenvectors in the columns of V (row-major): the sweeps,
// rotations and sort of the library's host solver.
__host__ __device__ inline void pair_eigh(int n, const double *Ain, double *w, double *V) {
  double A[36];
  for (int i = 0; i < n * n; ++i) A[i] = Ain[i];
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) V[i * n + j] = (i == j) ? 1.0 : 0.0;
  for (int sweep = 0; sweep < 100; ++sweep) {
    double off = 0.0, diag = 0.0;
    for (int i = 0; i < n; ++i) {
      diag += A[i * n + i] * A[i * n + i];
      for (int j = i + 1; j < n; ++j) off += A[i * n + j] * A[i * n + j];
    }
    if (off <= 1e-36 * (diag + 1e-300)) break;
    for (int p = 0; p < n; ++p) {
      for (int q = p + 1; q < n; ++q) {
        const double apq = A[p * n + q];
        if (apq == 0.0) continue;
        const double app = A[p * n + p], aqq = A[q * n + q];
        const double theta = (aqq - app) / (2.0 * apq);
        const double t = (theta >= 0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
        const double c = 1.0 / sqrt(t * t + 1.0), s = t * c;
        for (int k = 0; k < n; ++k) {  // A <- A J (columns p, q)
          const double akp = A[k * n + p], akq = A[k * n + q];
          A[k * n + p] = c * akp - s * akq;
          A[k * n + q] = s * akp + c * akq;
        }
        for (int k = 0; k < n; ++k) {  // A <- J^T A (rows p, q)
          const double apk = A[p * n + k], aqk = A[q * n + k];
          A[p * n + k] = c * apk - s * aqk;
          A[q * n + k] = s * apk + c * aqk;
        }
        for (int k = 0; k < n; ++k) {  // V <- V J
          const double vkp = V[k * n + p], vkq = V[k * n + q];
          V[k * n + p] = c * vkp - s * vkq;
          V[k * n + q] = s * vkp + c * vkq;
        }
      }
    }
  }
  for (int i = 0; i < n; ++i) w[i] = A[i * n + i];
  for (int i = 0; i < n; ++i) {  // ascending (selection sort on columns)
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

// Canonical orthogonalisation (overlap eigenvalues below 1e-14 dropped, Q5),
// subspace eigen-problem of (T + T^T)/2 (Q4) and the coefficients of one pair
// step on the requested path.  S6 and T6 are the 6x6 overlap and T of
// (x^a, x^b, y^a, y^b, z^a, z^b) (rows and columns of y unused on the first
// path).  Returns false if the step is undefined on that path.
__host__ __device__ inline bool pair_coef(const double *S6, const double *T6, bool first, PairCoef *pc) {
  const int kFirst[4] = {0, 1, 4, 5};
  const int nb = first ? 4 : 6;
  double S[36], Hs[36], s[6], U[36];
  for (int i = 0; i < nb; ++i)
    for (int j = 0; j < nb; ++j) {
      const int a = first ? kFirst[i] : i, b = first ? kFirst[j] : j;
      S[i * nb + j] = S6[a * 6 + b];
      Hs[i * nb + j] = 0.5 * (T6[a * 6 + b] + T6[b * 6 + a]);
    }
  pair_eigh(nb, S, s, U);
  double P[36];  // nb x r
  int r = 0;
  for (int c = 0; c < nb; ++c) {
    if (!(s[c] >= 1e-14)) continue;
    const double f = 1.0 / sqrt(s[c]);
    for (int i = 0; i < nb; ++i) P[i * 6 + r] = U[i * nb + c] * f;
    ++r;
  }
  if (r < 2) return false;
  double Hh[36], w[6], V[36];
  for (int a = 0; a < r; ++a)
    for (int b = 0; b < r; ++b) {
      double acc = 0.0;
      for (int i = 0; i < nb; ++i)
        for (int j = 0; j < nb; ++j) acc += P[i * 6 + a] * Hs[i * nb + j] * P[j * 6 + b];
      Hh[a * r + b] = acc;
    }
  for (int a = 0; a < r; ++a)
    for (int b = 0; b < a; ++b) Hh[a * r + b] = Hh[b * r + a] = 0.5 * (Hh[a * r + b] + Hh[b * r + a]);
  pair_eigh(r, Hh, w, V);
  pc->first = first;
  pc->nb = nb;
  for (int i = 0; i < nb; ++i)
    for (int col = 0; col < 2; ++col) {
      double acc = 0.0;
      for (int a = 0; a < r; ++a) acc += P[i * 6 + a] * V[a * r + col];
      pc->Vp[i][col] = acc;
    }
  pc->w[0] = w[0];
  pc->w[1] = w[1];
  const double(*Vp)[2] = pc->Vp;
  double a_ab, a_ba, k0, k1;
  if (first) {  // Eq. S93
    k0 = 1.0 / Vp[0][0];
    k1 = 1.0 / Vp[1][1];
    a_ab = Vp[1][0] / Vp[0][0];
    a_ba = Vp[0][1] / Vp[1][1];
    pc->C[0][0] = -Vp[2][0] / Vp[0][0];
    pc->C[0][1] = -Vp[3][0] / Vp[0][0];
    pc->C[1][0] = -Vp[2][1] / Vp[1][1];
    pc->C[1][1] = -Vp[3][1] / Vp[1][1];
    pc->B[0][0] = pc->B[1][1] = 1.0;
    pc->B[0][1] = pc->B[1][0] = 0.0;
  } else {  // Eqs. S116, S117, S112, S121
    a_ab = Vp[1][0] / Vp[2][0];
    a_ba = Vp[0][1] / Vp[3][1];
    k0 = 1.0 / (Vp[0][0] - Vp[3][0] * a_ba);
    k1 = 1.0 / (Vp[1][1] - Vp[2][1] * a_ab);
    pc->B[0][0] = k0 * Vp[2][0];
    pc->B[0][1] = k0 * Vp[3][0];
    pc->B[1][0] = k1 * Vp[2][1];
    pc->B[1][1] = k1 * Vp[3][1];
    const double m00 = Vp[2][0], m01 = Vp[3][0], m10 = Vp[2][1], m11 = Vp[3][1];
    const double det = m00 * m11 - m01 * m10;
    if (!(isfinite(det) && det != 0.0)) return false;
    const double r00 = Vp[4][0], r01 = Vp[5][0], r10 = Vp[4][1], r11 = Vp[5][1];
    // C = -M^-1 R
    pc->C[0][0] = -(m11 * r00 - m01 * r10) / det;
    pc->C[0][1] = -(m11 * r01 - m01 * r11) / det;
    pc->C[1][0] = -(-m10 * r00 + m00 * r10) / det;
    pc->C[1][1] = -(-m10 * r01 + m00 * r11) / det;
  }
  pc->A[0][0] = pc->A[1][1] = 0.0;
  pc->A[0][1] = a_ab;
  pc->A[1][0] = a_ba;
  pc->k[0] = k0;
  pc->k[1] = k1;
  const double chk[] = {k0, k1, a_ab, a_ba, pc->B[0][0], pc->B[0][1], pc->B[1][0], pc->B[1][1],
                        pc->C[0][0], pc->C[0][1], pc->C[1][0], pc->C[1][1], w[0], w[1]};
  for (int i = 0; i < 14; ++i)
    if (!isfinite(chk[i])) return false;
  return true;
}

// r[i * alpha + j] = x_c^j . z^i -> coefficients of the combination
// (z^a, z^b, x_c^0 ..) -> (z^a, z^b).
__host__ __device__ inline void pair_proj_coef(PairCtl &s, const double *r) {
  const int na = s.alpha;
  for (int q = 0; q < 2 + na; ++q)
    for (int j = 0; j < 2; ++j) s.proj[q * kDavMaxOut + j] = 0.0;
  s.proj[0 * kDavMaxOut + 0] = 1.0;
  s.proj[1 * kDavMaxOut + 1] = 1.0;
  for (int j = 0; j < na; ++j)
    for (int i = 0; i < 2; ++i) {
      const double v = r[i * na + j];
      if (!isfinite(v)) s.halt = PH_NUMERIC;
      s.proj[(2 + j) * kDavMaxOut + i] = -v;
    }
}

// r: the kPairDots dots of the step basis b = (x^a, x^b, y^a, y^b, z^a, z^b),
// S upper triangle (a <= b) then T[a][b] = b_a . H b_b.  Sets halt on an
// undefined step or a non-finite dot.
__host__ __device__ inline void pair_after_dots(PairCtl &s, const double *r) {
  double S6[36], T6[36];
  int q = 0;
  for (int a = 0; a < 6; ++a)
    for (int b = a; b < 6; ++b, ++q) S6[a * 6 + b] = S6[b * 6 + a] = r[q];
  for (int a = 0; a < 6; ++a)
    for (int b = 0; b < 6; ++b, ++q) T6[a * 6 + b] = r[q];
  for (int i = 0; i < kPairDots; ++i)
    if (!isfinite(r[i])) {
      s.halt = PH_NUMERIC;
      return;
    }
  PairCoef pc;
  bool ok = false;
  if (!s.first) ok = pair_coef(S6, T6, false, &pc);
  if (!ok) ok = pair_coef(S6, T6, true, &pc);  // first step, or Q6
  if (!ok) {
    s.halt = PH_UNDEF;
    return;
  }
  s.undef = (pc.first && !s.first) ? 1 : 0;
  for (int i = 0; i < kPairIn * kDavMaxOut; ++i) s.comb[i] = 0.0;
  const int kFirst[4] = {0, 1, 4, 5};
  // input b6 is basis vector b6, input 6 + b6 its H-image; outputs x 0-1,
  // X 2-3, y 4-5, Y 6-7, z' 8-9
  auto C = [&](int qin, int out) -> double & { return s.comb[qin * kDavMaxOut + out]; };
  for (int i = 0; i < 2; ++i) {
    for (int j = 0; j < pc.nb; ++j) {
      const int b6 = pc.first ? kFirst[j] : j;
      C(b6, i) = pc.k[i] * pc.Vp[j][i];          // x_{t+1}^i (Q9)
      C(6 + b6, 2 + i) = pc.k[i] * pc.Vp[j][i];  // X_{t+1}^i
      C(b6, 8 + i) = -pc.w[i] * pc.Vp[j][i];     // z'^i = sum_j V'_{j,i} (H b_j - E b_j)
      C(6 + b6, 8 + i) = pc.Vp[j][i];
    }
    // y_{t+1}^i = y_t^i - C_{i0} z^a - C_{i1} z^b + A_{i,1-i} x^{1-i}
    if (!pc.first) {
      C(2 + i, 4 + i) = 1.0;
      C(6 + 2 + i, 6 + i) = 1.0;
    }
    for (int j = 0; j < 2; ++j) {
      C(4 + j, 4 + i) = -pc.C[i][j];
      C(6 + 4 + j, 6 + i) = -pc.C[i][j];
    }
    C(1 - i, 4 + i) = pc.A[i][1 - i];
    C(6 + 1 - i, 6 + i) = pc.A[i][1 - i];
  }
  s.w[0] = pc.w[0];
  s.w[1] = pc.w[1];
  s.k[0] = pc.k[0];
  s.k[1] = pc.k[1];
  s.B00 = pc.B[0][0];
  s.B11 = pc.B[1][1];
  s.C00 = pc.C[0][0];
  s.sigma += 2;  // the step's two H-products
}

// r = (|z'^a|^2, |z'^b|^2, |x^a|^2, |x^b|^2) after the combination.  With
// the host's record, convergence test, restart causes and cap.
__host__ __device__ inline void pair_decide(PairCtl &s, const double *r) {
  for (int i = 0; i < 4; ++i)
    if (!isfinite(r[i])) {
      s.halt = PH_NUMERIC;
      return;
    }
  ++s.nstep;
  const double dz = sqrt(r[0]);
  const double nx0 = sqrt(r[2]), nx1 = sqrt(r[3]);  // |x_{t+1}| (= |k| up to rounding)
  const double dE = fabs(s.w[0] - s.E[0]);
  s.dz = dz;
  s.nx[0] = nx0;
  s.nx[1] = nx1;
  sbci_trace_record rec;
  rec.state = s.alpha;
  rec.t = s.t;
  rec.energy = s.w[0];
  rec.b = s.B00;
  rec.c = s.C00;
  rec.k = s.k[0];
  rec.dE = dE;
  rec.dz = dz;
  rec.event = s.undef ? 8 : 0;
  rec.prec = SBCI_FP64;
  rec.s136 = 0.0;
  s.restart = 0;
  auto push = [&]() {
    if (s.ntrace < s.trace_cap) s.trace[s.ntrace] = rec;
    ++s.ntrace;
  };
  const double ak0 = fabs(s.k[0]), ak1 = fabs(s.k[1]);
  if (dE < s.eps0 && dz < s.r0) {  // Eq. S99 / S127
    rec.event = 1;
    push();
    s.halt = PH_CONVERGED;
    return;
  }
  int cause = -1;  // Section S2.5
  if ((fabs(s.B00) < s.b_th || fabs(s.B11) < s.b_th) && dE < s.eps1) cause = 0;
  else if (fmin(ak0, ak1) < s.x_th1 || fmax(ak0, ak1) > s.x_th2) cause = 1;
  else if (dz > s.r1 && s.t > 0) cause = 2;
  else if (s.t + 1 >= s.max_cycle2) cause = 3;
  s.E[0] = s.w[0];
  s.E[1] = s.w[1];
  if (cause >= 0) {  // Q7: x, X normalised; z'_0 = X_0 - E_0 x_0 = z'_{t+1} k / |x_{t+1}|
    ++s.restarts[cause];
    rec.event = 2 + cause;
    push();
    const double f[6] = {1.0 / nx0, 1.0 / nx1, 1.0 / nx0, 1.0 / nx1, s.k[0] / nx0, s.k[1] / nx1};
    for (int q = 0; q < 6; ++q)
      for (int j = 0; j < 6; ++j) s.scale[q * kDavMaxOut + j] = q == j ? f[q] : 0.0;
    s.restart = 1;
    s.first = 1;
    s.t = 0;
  } else {
    push();
    s.first = 0;
    ++s.t;
  }
  if (s.sigma >= s.max_sigma) s.halt = PH_CAP;  // Q8 (checked where the next step would start)
}

}  // namespace sbci
