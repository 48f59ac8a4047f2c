// Host build of the SBCI2 pair controller (csrc/pair_ctl.h) for the CPU
// tests: the source the GPU runs on one thread, compiled by g++, with
// plain-array entry points for ctypes.  Test infrastructure only.
#include <cstring>

#include "pair_ctl.h"

using namespace sbci;

extern "C" {

// pair_coef on a 6x6 overlap S and T (row-major).  out: w0, w1, k0, k1,
// a_ab, a_ba, B (4, row-major), C (4), V' (6 x 2, row-major, rows of the
// path's basis), nb.  Returns 1 if the step is defined on that path.
int host_pair_coef(const double *S6, const double *T6, int first, double *out) {
  PairCoef pc;
  std::memset(&pc, 0, sizeof(pc));
  if (!pair_coef(S6, T6, first != 0, &pc)) return 0;
  out[0] = pc.w[0];
  out[1] = pc.w[1];
  out[2] = pc.k[0];
  out[3] = pc.k[1];
  out[4] = pc.A[0][1];
  out[5] = pc.A[1][0];
  for (int i = 0; i < 2; ++i)
    for (int j = 0; j < 2; ++j) {
      out[6 + 2 * i + j] = pc.B[i][j];
      out[10 + 2 * i + j] = pc.C[i][j];
    }
  for (int i = 0; i < 6; ++i)
    for (int c = 0; c < 2; ++c) out[14 + 2 * i + c] = pc.Vp[i][c];
  out[26] = pc.nb;
  return 1;
}

// One decision (pair_decide) on constructed scalars.  par: eps0, r0, b_th,
// eps1, x_th1, x_th2, r1; ip: max_sigma, max_cycle2, t, sigma, first;
// st: E0, E1, w0, w1, k0, k1, B00, B11; norms: |z'^a|^2, |z'^b|^2, |x^a|^2,
// |x^b|^2.  out: halt, event of the record, restart, first, t, scale factors
// (6), E0, E1.
void host_pair_decide(const double *par, const int *ip, const double *st, const double *norms, double *out) {
  static PairCtl s;
  static sbci_trace_record tr[4];
  std::memset(&s, 0, sizeof(s));
  s.eps0 = par[0];
  s.r0 = par[1];
  s.b_th = par[2];
  s.eps1 = par[3];
  s.x_th1 = par[4];
  s.x_th2 = par[5];
  s.r1 = par[6];
  s.max_sigma = ip[0];
  s.max_cycle2 = ip[1];
  s.t = ip[2];
  s.sigma = ip[3];
  s.first = ip[4];
  s.E[0] = st[0];
  s.E[1] = st[1];
  s.w[0] = st[2];
  s.w[1] = st[3];
  s.k[0] = st[4];
  s.k[1] = st[5];
  s.B00 = st[6];
  s.B11 = st[7];
  s.trace = tr;
  s.trace_cap = 4;
  pair_decide(s, norms);
  out[0] = s.halt;
  out[1] = s.ntrace > 0 ? tr[0].event : -1;
  out[2] = s.restart;
  out[3] = s.first;
  out[4] = s.t;
  for (int q = 0; q < 6; ++q) out[5 + q] = s.scale[q * kDavMaxOut + q];
  out[11] = s.E[0];
  out[12] = s.E[1];
}

}  // extern "C"
