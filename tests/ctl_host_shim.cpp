// Host build of the device controller's decision logic (csrc/ctl.h) for the
// CPU tests: the same source the GPU runs on one thread, compiled by g++, with
// plain-array entry points for ctypes.  Test infrastructure only.
#include <cstring>

#include "ctl.h"

using namespace sbci;

namespace {

void set_params(CtlParams &p, const double *pr, const int *ip) {
  p.eps0 = pr[0];
  p.r0 = pr[1];
  p.b_th = pr[2];
  p.eps1 = pr[3];
  p.x_th1 = pr[4];
  p.x_th2 = pr[5];
  p.r1 = pr[6];
  p.mixed_eps = pr[7];
  p.mixed_r = pr[8];
  p.gs_tol = pr[9];
  p.guard = 1e-8;
  p.max_cycle = ip[0];
  p.max_sigma = ip[1];
  p.refine_max_sigma = ip[2];
  p.user_prec = ip[3];
}

}  // namespace

extern "C" {

// One subspace solve (Eqs. S10-S24 or S33-S55, reading R15 included).
// dots: the 13 step dots in slot order S_NXX .. S_HZZ; first: first-step path
// on x_0 = sx x.  out: E, b, c, k, E2, r[0..2], sx, sy, first-after (0/1),
// event of the pending record.  Returns the halt code.
int host_ctl_solve(const double *dots, int first, double sx, double gs_tol, double *out) {
  static CtlState st;
  std::memset(&st, 0, sizeof(st));
  CtlHead &s = st;
  s.p.gs_tol = gs_tol;
  s.p.max_sigma = 1 << 30;
  s.p.max_cycle = 20;
  for (int i = 0; i <= S_HZZ; ++i) s.dots[i] = dots[i];
  s.first = first;
  s.sx_pending = sx;
  s.prec = SBCI_FP64;
  s.trace_ptr = st.trace;
  ctl_solve(s);
  out[0] = s.up.E;
  out[1] = s.up.b;
  out[2] = s.up.c;
  out[3] = s.pending.k;
  out[4] = s.E2;
  out[5] = s.second[0];
  out[6] = s.second[1];
  out[7] = s.second[2];
  out[8] = s.up.sx;
  out[9] = s.up.sy;
  out[10] = s.first;
  out[11] = s.pending.event;
  return s.halt;
}

// One end-of-step decision (Eq. S61, Eqs. S62a-c, max_cycle, the
// low-precision stage and refinement windows, the caps).
// pr: eps0, r0, b_th, eps1, x_th1, x_th2, r1, mixed_eps, mixed_r, gs_tol,
//     E_t, E_{t+1}, b, c, k
// ip: max_cycle, max_sigma, refine_max_sigma, user_prec, prec, stage, alpha,
//     t, n_sigma, n_stage1, n_sync
// dots: S_NXX, S_NXY, S_NYY, S_ZPZP after the update
// out_i: event of the committed record, t after, first after, restarts of
// causes a, b, c, max.  Returns the halt code.
int host_ctl_check(const double *pr, const int *ip, const double *dots, int *out_i) {
  static CtlState st;
  std::memset(&st, 0, sizeof(st));
  CtlHead &s = st;
  set_params(s.p, pr, ip);
  s.prec = ip[4];
  s.stage = ip[5];
  s.alpha = ip[6];
  s.t = ip[7];
  s.n_sigma = ip[8];
  s.n_stage1 = ip[9];
  s.n_sync = ip[10];
  s.E = pr[10];
  s.E_solve = pr[11];
  s.pending.state = s.alpha;
  s.pending.t = s.t;
  s.pending.energy = pr[11];
  s.pending.b = pr[12];
  s.pending.c = pr[13];
  s.pending.k = pr[14];
  s.pending.prec = s.prec;
  s.pending_check = 1;
  s.dots[S_NXX] = dots[0];
  s.dots[S_NXY] = dots[1];
  s.dots[S_NYY] = dots[2];
  s.dots[S_ZPZP] = dots[3];
  s.trace_ptr = st.trace;
  ctl_check(s);
  out_i[0] = s.ntrace > 0 ? st.trace[0].event : -1;
  out_i[1] = s.t;
  out_i[2] = s.first;
  for (int i = 0; i < 4; ++i) out_i[3 + i] = s.n_restart[i];
  return s.halt;
}

int host_ctl_sizes(int *out) {
  out[0] = (int)S_HZZ;
  out[1] = (int)sizeof(sbci_trace_record);
  return 0;
}

}  // extern "C"
