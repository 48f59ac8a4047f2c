// C ABI of libsbci: context and integral preparation, the sigma entry point,
// and the driver of SBCI1 (Algorithm 1 with Sections S1.1-S1.5).
//
// The SB steps run under a device-resident controller (ctl.h): one step is
//   update sweep (Eqs. 10-11, S56-S60; preconditioner Eqs. 6-7) whose last
//   block runs the convergence / restart test (Eqs. S61, S62)
//   -> projection against stored states (Eq. S31)
//   -> sigma of the next z (Eq. S32), whose last block solves the 2x2
//      (Eqs. S10-S24) or 3x3 (Eqs. S33-S55) subspace problem,
// and a CUDA graph repeats that body in a device-side while loop until the
// controller halts.  The host only handles the rare events: a state has
// converged (store it, start the next from the second Ritz vector, S1.4),
// the low-precision stage has ended (re-sync X = H x in FP64), a cap.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <queue>
#include <string>
#include <vector>

#include <cstddef>

#include "../../include/sbci.h"
#include "ctl.h"
#include "batch.h"
#include "lowrank.h"
#include "pair_ctl.h"
#include "pool.h"
#include "sbci_internal.h"
#include "step.h"

namespace sbci {
static thread_local std::string g_err;
void set_error(const std::string &msg) { g_err = msg; }
std::string last_error() { return g_err; }
}  // namespace sbci

using namespace sbci;

#define CK(expr)                                                                      \
  do {                                                                                \
    cudaError_t _e = (expr);                                                          \
    if (_e != cudaSuccess) {                                                          \
      set_error(std::string("CUDA error ") + cudaGetErrorName(_e) + " (" +            \
                cudaGetErrorString(_e) + ") at " + #expr);                            \
      return (_e == cudaErrorMemoryAllocation) ? SBCI_ERR_NOMEM : SBCI_ERR_CUDA;      \
    }                                                                                 \
  } while (0)

#define RET(st)                         \
  do {                                  \
    sbci_status _s = (st);              \
    if (_s != SBCI_OK) return _s;       \
  } while (0)

namespace {

// Per-kernel launch counts (always) and CUDA-event times on the context stream
// (when profiling is enabled).
enum Kid { K_GC = 0, K_SC, K_UPD, K_PROJ, K_RED, K_LIN, K_DOTS, K_DIAG, K_GCTC, K_SF,
           K_DAVD, K_DAVC, K_DAVP, K_GCOS, K_GCLR, K_FC, K_GCBF, K_GCTCLR, K_PAIR, K_COUNT };
const char *const kKidName[K_COUNT] = {"sigma_gather_contract", "sigma_scatter", "sb_update",
                                       "sb_project", "reduce", "lincomb", "dots", "diagonal",
                                       "sigma_gather_contract_tc", "sigma_symfinish",
                                       "davidson_dots", "davidson_combine", "davidson_precond",
                                       "sigma_gather_contract_os", "sigma_gather_contract_lr",
                                       "sigma_fused_column", "sigma_gather_contract_bf16",
                                       "sigma_gather_contract_tc_lr", "sbci2_pair_ctl"};

struct Prof {
  bool on = false;
  long long launches[K_COUNT] = {};
  double ms[K_COUNT] = {};
  std::vector<cudaEvent_t> pool;
  size_t used = 0;
  std::vector<int> kid;
};

struct Solver {
  bool active = false, done = false;
  int k = 0;
  sbci_params p{};
  // device vectors [ndet] each
  double *x = nullptr, *X = nullptr, *y = nullptr, *Y = nullptr, *w = nullptr;
  double *z[2] = {nullptr, nullptr}, *Z[2] = {nullptr, nullptr};
  double *xc = nullptr;  // [k][ndet]
  float *zf = nullptr;   // FP32 copy of the next z (split and FP32 sigma modes)
  double *pinv = nullptr;  // excited-state preconditioner 1 / guarded(D - Ec0)
  CtlState *d_ctl = nullptr;  // device controller state
  CtlState *h_ctl = nullptr;  // pinned host mirror
  unsigned int *d_counters = nullptr;
  int verified = 0;  // the current state passed its FP64 residual check
  std::vector<double> Ec;
  std::vector<sbci_report> rep;
  std::vector<sbci_trace_record> trace;
  int any_unconverged = 0;
  // while-loop graphs, one per sigma precision
  cudaGraph_t graph[4] = {};
  cudaGraphExec_t gexec[4] = {};
};

}  // namespace

struct sbci_ctx {
  int n = 0, ne_a = 0, ne_b = 0;
  StringSet sa, sb;
  int Na = 0, Nb = 0, npair = 0, npair_pad = 0;
  long long ndet = 0;
  double e_core = 0.0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  int grid = 0;
  uint32_t *d_link_a = nullptr, *d_link_b = nullptr, *d_mask_b = nullptr;
  uint32_t *d_link_bT = nullptr;  // beta lists transposed, [nlink_b][Nb]
  double *d_W = nullptr;
  float *d_Wf = nullptr;
  float *d_cf = nullptr;      // FP32 copy of a plain sigma's input (tensor-core mode)
  uint32_t *d_Wtc = nullptr;  // TF32 hi/lo operand B of the tensor-core sigma (nullptr: unsupported)
  uint16_t *d_Wbf = nullptr;  // BF16 hi/lo operand B of the BF16x3 sigma (nullptr: unsupported)
  int bf_grid = 0;            // CTAs of the BF16x3 kernel (0: unsupported shape)
  void *d_Wos = nullptr;      // BF16 integer slices of W for the FP64 tensor-core contraction (nullptr: off)
  int *d_fexp = nullptr;      // their per-output-pair exponents
  int os_grid = 0;
  // factored form W = F M F^T of the FP64 SIMT contraction (lowrank.h, df_factor): its rank, 0: off
  int lr_rank = 0;
  void *d_lrUt64 = nullptr, *d_lrUL64 = nullptr;
  // the same factor as pre-split TF32 operands of the factored tensor-core
  // contraction (kernels_tclr.cu), and that kernel's CTAs (0: full form)
  uint32_t *d_Wtclr = nullptr;
  int tclr_grid = 0;
  bool tclr_first = false;  // SBCI_TC_LOWRANK=1: the factored form also where the full one fits
  double *d_diag = nullptr;
  double *d_ea = nullptr, *d_eb = nullptr, *d_ja = nullptr;
  void *d_G = nullptr;
  size_t G_bytes = 0;
  double *d_partials = nullptr, *d_result = nullptr, *h_result = nullptr;
  int *d_status = nullptr, *h_status = nullptr;  // device error word (bounded waits)
  cudaEvent_t ev_fence = nullptr;  // marks the end of the host-issued work on the context stream
  int nsm = 1;
  int device = -1;  // the CUDA device the context was created on
  int tc_grid = 0;  // resident CTAs of the tensor-core kernel (0: unsupported shape)
  int tcp_grid = 0;  // resident CTAs of its pipelined form (0: the plain kernel)
  bool sbci2_device = false;  // SBCI_SBCI2_DEVICE=1: SBCI2 pair steps on the device controller
  int fc_grid = 0;  // CTAs of the column-fused sector kernel (0: unsupported shape or turned off)
  uint16_t *d_fc_link_a = nullptr;  // its 16-bit alpha links (J | pair << 8 | sign << 15)
  double *d_tmp_in = nullptr, *d_tmp_out = nullptr;  // staging for host sigma calls
  size_t tmp_elems = 0;
  std::vector<double> W_host;
  Solver s;
  Prof prof;
};

namespace {

sbci_status check_finite(const double *v, size_t n, const char *what) {
  for (size_t i = 0; i < n; ++i)
    if (!std::isfinite(v[i])) {
      set_error(std::string("non-finite value in ") + what);
      return SBCI_ERR_NUMERIC;
    }
  return SBCI_OK;
}

template <typename T>
sbci_status dmalloc(T **p, size_t count) {
  *p = nullptr;
  if (count == 0) count = 1;
  CK(pool_malloc((void **)p, count * sizeof(T)));
  return SBCI_OK;
}

sbci_status ensure_G(sbci_ctx *c, int prec) {
  const size_t need = sigma_scratch_bytes(c->npair, c->ndet, prec == SBCI_FP64 ? 0 : 1);
  if (c->G_bytes >= need) return SBCI_OK;
  if (c->d_G) {
    CK(cudaStreamSynchronize(c->stream));  // queued kernels may still read the old scratch
    CK(pool_free(c->d_G));
  }
  c->d_G = nullptr;
  c->G_bytes = 0;
  CK(pool_malloc(&c->d_G, need));
  c->G_bytes = need;
  return SBCI_OK;
}

sbci_status prof_flush(sbci_ctx *c) {
  Prof &p = c->prof;
  for (size_t i = 0; i < p.kid.size(); ++i) {
    float ms = 0.0f;
    CK(cudaEventSynchronize(p.pool[2 * i + 1]));
    CK(cudaEventElapsedTime(&ms, p.pool[2 * i], p.pool[2 * i + 1]));
    p.ms[p.kid[i]] += ms;
  }
  p.kid.clear();
  p.used = 0;
  return SBCI_OK;
}

// Launch wrapper: counts the launch and, when profiling, brackets it with events.
template <typename F>
sbci_status timed(sbci_ctx *c, int kid, F &&launch) {
  Prof &p = c->prof;
  p.launches[kid] += 1;
  if (!p.on) {
    CK(launch());
    return SBCI_OK;
  }
  if (p.used + 2 > 8192) RET(prof_flush(c));
  while (p.pool.size() < p.used + 2) {
    cudaEvent_t e;
    CK(cudaEventCreate(&e));
    p.pool.push_back(e);
  }
  CK(cudaEventRecord(p.pool[p.used], c->stream));
  CK(launch());
  CK(cudaEventRecord(p.pool[p.used + 1], c->stream));
  p.used += 2;
  p.kid.push_back(kid);
  return SBCI_OK;
}

// SBCI_ERR_INVALID for a precision this context cannot run (TF32x3 beyond
// n = 14, BF16x3 beyond n = 16).
sbci_status check_prec(const sbci_ctx *c, int prec) {
  if (prec == SBCI_FP64 || prec == SBCI_FP32) return SBCI_OK;
  if (prec == SBCI_TF32X3) {
    int Kp, Np;
    uint32_t cols;
    size_t smem;
    if ((tc_dims(c->npair, &Kp, &Np, &cols, &smem) && c->tc_grid > 0) || c->tclr_grid > 0) return SBCI_OK;
    set_error("SBCI_TF32X3: operands of this orbital count exceed shared memory (n <= 14, n = 15 with "
              "density-fitted integrals); use SBCI_BF16X3 or SBCI_FP32");
    return SBCI_ERR_INVALID;
  }
  if (prec == SBCI_BF16X3) {
    if (c->d_Wbf && c->bf_grid > 0) return SBCI_OK;
    set_error("SBCI_BF16X3: not available for this space");
    return SBCI_ERR_INVALID;
  }
  set_error("unknown precision mode");
  return SBCI_ERR_INVALID;
}

// The gather + contract kernel family of a sigma precision, and its launch.
int gc_kid(const sbci_ctx *c, int prec) {
  if (prec == SBCI_TF32X3) return c->tclr_grid > 0 && (c->tc_grid <= 0 || c->tclr_first) ? K_GCTCLR : K_GCTC;
  if (prec == SBCI_BF16X3) return K_GCBF;
  if (prec == SBCI_FP64 && c->d_Wos) return K_GCOS;
  if (prec == SBCI_FP64 && c->lr_rank > 0) return K_GCLR;
  return K_GC;
}

cudaError_t launch_gc(const sbci_ctx *c, const SigmaArgs &a, int prec) {
  switch (gc_kid(c, prec)) {
    case K_GCTC:
      if (c->tcp_grid > 0) return launch_gather_contract_tcp(a, c->d_status, c->tcp_grid, c->stream);
      return launch_gather_contract_tc(a, c->d_status, c->tc_grid, c->stream);
    case K_GCTCLR:
      return launch_gather_contract_tclr(a, c->d_Wtclr, c->lr_rank, c->d_status, c->tclr_grid, c->stream);
    case K_GCBF:
      return launch_gather_contract_bf(a, c->d_Wbf, c->d_status, c->bf_grid, c->stream);
    case K_GCOS:
      return launch_gather_contract_os(a, c->d_Wos, c->d_fexp, c->d_status, c->os_grid, c->stream);
    case K_GCLR:
      return launch_gather_contract_lr(a, 0, c->d_lrUt64, c->d_lrUL64, c->lr_rank, c->stream);
    default:
      return launch_gather_contract(a, prec == SBCI_FP64 ? 0 : 1, c->stream);
  }
}

// Arguments of a plain (not device-controlled) sigma out = H in.
SigmaArgs plain_sigma_args(const sbci_ctx *c, const double *in, double *out) {
  SigmaArgs a{};
  a.c = in;
  a.sigma = out;
  a.G = c->d_G;
  a.link_a = c->d_link_a;
  a.link_b = c->d_link_b;
  a.link_bT = c->d_link_bT;
  a.W = c->d_W;
  a.Wf = c->d_Wf;
  a.Wtc = c->d_Wtc;
  a.na = c->Na;
  a.nb = c->Nb;
  a.nlink_a = c->sa.nlink;
  a.nlink_b = c->sb.nlink;
  a.npair = c->npair;
  a.npair_pad = c->npair_pad;
  a.ndet = c->ndet;
  a.partials = c->d_partials;  // (no dots: dot_u all null)
  a.grid = scatter_grid(c->ndet, c->nsm);
  return a;
}

// sigma of one device vector in the given precision (out = H in).
sbci_status run_sigma(sbci_ctx *c, const double *in, double *out, int prec) {
  RET(check_prec(c, prec));
  RET(ensure_G(c, prec));
  SigmaArgs a = plain_sigma_args(c, in, out);
  const int p32 = (prec == SBCI_FP64) ? 0 : 1;
  if (prec == SBCI_TF32X3 || prec == SBCI_BF16X3) {  // the tensor-core gathers read an FP32 copy
    if (!c->d_cf) RET(dmalloc(&c->d_cf, (size_t)c->ndet));
    CK(launch_to_float(in, c->d_cf, c->ndet, c->stream));
    a.cf = c->d_cf;
  }
  RET(timed(c, gc_kid(c, prec), [&] { return launch_gc(c, a, prec); }));
  RET(timed(c, K_SC, [&] { return launch_scatter(a, p32, c->stream); }));
  return SBCI_OK;
}

// The reduction of slots [s0, s1) and the copies of its results and of the
// status word to the host, queued on the context stream (fetch_complete waits).
sbci_status reduce_issue(sbci_ctx *c, int s0, int s1, int grid) {
  RET(timed(c, K_RED, [&] { return launch_reduce(c->d_partials, grid, s0, s1, c->d_result, c->stream); }));
  CK(cudaMemcpyAsync(c->h_result + s0, c->d_result + s0, sizeof(double) * (s1 - s0),
                     cudaMemcpyDeviceToHost, c->stream));
  CK(cudaMemcpyAsync(c->h_status, c->d_status, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  return SBCI_OK;
}

sbci_status fetch_complete(sbci_ctx *c, int s0, int s1) {
  CK(cudaStreamSynchronize(c->stream));
  if (*c->h_status != 0) {
    set_error("a bounded device wait ran out (tensor-core MMA completion)");
    return SBCI_ERR_TIMEOUT;
  }
  for (int i = s0; i < s1; ++i)
    if (!std::isfinite(c->h_result[i])) {
      set_error("non-finite dot product in a device reduction");
      return SBCI_ERR_NUMERIC;
    }
  return SBCI_OK;
}

sbci_status reduce_and_fetch(sbci_ctx *c, int s0, int s1, int grid) {
  RET(reduce_issue(c, s0, s1, grid));
  return fetch_complete(c, s0, s1);
}

// dots over up to 16 pairs, results in h_result[S_GEN0 + i] once
// fetch_complete(c, S_GEN0, S_GEN0 + u.size()) has returned
sbci_status gen_dots_issue(sbci_ctx *c, const std::vector<const double *> &u, const std::vector<const double *> &v) {
  // about four elements per thread, at most the partials' capacity of blocks
  long long g = (c->ndet + 1023) / 1024;
  if (g > c->grid) g = c->grid;
  if (g < 1) g = 1;
  const int grid = (int)g;
  RET(timed(c, K_DOTS, [&] {
    return launch_dots(u.data(), v.data(), (int)u.size(), c->ndet, c->d_partials, grid, c->stream);
  }));
  return reduce_issue(c, S_GEN0, S_GEN0 + (int)u.size(), grid);
}

sbci_status gen_dots(sbci_ctx *c, std::vector<const double *> u, std::vector<const double *> v) {
  RET(gen_dots_issue(c, u, v));
  return fetch_complete(c, S_GEN0, S_GEN0 + (int)u.size());
}

sbci_status lincomb(sbci_ctx *c, double *out, std::vector<const double *> in, std::vector<double> co) {
  RET(timed(c, K_LIN, [&] { return launch_lincomb(out, in.data(), co.data(), (int)in.size(), c->ndet, c->stream); }));
  return SBCI_OK;
}

// ---------------------------------------------------------------------------
// SBCI1 driver around the device controller

double shift_for(const sbci_ctx *c, int alpha, double E) {
  return alpha == 0 ? E : c->s.Ec[0];  // newest ground-state Rayleigh quotient (Eqs. 6-7)
}

// Copies the controller header (and any committed trace records) to the host.
sbci_status ctl_read(sbci_ctx *c) {
  Solver &s = c->s;
  const size_t hdr = sizeof(CtlHead);
  CK(cudaMemcpyAsync(s.h_ctl, s.d_ctl, hdr, cudaMemcpyDeviceToHost, c->stream));
  CK(cudaMemcpyAsync(c->h_status, c->d_status, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  if (*c->h_status != 0) {
    set_error("a bounded device wait ran out (tensor-core MMA completion)");
    return SBCI_ERR_TIMEOUT;
  }
  const int n = std::min(s.h_ctl->ntrace, kTraceCap);
  if (n > 0) {
    CK(cudaMemcpyAsync(s.h_ctl->trace, s.d_ctl->trace, sizeof(sbci_trace_record) * n,
                       cudaMemcpyDeviceToHost, c->stream));
    CK(cudaMemsetAsync(&s.d_ctl->ntrace, 0, sizeof(int), c->stream));
    CK(cudaStreamSynchronize(c->stream));
    s.trace.insert(s.trace.end(), s.h_ctl->trace, s.h_ctl->trace + n);
    s.h_ctl->ntrace = 0;
  }
  return SBCI_OK;
}

sbci_status ctl_write(sbci_ctx *c) {
  Solver &s = c->s;
  s.h_ctl->ntrace = 0;
  CK(cudaMemcpyAsync(s.d_ctl, s.h_ctl, sizeof(CtlHead), cudaMemcpyHostToDevice, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  return SBCI_OK;
}

StepArgs step_args(sbci_ctx *c, unsigned long long cond) {
  Solver &s = c->s;
  StepArgs a{};
  a.ctl = s.d_ctl;
  a.x = s.x;
  a.X = s.X;
  a.y = s.y;
  a.Y = s.Y;
  a.w = s.w;
  a.diag = c->d_diag;
  a.xc = s.xc;
  a.pinv = s.pinv;
  a.n = c->ndet;
  a.sector = s.p.sector;
  a.na = c->Na;
  a.nb = c->Nb;
  a.partials = c->d_partials;
  a.counter = s.d_counters;
  a.cond = cond;
  return a;
}

// The singlet-sector split needs c = c^T exactly (the projection symmetrises
// z in sector mode) and the same strings for both spins.
bool use_symfin(const sbci_ctx *c) { return c->s.p.sector != 0 && c->ne_a == c->ne_b; }

SigmaArgs sigma_ctl_args(sbci_ctx *c, int prec, unsigned long long cond) {
  Solver &s = c->s;
  SigmaArgs a{};
  ctx_sigma_args(c, &a, nullptr);
  a.G = c->d_G;
  a.dot_u[0] = s.x;
  a.dot_u[1] = s.y;
  a.dot_u[2] = nullptr;  // the controller's next z
  a.dot_slot[0] = S_HXZ;
  a.dot_slot[1] = S_HYZ;
  a.dot_slot[2] = S_HZZ;
  a.partials = c->d_partials;
  a.grid = scatter_grid(c->ndet, c->nsm);
  if (use_symfin(c)) {  // singlet sector: sigma = A + A^T, A kept in w (free after the projection)
    a.symA = s.w;
    a.sf_grid = symfin_grid(c->Na, c->nsm);
  }
  a.ctl = s.d_ctl;
  a.counter = s.d_counters + 2;
  a.cond = cond;
  return a;
}

// Virtual blocks of the update and projection sweeps: a singlet-sector solve
// sweeps pairs of 16 x 16 tiles, four tile pairs per virtual block (each
// block ends with an FP64 reduction of its 19 dot products, which costs as
// many FP64 instructions as about one tile pair of the sweep itself); every
// other solve ~4 elements per thread.
int step_blocks(const sbci_ctx *c) {
  if (!use_symfin(c)) return step_grid(c->ndet, c->nsm);
  const long long T = (c->Na + 15) / 16, units = T * (T + 1) / 2;
  return (int)std::max(1LL, std::min((units + 3) / 4, (long long)c->grid));
}

// The sector sigma of a TF32x3 step runs as the column-fused kernel (gather,
// contraction and alpha-only scatter in one launch, G never in global memory)
// where the shape allows it.
bool use_fused(const sbci_ctx *c, int prec) { return prec == SBCI_TF32X3 && use_symfin(c) && c->fc_grid > 0; }

// Counts the kernels of `bodies` step bodies run by a graph.
void count_bodies(sbci_ctx *c, int prec, long long bodies) {
  Prof &pf = c->prof;
  pf.launches[K_UPD] += bodies;
  pf.launches[K_PROJ] += bodies;
  if (use_fused(c, prec)) {
    pf.launches[K_FC] += bodies;
  } else {
    pf.launches[gc_kid(c, prec)] += bodies;
    pf.launches[K_SC] += bodies;
  }
  if (use_symfin(c)) pf.launches[K_SF] += bodies;
}

// One step body: update -> projection -> sigma (gather+contract, scatter, or
// the column-fused kernel) -> symmetric finish (singlet sector).
// timing = 1: each launch is counted and bracketed with events (not in capture).
sbci_status launch_body(sbci_ctx *c, int prec, unsigned long long cond, bool timing) {
  const StepArgs st = step_args(c, cond);
  const SigmaArgs sa = sigma_ctl_args(c, prec, cond);
  const int g = step_blocks(c);
  const int p32 = (prec == SBCI_FP64) ? 0 : 1;
  auto L = [&](int kid, auto &&f) -> sbci_status {
    if (timing) return timed(c, kid, f);
    CK(f());
    return SBCI_OK;
  };
  RET(L(K_UPD, [&] { return launch_update_ctl(st, g, c->stream); }));
  RET(L(K_PROJ, [&] { return launch_project_ctl(st, g, c->stream); }));
  if (use_fused(c, prec)) {
    RET(L(K_FC, [&] { return launch_fused_column(sa, c->d_status, c->fc_grid, c->stream); }));
  } else {
    RET(L(gc_kid(c, prec), [&] { return launch_gc(c, sa, prec); }));
    RET(L(K_SC, [&] { return launch_scatter(sa, p32, c->stream); }));
  }
  if (sa.symA) RET(L(K_SF, [&] { return launch_symfin(sa, p32, c->stream); }));
  return SBCI_OK;
}

// While-loop graph over the step body for one sigma precision.
sbci_status build_graph(sbci_ctx *c, int prec) {
  Solver &s = c->s;
  cudaGraph_t g = nullptr;
  CK(cudaGraphCreate(&g, 0));
  cudaGraphConditionalHandle h;
  CK(cudaGraphConditionalHandleCreate(&h, g, 1u, cudaGraphCondAssignDefault));
  cudaGraphNodeParams np{};
  np.type = cudaGraphNodeTypeConditional;
  np.conditional.handle = h;
  np.conditional.type = cudaGraphCondTypeWhile;
  np.conditional.size = 1;
  cudaGraphNode_t node;
  CK(cudaGraphAddNode(&node, g, nullptr, nullptr, 0, &np));
  cudaGraph_t body = np.conditional.phGraph_out[0];
  CK(cudaStreamBeginCaptureToGraph(c->stream, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
  sbci_status st = launch_body(c, prec, (unsigned long long)h, false);
  cudaGraph_t captured = nullptr;
  cudaError_t e = cudaStreamEndCapture(c->stream, &captured);
  if (st != SBCI_OK) return st;
  CK(e);
  CK(cudaGraphInstantiate(&s.gexec[prec], g, 0));
  s.graph[prec] = g;
  return SBCI_OK;
}

bool use_graphs(const sbci_ctx *c) {
  if (c->prof.on) return false;  // per-kernel event timing needs separate launches
  const char *e = std::getenv("SBCI_NO_GRAPH");
  return !(e && e[0] == '1');
}

// Runs step bodies until the controller halts.
sbci_status run_until_halt(sbci_ctx *c) {
  Solver &s = c->s;
  const int prec = s.h_ctl->prec;
  if (use_graphs(c)) {
    if (!s.gexec[prec]) RET(build_graph(c, prec));
    CK(cudaGraphLaunch(s.gexec[prec], c->stream));
    RET(ctl_read(c));
    // kernels the graph ran
    count_bodies(c, prec, s.h_ctl->iters);
    s.h_ctl->iters = 0;
    CK(cudaMemsetAsync(&s.d_ctl->iters, 0, sizeof(int), c->stream));
    return SBCI_OK;
  }
  // chunks of bodies (bodies after a halt do no work); one body per chunk
  // under kernel timing, so that no empty launch enters the statistics
  const int chunk = c->prof.on ? 1 : 8;
  for (;;) {
    for (int i = 0; i < chunk; ++i) RET(launch_body(c, prec, 0, true));
    RET(ctl_read(c));
    if (s.h_ctl->halt) return SBCI_OK;
  }
}

// (Re)starts the SB iteration of the current state from x, X with |x| = 1/sx.
sbci_status start_iteration(sbci_ctx *c, double sx, double E, int stage, int prec = -1) {
  Solver &s = c->s;
  CtlState &h = *s.h_ctl;
  h.halt = H_RUN;
  h.pending_check = 0;
  h.first = 1;
  h.sx_pending = 1.0;
  h.t = 0;
  h.E = E;
  h.stage = stage;
  h.n_sync = 0;
  h.prec = prec >= 0 ? prec : s.p.prec;
  h.zf = h.prec != SBCI_FP64 ? s.zf : nullptr;
  h.up.sx = sx;
  h.up.sy = 0.0;
  h.up.b = 0.0;
  h.up.c = 0.0;
  h.up.E = E;
  h.up.kinv = 1.0;
  h.up.Epre = shift_for(c, h.alpha, E);
  h.iters = 0;
  h.iter_cap = 4 * s.p.max_sigma + 256;
  h.zc = s.z[0];
  h.Zc = s.Z[0];
  h.zn = s.z[1];
  h.Zn = s.Z[1];
  return ctl_write(c);
}

sbci_status start_state(sbci_ctx *c, int alpha, double E0) {
  Solver &s = c->s;
  CtlState &h = *s.h_ctl;
  h.alpha = alpha;
  h.Ec0 = alpha > 0 ? s.Ec[0] : 0.0;
  h.pinv_ready = 0;
  if (alpha > 0 && s.pinv) {  // the shift is fixed for the state: precompute its preconditioner
    CK(launch_pinv(c->d_diag, h.Ec0, s.p.guard, c->ndet, s.pinv, c->stream));
    h.pinv_ready = 1;
  }
  h.n_sigma = h.n_sigma_fp64 = h.n_step = h.n_stage1 = 0;
  h.ctl_cycles = 0;
  for (int i = 0; i < 4; ++i) h.n_restart[i] = 0;
  s.verified = 0;
  return start_iteration(c, 1.0, E0, s.p.prec == SBCI_FP64 ? 1 : 0);
}

// X <- H x in FP64; returns x.x, x.X and X.X.  resync_issue queues it on the
// context stream, resync_complete waits for it.
sbci_status resync_issue(sbci_ctx *c) {
  Solver &s = c->s;
  RET(run_sigma(c, s.x, s.X, SBCI_FP64));
  return gen_dots_issue(c, {s.x, s.x, s.X}, {s.x, s.X, s.X});
}

sbci_status resync_complete(sbci_ctx *c, double *xx, double *xX, double *XX) {
  Solver &s = c->s;
  RET(fetch_complete(c, S_GEN0, S_GEN0 + 3));
  *xx = c->h_result[S_GEN0];
  *xX = c->h_result[S_GEN0 + 1];
  *XX = c->h_result[S_GEN0 + 2];
  s.h_ctl->n_sigma += 1;
  s.h_ctl->n_sigma_fp64 += 1;
  return SBCI_OK;
}

sbci_status resync(sbci_ctx *c, double *xx, double *xX, double *XX) {
  RET(resync_issue(c));
  return resync_complete(c, xx, xX, XX);
}

// Start of state alpha with a seeded full-symmetry component:
// x <- x/|x| + eta r/|r|, X <- X/|x| + eta (H r)/|r|, E0 = x.X / x.x.
// y and Y serve as scratch (the next start zeroes them).
sbci_status mix_noise(sbci_ctx *c, int alpha, double *E0) {
  Solver &s = c->s;
  CK(launch_splitmix(s.y, c->ndet, (unsigned long long)s.p.noise_seed, alpha, c->stream));
  if (s.p.sector) CK(launch_symmetrize(s.y, c->Na, c->stream));
  RET(run_sigma(c, s.y, s.Y, SBCI_FP64));
  RET(gen_dots(c, {s.y, s.x}, {s.y, s.x}));
  const double nr = std::sqrt(c->h_result[S_GEN0]), nx = std::sqrt(c->h_result[S_GEN0 + 1]);
  const double eta = s.p.start_noise;
  RET(lincomb(c, s.x, {s.x, s.y}, {1.0 / nx, eta / nr}));
  RET(lincomb(c, s.X, {s.X, s.Y}, {1.0 / nx, eta / nr}));
  RET(gen_dots(c, {s.x, s.x}, {s.x, s.X}));
  *E0 = c->h_result[S_GEN0 + 1] / c->h_result[S_GEN0];
  return SBCI_OK;
}

sbci_status finalize_state(sbci_ctx *c, bool converged, double E, double residual) {
  Solver &s = c->s;
  CtlState &h = *s.h_ctl;
  const int alpha = h.alpha;
  const double nx = std::sqrt(h.dots[S_NXX]);
  double *xca = s.xc + (size_t)alpha * c->ndet;
  RET(lincomb(c, xca, {s.x}, {1.0 / nx}));
  s.Ec.push_back(E);
  sbci_report &r = s.rep[alpha];
  r.energy = E + c->e_core;
  r.residual = residual;
  r.converged = converged ? 1 : 0;
  r.n_sigma = h.n_sigma;
  r.n_sigma_fp64 = h.n_sigma_fp64;
  r.n_step = h.n_step;
  for (int i = 0; i < 4; ++i) r.n_restart[i] = h.n_restart[i];
  r.ctl_cycles = h.ctl_cycles;
  {  // Eq. S136 health of the state from its trace (consecutive later steps)
    double lsum = 0.0;
    int n = 0;
    for (size_t i = 1; i < s.trace.size(); ++i) {
      const sbci_trace_record &p = s.trace[i - 1], &q = s.trace[i];
      if (q.state != alpha || p.state != alpha || q.t <= 0 || !std::isfinite(q.s136) || q.s136 == 0.0) continue;
      const double dE = p.energy - q.energy;
      if (std::fabs(dE) <= 1e-6) continue;
      lsum += std::log(std::fabs(dE / q.s136));
      ++n;
    }
    r.s136_ratio = n ? std::exp(lsum / n) : 0.0;
    r.s136_steps = n;
  }
  if (!converged) s.any_unconverged = 1;
  if (alpha + 1 >= s.k) {
    s.done = true;
    return SBCI_OK;
  }
  double E_next = h.E2;
  // next state's start: second Ritz vector of the last subspace (S1.4)
  const double *r3 = h.second;
  RET(lincomb(c, s.x, {s.x, s.y, h.zc}, {r3[0], r3[1], r3[2]}));
  RET(lincomb(c, s.X, {s.X, s.Y, h.Zc}, {r3[0], r3[1], r3[2]}));
  if (s.p.start_noise > 0.0) RET(mix_noise(c, alpha + 1, &E_next));
  // Eqs. S4-S7: project against every stored state, X via H x_c = E_c x_c
  std::vector<const double *> u, v;
  for (int i = 0; i <= alpha; ++i) {
    u.push_back(s.xc + (size_t)i * c->ndet);
    v.push_back(s.x);
  }
  RET(gen_dots(c, u, v));
  std::vector<double> ov(alpha + 1);
  for (int i = 0; i <= alpha; ++i) ov[i] = c->h_result[S_GEN0 + i];
  for (int i = 0; i <= alpha; ++i) {
    const double *xci = s.xc + (size_t)i * c->ndet;
    RET(lincomb(c, s.x, {s.x, xci}, {1.0, -ov[i]}));
    RET(lincomb(c, s.X, {s.X, xci}, {1.0, -s.Ec[i] * ov[i]}));
  }
  RET(gen_dots(c, {s.x}, {s.x}));
  const double nrm = std::sqrt(c->h_result[S_GEN0]);
  if (!(nrm > 0.0)) {
    set_error("excited-state start vector vanished after projection");
    return SBCI_ERR_NUMERIC;
  }
  RET(lincomb(c, s.x, {s.x}, {1.0 / nrm}));
  RET(lincomb(c, s.X, {s.X}, {1.0 / nrm}));
  return start_state(c, alpha + 1, E_next);
}

// The end of the low-precision stage or of a refinement window without a
// host round trip: the FP64 sigma X = H x, the dots x.x and x.X and the
// restart all go onto the context stream (the host mirror takes the fields it
// can know; the energy and scale stay on the device until the next read).
// SBCI_ASYNC_SWITCH=0 keeps the synchronous path.
bool async_switch() {
  const char *e = std::getenv("SBCI_ASYNC_SWITCH");
  return !(e && e[0] == '0');
}

sbci_status switch_async(sbci_ctx *c) {
  Solver &s = c->s;
  CtlState &h = *s.h_ctl;
  RET(run_sigma(c, s.x, s.X, SBCI_FP64));
  long long g = (c->ndet + 1023) / 1024;
  if (g > c->grid) g = c->grid;
  if (g < 1) g = 1;
  const double *u[2] = {s.x, s.x}, *v[2] = {s.x, s.X};
  RET(timed(c, K_DOTS, [&] { return launch_dots(u, v, 2, c->ndet, c->d_partials, (int)g, c->stream); }));
  RET(timed(c, K_RED, [&] { return launch_reduce(c->d_partials, (int)g, S_GEN0, S_GEN0 + 2, c->d_result, c->stream); }));
  RestartArgs r{};
  r.z0 = s.z[0];
  r.Z0 = s.Z[0];
  r.z1 = s.z[1];
  r.Z1 = s.Z[1];
  r.prec = s.p.prec;
  r.zf = s.p.prec != SBCI_FP64 ? s.zf : nullptr;
  r.iter_cap = 4 * s.p.max_sigma + 256;
  r.ground = h.alpha == 0 ? 1 : 0;
  r.Epre_fixed = h.alpha == 0 ? 0.0 : s.Ec[0];
  CK(launch_restart_resync(s.d_ctl, c->d_result + S_GEN0, r, c->stream));
  // the host mirror: everything but E, the scale and the update scalars
  h.halt = H_RUN;
  h.pending_check = 0;
  h.first = 1;
  h.sx_pending = 1.0;
  h.t = 0;
  h.stage = 1;
  h.n_sync = 0;
  h.prec = r.prec;
  h.zf = r.zf;
  h.iters = 0;
  h.iter_cap = r.iter_cap;
  h.zc = r.z0;
  h.Zc = r.Z0;
  h.zn = r.z1;
  h.Zn = r.Z1;
  h.n_sigma += 1;
  h.n_sigma_fp64 += 1;
  h.ntrace = 0;
  return SBCI_OK;
}

// Acts on a halted controller.
// A converged low-precision state is verified in FP64: its host work starts
// with a re-sync (exact X = H x).
bool halt_needs_resync(const sbci_ctx *c) {
  const Solver &s = c->s;
  const CtlState &h = *s.h_ctl;
  return h.halt == H_CONVERGED && !(s.p.prec == SBCI_FP64 || h.prec == SBCI_FP64);
}

// The FP64 residual check of a converged low-precision state from its
// re-sync (x.x, x.X, X.X): Rayleigh quotient and |H x - E x| / |x|; the state
// is stored, or continues in the FP64 stage.
sbci_status converged_after_resync(sbci_ctx *c, double xx, double xX, double XX) {
  Solver &s = c->s;
  const CtlState &h = *s.h_ctl;
  const double Erq = xX / xx;
  const double r = std::sqrt(std::max(XX / xx - Erq * Erq, 0.0));
  if (r < s.p.r0 && std::fabs(Erq - h.E) < s.p.eps0) return finalize_state(c, true, Erq, r);
  return start_iteration(c, 1.0 / std::sqrt(xx), Erq, 1);
}

sbci_status handle_halt(sbci_ctx *c) {
  Solver &s = c->s;
  CtlState &h = *s.h_ctl;
  switch (h.halt) {
    case H_RUN:
      return SBCI_OK;
    case H_NUMERIC:
      set_error("non-finite values in the SB step");
      return SBCI_ERR_NUMERIC;
    case H_SWITCH: {  // end of the low-precision stage or of a refinement window: exact H-image, stage 1
      if (async_switch()) return switch_async(c);
      double xx, xX, XX;
      RET(resync(c, &xx, &xX, &XX));
      return start_iteration(c, 1.0 / std::sqrt(xx), xX / xx, 1);
    }
    case H_CAP:
      if (h.prec != SBCI_FP64 && h.n_sigma < s.p.max_sigma) {
        // the low-precision refinement used its budget without reaching the
        // paper's thresholds: finish the state with FP64 sigma from the exact X
        double xx, xX, XX;
        RET(resync(c, &xx, &xX, &XX));
        sbci_trace_record r{};
        r.state = h.alpha;
        r.energy = xX / xx;
        r.event = 7;
        r.prec = SBCI_FP64;
        s.trace.push_back(r);
        return start_iteration(c, 1.0 / std::sqrt(xx), xX / xx, 1, SBCI_FP64);
      }
      s.h_ctl->halt = H_RUN;
      set_error("state reached its H-product cap without converging");
      RET(finalize_state(c, false, h.E, std::sqrt(h.dots[S_ZPZP])));
      return SBCI_ERR_NOT_CONVERGED;
    case H_CONVERGED: {
      if (s.p.prec == SBCI_FP64 || h.prec == SBCI_FP64)  // FP64 sigma throughout (or after a fallback)
        return finalize_state(c, true, h.E, std::sqrt(h.dots[S_ZPZP]));
      double xx, xX, XX;
      RET(resync(c, &xx, &xX, &XX));
      return converged_after_resync(c, xx, xX, XX);
    }
  }
  return SBCI_OK;
}

void free_solver(sbci_ctx *c) {
  Solver &s = c->s;
  for (int i = 0; i < 4; ++i) {
    if (s.gexec[i]) cudaGraphExecDestroy(s.gexec[i]);
    if (s.graph[i]) cudaGraphDestroy(s.graph[i]);
    s.gexec[i] = nullptr;
    s.graph[i] = nullptr;
  }
  if (s.x && c->stream) cudaStreamSynchronize(c->stream);  // its buffers go back to the pool
  double **ptrs[] = {&s.x, &s.X, &s.y, &s.Y, &s.w, &s.z[0], &s.z[1], &s.Z[0], &s.Z[1], &s.xc};
  for (double **p : ptrs) {
    if (*p) pool_free(*p);
    *p = nullptr;
  }
  if (s.zf) pool_free(s.zf);
  s.zf = nullptr;
  if (s.pinv) pool_free(s.pinv);
  s.pinv = nullptr;
  if (s.d_ctl) pool_free(s.d_ctl);
  if (s.h_ctl) pool_free_host(s.h_ctl);
  if (s.d_counters) pool_free(s.d_counters);
  s.d_ctl = nullptr;
  s.h_ctl = nullptr;
  s.d_counters = nullptr;
  s.active = false;
}

sbci_status alloc_solver(sbci_ctx *c, int k) {
  Solver &s = c->s;
  free_solver(c);
  double **ptrs[] = {&s.x, &s.X, &s.y, &s.Y, &s.w, &s.z[0], &s.z[1], &s.Z[0], &s.Z[1]};
  for (double **p : ptrs) {
    RET(dmalloc(p, (size_t)c->ndet));
    CK(cudaMemsetAsync(*p, 0, sizeof(double) * c->ndet, c->stream));
  }
  RET(dmalloc(&s.xc, (size_t)k * c->ndet));
  if (s.p.prec != SBCI_FP64) RET(dmalloc(&s.zf, (size_t)c->ndet));
  if (k > 1) RET(dmalloc(&s.pinv, (size_t)c->ndet));
  CK(cudaMemsetAsync(s.xc, 0, sizeof(double) * (size_t)k * c->ndet, c->stream));
  CK(pool_malloc((void **)&s.d_ctl, sizeof(CtlState)));
  CK(cudaMemsetAsync(s.d_ctl, 0, sizeof(CtlState), c->stream));
  CK(pool_malloc_host((void **)&s.h_ctl, sizeof(CtlState)));
  std::memset(s.h_ctl, 0, sizeof(CtlState));
  s.h_ctl->trace_ptr = s.d_ctl->trace;  // device address of the ring (no dereference)
  CK(pool_malloc((void **)&s.d_counters, 4 * sizeof(unsigned int)));
  CK(cudaMemsetAsync(s.d_counters, 0, 4 * sizeof(unsigned int), c->stream));
  return SBCI_OK;
}
// S1.1: lowest-diagonal determinants -> GS -> H in the subspace -> x_0, X_0, E_0.
sbci_status initial_guess(sbci_ctx *c, int k, double *E0) {
  Solver &s = c->s;
  const int n_init = s.p.n_init > 0 ? s.p.n_init : std::max(k, 2);
  std::vector<double> D(c->ndet);
  CK(cudaMemcpyAsync(D.data(), c->d_diag, sizeof(double) * c->ndet, cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  // n_init smallest (D_I, I) with a bounded max-heap
  typedef std::pair<double, long long> Key;
  std::priority_queue<Key> heap;
  for (long long i = 0; i < c->ndet; ++i) {
    Key kk(D[i], i);
    if ((int)heap.size() < n_init) heap.push(kk);
    else if (kk < heap.top()) {
      heap.pop();
      heap.push(kk);
    }
  }
  std::vector<Key> sel;
  while (!heap.empty()) {
    sel.push_back(heap.top());
    heap.pop();
  }
  std::sort(sel.begin(), sel.end());
  // sparse basis vectors with Gram-Schmidt (S1.1)
  typedef std::map<long long, double> Sparse;
  std::vector<Sparse> basis;
  for (const Key &kk : sel) {
    Sparse e;
    const long long I = kk.second;
    if (s.p.sector) {
      const long long ia = I / c->Nb, ib = I % c->Nb, T = ib * c->Nb + ia;
      e[I] += 0.5;
      e[T] += 0.5;
    } else {
      e[I] = 1.0;
    }
    for (const Sparse &b : basis) {
      double ov = 0.0;
      for (auto &kv : e) {
        auto it = b.find(kv.first);
        if (it != b.end()) ov += it->second * kv.second;
      }
      for (auto &kv : b) e[kv.first] -= ov * kv.second;
    }
    double nrm = 0.0;
    for (auto &kv : e) nrm += kv.second * kv.second;
    nrm = std::sqrt(nrm);
    if (nrm < s.p.gs_tol) continue;
    for (auto &kv : e) kv.second /= nrm;
    basis.push_back(e);
  }
  const int m = (int)basis.size();
  if (m == 0 || m > 8) {
    set_error("initial guess: unsupported subspace size");
    return SBCI_ERR_INVALID;
  }
  // X_{-1}^i = H x_{-1}^i (Eq. S1); X buffers: use xc storage rows as scratch when k >= m,
  // otherwise a temporary allocation.
  double *tmp = nullptr;
  RET(dmalloc(&tmp, (size_t)m * c->ndet));
  // the sparse vectors' (index, value) pairs, and the entries of the H-images
  // that the subspace matrix needs, move in one copy each (one small device
  // buffer: the pairs of every basis vector, then the entry offsets and values)
  std::vector<double> pairs;
  std::vector<size_t> pofs(m + 1, 0);
  size_t nA = 0;
  for (int i = 0; i < m; ++i) {
    for (auto &kv : basis[i]) {
      pairs.push_back((double)kv.first);
      pairs.push_back(kv.second);
    }
    pofs[i + 1] = pairs.size() / 2;
    nA += (size_t)m * basis[i].size();
  }
  double *d_aux = nullptr;
  RET(dmalloc(&d_aux, pairs.size() + 2 * nA));
  CK(cudaMemcpyAsync(d_aux, pairs.data(), sizeof(double) * pairs.size(), cudaMemcpyHostToDevice, c->stream));
  std::vector<double> A(m * m);
  // FP64, or the stage precision with init_stage (the start is then as exact
  // as the stage's own steps; the first re-sync makes X an FP64 H x)
  const int ip = s.p.init_stage ? s.p.prec : SBCI_FP64;
  for (int i = 0; i < m; ++i) {
    CK(cudaMemsetAsync(s.w, 0, sizeof(double) * c->ndet, c->stream));
    CK(launch_sparse_set(s.w, d_aux + 2 * pofs[i], (int)(pofs[i + 1] - pofs[i]), c->stream));
    RET(run_sigma(c, s.w, tmp + (size_t)i * c->ndet, ip));
  }
  {  // A[i][j] = sum over the entries (I, v) of basis i of v (H b_j)[I], in that order
    std::vector<double> offs;
    offs.reserve(nA);
    for (int i = 0; i < m; ++i)
      for (int j = 0; j < m; ++j)
        for (auto &kv : basis[i]) offs.push_back((double)((size_t)j * c->ndet + (size_t)kv.first));
    double *d_offs = d_aux + pairs.size(), *d_vals = d_offs + nA;
    std::vector<double> vals(nA);
    CK(cudaMemcpyAsync(d_offs, offs.data(), sizeof(double) * nA, cudaMemcpyHostToDevice, c->stream));
    CK(launch_gather_at(tmp, d_offs, (int)nA, d_vals, c->stream));
    CK(cudaMemcpyAsync(vals.data(), d_vals, sizeof(double) * nA, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    size_t q = 0;
    for (int i = 0; i < m; ++i)
      for (int j = 0; j < m; ++j) {
        double a = 0.0;
        for (auto &kv : basis[i]) a += kv.second * vals[q++];
        A[i * m + j] = a;
      }
  }
  for (int i = 0; i < m; ++i)
    for (int j = 0; j < i; ++j) A[i * m + j] = A[j * m + i] = 0.5 * (A[i * m + j] + A[j * m + i]);
  std::vector<double> w(m), U(m * m);
  jacobi_eigh(m, A.data(), w.data(), U.data());
  // x_0 = sum_i U[i,0] x_{-1}^i (Eq. S2), X_0 = sum_i U[i,0] X_{-1}^i (Eq. S3)
  Sparse x0;
  for (int i = 0; i < m; ++i)
    for (auto &kv : basis[i]) x0[kv.first] += U[i * m] * kv.second;
  CK(cudaMemsetAsync(s.x, 0, sizeof(double) * c->ndet, c->stream));
  {
    std::vector<double> xp;
    for (auto &kv : x0) {
      xp.push_back((double)kv.first);
      xp.push_back(kv.second);
    }
    // (the pairs of the basis are consumed: the stream has run past their scatters)
    CK(cudaMemcpyAsync(d_aux, xp.data(), sizeof(double) * xp.size(), cudaMemcpyHostToDevice, c->stream));
    CK(launch_sparse_set(s.x, d_aux, (int)(xp.size() / 2), c->stream));
  }
  std::vector<const double *> in;
  std::vector<double> co;
  for (int i = 0; i < m; ++i) {
    in.push_back(tmp + (size_t)i * c->ndet);
    co.push_back(U[i * m]);
  }
  RET(lincomb(c, s.X, in, co));
  CK(cudaStreamSynchronize(c->stream));
  CK(pool_free(tmp));
  CK(pool_free(d_aux));
  *E0 = w[0];
  return SBCI_OK;
}

sbci_status init_from_vector(sbci_ctx *c, const double *c0, double *E0) {
  Solver &s = c->s;
  std::vector<double> v(c0, c0 + c->ndet);
  RET(check_finite(v.data(), v.size(), "c0"));
  if (s.p.sector) {
    for (int a = 0; a < c->Na; ++a)
      for (int b = a + 1; b < c->Nb; ++b) {
        const double m = 0.5 * (v[(size_t)a * c->Nb + b] + v[(size_t)b * c->Nb + a]);
        v[(size_t)a * c->Nb + b] = m;
        v[(size_t)b * c->Nb + a] = m;
      }
  }
  CK(cudaMemcpyAsync(s.x, v.data(), sizeof(double) * c->ndet, cudaMemcpyHostToDevice, c->stream));
  RET(gen_dots(c, {s.x}, {s.x}));
  const double nrm = std::sqrt(c->h_result[S_GEN0]);
  if (!(nrm > 0.0)) {
    set_error("c0 is zero");
    return SBCI_ERR_INVALID;
  }
  RET(lincomb(c, s.x, {s.x}, {1.0 / nrm}));
  RET(run_sigma(c, s.x, s.X, SBCI_FP64));
  RET(gen_dots(c, {s.x}, {s.X}));
  *E0 = c->h_result[S_GEN0];
  return SBCI_OK;
}

// ---------------------------------------------------------------------------
// Block Davidson-Liu (Davidson 1975; Liu 1978) on the same FP64 sigma: the
// method the paper compares SBCI with (Introduction; Materials and Methods:
// PySCF's Davidson with the preconditioner (D - E^0 I)^-1).  The paper does
// not state its schedule; this one is fixed as follows:
//  D1 start: determinants by ascending (D_I, I), symmetrised in the sector,
//     Gram-Schmidt orthonormalised (dropped below gs_tol), until
//     max(k, n_init or 2) vectors; one H-product each;
//  D2 subspace matrix (T + T^T)/2, T = V^T (H V); Ritz values theta_a and
//     residuals r_a = (H V) s_a - theta_a V s_a;
//  D3 converged when |theta_a - previous theta_a| < eps0 and |r_a| < r0 for
//     every a (the thresholds of Eq. S61);
//  D4 collapse onto the k Ritz vectors (and their H-images) when the
//     corrections would overflow max_space;
//  D5 per unconverged a: t = r_a / guarded(D - theta_a), symmetrised in the
//     sector, projected twice against V, dropped if |t|^2 < gs_tol |t_0|^2,
//     normalised, appended, one H-product;
//  D6 an iteration that adds no vector (all dropped, or the H-product cap
//     max_sigma * k reached) ends the solve, converged if every |r_a| < r0.
// The subspace lives in a pool of slot buffers (vector, H-image); the k
// residuals take free slots and become the appended corrections in place.

// Block dot products and linear combinations of whole vectors for the
// host-driven solvers (Davidson-Liu, SBCI2): reduction scratch and a pinned
// result buffer.
struct VecScratch {
  sbci_ctx *c = nullptr;
  double *partials = nullptr, *d_res = nullptr, *h_res = nullptr;
  int grid = 1;
  ~VecScratch() {
    if (c && c->stream) cudaStreamSynchronize(c->stream);  // the buffers go back to the pool
    if (partials) pool_free(partials);
    if (d_res) pool_free(d_res);
    if (h_res) pool_free_host(h_res);
  }
};

sbci_status scratch_init(VecScratch &d, sbci_ctx *c) {
  d.c = c;
  d.grid = dav_dots_grid(c->ndet, c->nsm);
  RET(dmalloc(&d.partials, (size_t)kDavMaxPairs * d.grid));
  RET(dmalloc(&d.d_res, (size_t)kDavMaxPairs));
  CK(pool_malloc_host((void **)&d.h_res, sizeof(double) * kDavMaxPairs));
  return SBCI_OK;
}

struct DavSolve : VecScratch {
  std::vector<double *> vb, ab;  // slot buffers: subspace vector, its H-image
  std::vector<int> V;            // the subspace, as slots in order
  std::vector<int> free_slots;
  ~DavSolve() {
    if (c && c->stream) cudaStreamSynchronize(c->stream);  // the buffers go back to the pool
    for (double *p : vb)
      if (p) pool_free(p);
    for (double *p : ab)
      if (p) pool_free(p);
  }
  int take() {
    const int sl = free_slots.back();
    free_slots.pop_back();
    return sl;
  }
};

sbci_status dav_dots(VecScratch &d, const std::vector<const double *> &u, const std::vector<const double *> &v,
                     std::vector<double> &out) {
  sbci_ctx *c = d.c;
  out.assign(u.size(), 0.0);
  for (size_t p0 = 0; p0 < u.size(); p0 += kDavMaxPairs) {
    const int np = (int)std::min<size_t>(kDavMaxPairs, u.size() - p0);
    RET(timed(c, K_DAVD, [&] {
      return launch_dav_dots(u.data() + p0, v.data() + p0, np, c->ndet, d.partials, d.grid, c->stream);
    }));
    RET(timed(c, K_RED, [&] { return launch_reduce(d.partials, d.grid, 0, np, d.d_res, c->stream); }));
    CK(cudaMemcpyAsync(d.h_res, d.d_res, sizeof(double) * np, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    for (int p = 0; p < np; ++p) {
      if (!std::isfinite(d.h_res[p])) {
        set_error("non-finite dot product in a device reduction (Davidson)");
        return SBCI_ERR_NUMERIC;
      }
      out[p0 + p] = d.h_res[p];
    }
  }
  return SBCI_OK;
}

// out_j = sum_q coef[q * nout + j] in_q (an output may be one of the inputs)
sbci_status dav_combine(VecScratch &d, const std::vector<double *> &out, const std::vector<const double *> &in,
                        const std::vector<double> &coef) {
  sbci_ctx *c = d.c;
  return timed(c, K_DAVC, [&] {
    return launch_dav_combine(out.data(), (int)out.size(), in.data(), (int)in.size(), coef.data(), c->ndet,
                              c->nsm, c->stream);
  });
}

// T[i][j] = V_i . (H V)_j for all i, j < m (row stride kDavMaxSpace)
sbci_status dav_full_T(DavSolve &d, std::vector<double> &T) {
  const int m = (int)d.V.size();
  std::vector<const double *> u, v;
  for (int i = 0; i < m; ++i)
    for (int j = 0; j < m; ++j) {
      u.push_back(d.vb[d.V[i]]);
      v.push_back(d.ab[d.V[j]]);
    }
  std::vector<double> r;
  RET(dav_dots(d, u, v, r));
  for (int i = 0; i < m; ++i)
    for (int j = 0; j < m; ++j) T[(size_t)i * kDavMaxSpace + j] = r[(size_t)i * m + j];
  return SBCI_OK;
}

typedef std::map<long long, double> Sparse;

// Start vectors of the host-driven solvers (Davidson D1, SBCI2 Q1):
// determinants by ascending (D_I, I), symmetrised in the sector (c = c^T),
// Gram-Schmidt orthonormalised (dropped below gs_tol), until n_v vectors hold
// or the space is exhausted.
sbci_status lowest_diagonal_basis(sbci_ctx *c, int n_v, const sbci_params &p, std::vector<Sparse> &basis) {
  const long long N = c->ndet;
  std::vector<double> D(N);
  CK(cudaMemcpyAsync(D.data(), c->d_diag, sizeof(double) * N, cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  typedef std::pair<double, long long> Key;
  long long ncand = std::min<long long>(N, 2LL * n_v + 2);
  for (;;) {
    std::priority_queue<Key> heap;  // the ncand smallest (D_I, I)
    for (long long i = 0; i < N; ++i) {
      const Key kk(D[i], i);
      if ((long long)heap.size() < ncand) heap.push(kk);
      else if (kk < heap.top()) {
        heap.pop();
        heap.push(kk);
      }
    }
    std::vector<Key> sel;
    while (!heap.empty()) {
      sel.push_back(heap.top());
      heap.pop();
    }
    std::sort(sel.begin(), sel.end());
    basis.clear();
    for (const Key &kk : sel) {
      if ((int)basis.size() >= n_v) break;
      Sparse e;
      const long long I = kk.second;
      if (p.sector) {
        const long long ia = I / c->Nb, ib = I % c->Nb;
        e[I] += 0.5;
        e[ib * c->Nb + ia] += 0.5;
      } else {
        e[I] = 1.0;
      }
      for (const Sparse &b : basis) {
        double ov = 0.0;
        for (auto &kv : e) {
          auto it = b.find(kv.first);
          if (it != b.end()) ov += it->second * kv.second;
        }
        for (auto &kv : b) e[kv.first] -= ov * kv.second;
      }
      double nrm = 0.0;
      for (auto &kv : e) nrm += kv.second * kv.second;
      nrm = std::sqrt(nrm);
      if (nrm < p.gs_tol) continue;
      for (auto &kv : e) kv.second /= nrm;
      basis.push_back(e);
    }
    if ((int)basis.size() >= n_v || ncand >= N) break;
    ncand = std::min(N, 2 * ncand);
  }
  return SBCI_OK;
}

// dense copy of a sparse vector into a device buffer
sbci_status upload_sparse(sbci_ctx *c, const Sparse &b, double *dst) {
  CK(cudaMemsetAsync(dst, 0, sizeof(double) * c->ndet, c->stream));
  for (auto &kv : b)
    CK(cudaMemcpyAsync(dst + kv.first, &kv.second, sizeof(double), cudaMemcpyHostToDevice, c->stream));
  return SBCI_OK;
}

sbci_status davidson_run(sbci_ctx *c, int k, const sbci_params &p, int max_space, double *energies, double *vecs,
                         sbci_report *rep, long long *vector_bytes) {
  const long long N = c->ndet;
  // D1: start vectors
  const int n_v = std::max(k, p.n_init > 0 ? p.n_init : 2);
  std::vector<Sparse> basis;
  RET(lowest_diagonal_basis(c, n_v, p, basis));
  if ((int)basis.size() < k) {
    set_error("sbci_davidson: the space holds fewer than k start vectors");
    return SBCI_ERR_INVALID;
  }
  // slot pool: the subspace plus the k residuals / corrections
  DavSolve d;
  RET(scratch_init(d, c));
  const int cap = max_space + k;
  d.vb.assign(cap, nullptr);
  d.ab.assign(cap, nullptr);
  for (int sl = 0; sl < cap; ++sl) {
    RET(dmalloc(&d.vb[sl], (size_t)N));
    RET(dmalloc(&d.ab[sl], (size_t)N));
  }
  for (int sl = cap - 1; sl >= 0; --sl) d.free_slots.push_back(sl);
  if (vector_bytes) *vector_bytes = 2LL * cap * N * (long long)sizeof(double);
  for (const Sparse &b : basis) {
    const int sl = d.take();
    RET(upload_sparse(c, b, d.vb[sl]));
    d.V.push_back(sl);
  }
  const long long max_sigma = (long long)p.max_sigma * k;
  long long n_sigma = 0;
  for (int sl : d.V) {
    RET(run_sigma(c, d.vb[sl], d.ab[sl], SBCI_FP64));
    ++n_sigma;
  }
  std::vector<double> T((size_t)kDavMaxSpace * kDavMaxSpace, 0.0);
  RET(dav_full_T(d, T));
  std::vector<double> theta(k), theta_prev(k), rn(k), S, r;
  std::vector<int> R(k, -1);
  bool have_prev = false, converged = false;
  int n_iter = 0, n_collapse = 0;
  for (;;) {
    ++n_iter;
    int m = (int)d.V.size();
    // D2: Ritz pairs of the symmetrised subspace matrix
    std::vector<double> A((size_t)m * m), w(m), U((size_t)m * m);
    for (int i = 0; i < m; ++i)
      for (int j = 0; j < m; ++j)
        A[(size_t)i * m + j] = 0.5 * (T[(size_t)i * kDavMaxSpace + j] + T[(size_t)j * kDavMaxSpace + i]);
    jacobi_eigh(m, A.data(), w.data(), U.data());
    S.assign((size_t)m * k, 0.0);  // S[i * k + a]
    for (int a = 0; a < k; ++a) {
      theta[a] = w[a];
      for (int i = 0; i < m; ++i) S[(size_t)i * k + a] = U[(size_t)i * m + a];
    }
    // residuals r_a = (H V) s_a - theta_a V s_a, in free slots
    std::vector<double *> Rout(k);
    for (int a = 0; a < k; ++a) {
      R[a] = d.take();
      Rout[a] = d.vb[R[a]];
    }
    {
      std::vector<const double *> in;
      for (int i = 0; i < m; ++i) in.push_back(d.ab[d.V[i]]);
      RET(dav_combine(d, Rout, in, S));
      std::vector<const double *> in2;
      std::vector<double> co((size_t)(k + m) * k, 0.0);
      for (int a = 0; a < k; ++a) {
        in2.push_back(Rout[a]);
        co[(size_t)a * k + a] = 1.0;
      }
      for (int i = 0; i < m; ++i) {
        in2.push_back(d.vb[d.V[i]]);
        for (int a = 0; a < k; ++a) co[(size_t)(k + i) * k + a] = -theta[a] * S[(size_t)i * k + a];
      }
      RET(dav_combine(d, Rout, in2, co));
      std::vector<const double *> u(Rout.begin(), Rout.end());
      RET(dav_dots(d, u, u, r));
      for (int a = 0; a < k; ++a) rn[a] = std::sqrt(r[a]);
    }
    // D3
    std::vector<int> unconv;
    for (int a = 0; a < k; ++a) {
      const bool ok = have_prev && std::fabs(theta[a] - theta_prev[a]) < p.eps0 && rn[a] < p.r0;
      if (!ok) unconv.push_back(a);
    }
    if (unconv.empty()) {
      converged = true;
      break;
    }
    theta_prev = theta;
    have_prev = true;
    // D4: collapse in place onto the k Ritz vectors
    if (m + (int)unconv.size() > max_space) {
      std::vector<double *> outv, outa;
      std::vector<const double *> inv, ina;
      for (int a = 0; a < k; ++a) {
        outv.push_back(d.vb[d.V[a]]);
        outa.push_back(d.ab[d.V[a]]);
      }
      for (int i = 0; i < m; ++i) {
        inv.push_back(d.vb[d.V[i]]);
        ina.push_back(d.ab[d.V[i]]);
      }
      RET(dav_combine(d, outv, inv, S));
      RET(dav_combine(d, outa, ina, S));
      for (int i = k; i < m; ++i) d.free_slots.push_back(d.V[i]);
      d.V.resize(k);
      m = k;
      S.assign((size_t)k * k, 0.0);
      for (int a = 0; a < k; ++a) S[(size_t)a * k + a] = 1.0;
      RET(dav_full_T(d, T));
      ++n_collapse;
    }
    // D5 in block form (the same vectors as one correction at a time in exact
    // arithmetic): all corrections, projected twice against V, then
    // orthonormalised among themselves in order (drop rule of D5) by classical
    // Gram-Schmidt on their Gram matrix, twice; one dot-product batch and one
    // combination per pass instead of a host round trip per correction
    int added = 0;
    std::vector<int> ca;  // states whose correction is formed
    for (int a : unconv)
      if (n_sigma + (long long)ca.size() < max_sigma) ca.push_back(a);
    const int nu = (int)ca.size();
    std::vector<double *> tv(nu);
    for (int j = 0; j < nu; ++j) {
      tv[j] = d.vb[R[ca[j]]];
      double *t = tv[j];
      const double sh = theta[ca[j]];
      RET(timed(c, K_DAVP, [&] { return launch_dav_precond(t, t, c->d_diag, sh, p.guard, N, c->nsm, c->stream); }));
      if (p.sector) RET(timed(c, K_DAVP, [&] { return launch_symmetrize(t, c->Na, c->stream); }));
    }
    std::vector<double> n0(nu, 0.0);
    if (nu > 0) {
      for (int pass = 0; pass < 2; ++pass) {  // T <- T - V (V^T T)
        std::vector<const double *> u, v;
        for (int j = 0; j < nu; ++j)
          for (int i = 0; i < m; ++i) {
            u.push_back(d.vb[d.V[i]]);
            v.push_back(tv[j]);
          }
        if (pass == 0)
          for (int j = 0; j < nu; ++j) {
            u.push_back(tv[j]);
            v.push_back(tv[j]);
          }
        RET(dav_dots(d, u, v, r));
        if (pass == 0)
          for (int j = 0; j < nu; ++j) n0[j] = r[(size_t)nu * m + j];
        std::vector<const double *> in(tv.begin(), tv.end());
        for (int i = 0; i < m; ++i) in.push_back(d.vb[d.V[i]]);
        std::vector<double> co((size_t)(nu + m) * nu, 0.0);
        for (int j = 0; j < nu; ++j) {
          co[(size_t)j * nu + j] = 1.0;
          for (int i = 0; i < m; ++i) co[(size_t)(nu + i) * nu + j] = -r[(size_t)j * m + i];
        }
        RET(dav_combine(d, tv, in, co));
      }
    }
    // among themselves: coefficients Q = T C (C upper triangular over the
    // kept columns), from the Gram matrix G = T^T T, twice
    std::vector<int> keep;
    for (int j = 0; j < nu; ++j) keep.push_back(j);
    for (int pass = 0; pass < 2 && !keep.empty(); ++pass) {
      const int nk = (int)keep.size();
      std::vector<const double *> u, v;
      for (int a2 = 0; a2 < nk; ++a2)
        for (int b2 = 0; b2 <= a2; ++b2) {
          u.push_back(tv[keep[a2]]);
          v.push_back(tv[keep[b2]]);
        }
      RET(dav_dots(d, u, v, r));
      std::vector<double> G((size_t)nk * nk);
      size_t qi = 0;
      for (int a2 = 0; a2 < nk; ++a2)
        for (int b2 = 0; b2 <= a2; ++b2, ++qi) G[(size_t)a2 * nk + b2] = G[(size_t)b2 * nk + a2] = r[qi];
      std::vector<std::vector<double>> Cq;  // coefficient vectors (length nk) of the kept q's
      std::vector<int> kept_next;
      for (int a2 = 0; a2 < nk; ++a2) {
        std::vector<double> uvec(nk, 0.0);
        uvec[a2] = 1.0;
        std::vector<double> proj(Cq.size());
        for (size_t b2 = 0; b2 < Cq.size(); ++b2) {  // q_b . t_a from the original t_a
          double acc = 0.0;
          for (int c2 = 0; c2 < nk; ++c2) acc += Cq[b2][c2] * G[(size_t)c2 * nk + a2];
          proj[b2] = acc;
        }
        for (size_t b2 = 0; b2 < Cq.size(); ++b2)
          for (int c2 = 0; c2 < nk; ++c2) uvec[c2] -= proj[b2] * Cq[b2][c2];
        double nrm2 = 0.0;
        for (int c2 = 0; c2 < nk; ++c2)
          for (int e2 = 0; e2 < nk; ++e2) nrm2 += uvec[c2] * G[(size_t)c2 * nk + e2] * uvec[e2];
        const double ref = pass == 0 ? n0[keep[a2]] : 1.0;
        if (!(nrm2 > 0.0 && nrm2 >= p.gs_tol * ref)) continue;
        const double f = 1.0 / std::sqrt(nrm2);
        for (double &x : uvec) x *= f;
        Cq.push_back(uvec);
        kept_next.push_back(keep[a2]);
      }
      // q's into the slots of the kept corrections, in place
      const int nq = (int)Cq.size();
      if (nq > 0) {
        std::vector<double *> out;
        std::vector<const double *> in;
        for (int a2 = 0; a2 < nq; ++a2) out.push_back(tv[kept_next[a2]]);
        for (int c2 = 0; c2 < nk; ++c2) in.push_back(tv[keep[c2]]);
        std::vector<double> co((size_t)nk * nq, 0.0);
        for (int a2 = 0; a2 < nq; ++a2)
          for (int c2 = 0; c2 < nk; ++c2) co[(size_t)c2 * nq + a2] = Cq[a2][c2];
        RET(dav_combine(d, out, in, co));
      }
      keep = kept_next;
    }
    // the kept corrections join V with their H-images
    const int m_old = m;
    for (int j : keep) {
      const int ts = R[ca[j]];
      RET(run_sigma(c, d.vb[ts], d.ab[ts], SBCI_FP64));
      ++n_sigma;
      d.V.push_back(ts);
      R[ca[j]] = -1;
      ++m;
      ++added;
    }
    if (added > 0) {  // new rows and columns of T
      std::vector<const double *> u, v;
      for (int j = m_old; j < m; ++j)
        for (int i = 0; i < m; ++i) {
          u.push_back(d.vb[d.V[i]]);
          v.push_back(d.ab[d.V[j]]);
        }
      for (int j = m_old; j < m; ++j)
        for (int i = 0; i < m_old; ++i) {
          u.push_back(d.vb[d.V[j]]);
          v.push_back(d.ab[d.V[i]]);
        }
      RET(dav_dots(d, u, v, r));
      size_t qi = 0;
      for (int j = m_old; j < m; ++j)
        for (int i = 0; i < m; ++i) T[(size_t)i * kDavMaxSpace + j] = r[qi++];
      for (int j = m_old; j < m; ++j)
        for (int i = 0; i < m_old; ++i) T[(size_t)j * kDavMaxSpace + i] = r[qi++];
    }
    for (int a = 0; a < k; ++a)
      if (R[a] >= 0) {
        d.free_slots.push_back(R[a]);
        R[a] = -1;
      }
    if (added == 0) {  // D6
      converged = true;
      for (int a = 0; a < k; ++a) converged = converged && rn[a] < p.r0;
      break;
    }
  }
  // results: Ritz vectors V s_a (the residual slots are no longer needed)
  for (int a = 0; a < k; ++a)
    if (R[a] >= 0) {
      d.free_slots.push_back(R[a]);
      R[a] = -1;
    }
  if (vecs) {
    const int m = (int)d.V.size();
    std::vector<double *> out;
    std::vector<const double *> in;
    for (int a = 0; a < k; ++a) out.push_back(d.vb[d.take()]);
    for (int i = 0; i < m; ++i) in.push_back(d.vb[d.V[i]]);
    RET(dav_combine(d, out, in, S));
    for (int a = 0; a < k; ++a)
      CK(cudaMemcpyAsync(vecs + (size_t)a * N, out[a], sizeof(double) * N, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
  }
  for (int a = 0; a < k; ++a) {
    energies[a] = theta[a] + c->e_core;
    if (rep) {
      sbci_report &o = rep[a];
      o = sbci_report{};
      o.energy = energies[a];
      o.residual = rn[a];
      o.converged = converged ? 1 : 0;
      o.n_sigma = (int)n_sigma;
      o.n_sigma_fp64 = (int)n_sigma;
      o.n_step = n_iter;
      o.n_restart[0] = n_collapse;
    }
  }
  if (!converged) {
    set_error("sbci_davidson: stopped before every state converged");
    return SBCI_ERR_NOT_CONVERGED;
  }
  return SBCI_OK;
}

// Everything a solve needs before its first start vector: parameters,
// per-solve vectors, the controller's thresholds.
sbci_status begin_common(sbci_ctx *c, int k, const sbci_params *params, const char *who) {
  if (!c || k < 1 || k > kMaxStates) {
    set_error(std::string(who) + ": need a context and 1 <= k <= 8");
    return SBCI_ERR_INVALID;
  }
  Solver &s = c->s;
  if (params) s.p = *params;
  else sbci_params_init(&s.p);
  if (s.p.sector && c->ne_a != c->ne_b) {
    set_error("sector = 1 needs nalpha == nbeta");
    return SBCI_ERR_INVALID;
  }
  if (s.p.init_stage != 0 && s.p.init_stage != 1) {
    set_error("init_stage must be 0 or 1");
    return SBCI_ERR_INVALID;
  }
  RET(check_prec(c, s.p.prec));
  if ((long long)k > c->ndet) {
    set_error(std::string(who) + ": more states than determinants");
    return SBCI_ERR_INVALID;
  }
  RET(alloc_solver(c, k));
  RET(ensure_G(c, SBCI_FP64));
  if (s.p.prec != SBCI_FP64) RET(ensure_G(c, s.p.prec));
  s.k = k;
  s.done = false;
  s.Ec.clear();
  s.trace.clear();
  s.rep.assign(k, sbci_report{});
  s.any_unconverged = 0;
  s.active = true;
  CtlState &h = *s.h_ctl;
  h.p.eps0 = s.p.eps0;
  h.p.r0 = s.p.r0;
  h.p.b_th = s.p.b_th;
  h.p.eps1 = s.p.eps1;
  h.p.x_th1 = s.p.x_th1;
  h.p.x_th2 = s.p.x_th2;
  h.p.r1 = s.p.r1;
  h.p.guard = s.p.guard;
  h.p.gs_tol = s.p.gs_tol;
  h.p.mixed_eps = s.p.mixed_eps;
  h.p.mixed_r = s.p.mixed_r;
  h.p.max_cycle = s.p.max_cycle;
  h.p.max_sigma = s.p.max_sigma;
  h.p.refine_max_sigma = s.p.refine_max_sigma;
  h.p.user_prec = s.p.prec;
  return SBCI_OK;
}

// ---------------------------------------------------------------------------
// SBCI2 (Algorithm 2, Sections S2.1-S2.5): the pair (alpha, alpha+1) advances
// together, the lower state is stored when it converges, and the highest
// state runs SBCI1 on the device controller (Fig. 1B).  Pair steps are
// host-driven: two FP64 H-products, one batch of dot products (overlap S and
// T = B^T [H B] of the step's basis), the 6x6 canonical orthogonalisation and
// eigen-problem on the host, and one in-place combination kernel for x, X, y,
// Y and the new residuals.  Readings Q1-Q10 (as the oracle):
//  Q1 start vectors from max(k, n_init or 2) lowest-diagonal vectors (S74-S76);
//  Q2 a later pair's upper start: projected against the stored states and the
//     new lower vector, normalised, E_0 its Rayleigh quotient;
//  Q3 preconditioner shift E_t of state 0 in the ground pair, E_c^0 after;
//  Q4 subspace matrix (T + T^T)/2;  Q5 overlap eigenvalues below 1e-14 dropped;
//  Q6 undefined later-step coefficients: first-step path from the same x, z;
//  Q7 restart: x/|x|, X/|x|, E_0 = E_{t+1}, y = 0, first-step path;
//  Q8 max_sigma H-products per lower state;
//  Q9 x_{t+1} = k v, X_{t+1} = k [H-images] V' (no cancellation of S124);
//  Q10 the upper start of a later pair gets X_0 by one H-product.

struct DevBuffers {
  std::vector<double *> v;
  cudaStream_t stream = nullptr;
  ~DevBuffers() {
    if (stream) cudaStreamSynchronize(stream);  // the buffers go back to the pool
    for (double *p : v)
      if (p) pool_free(p);
  }
  sbci_status get(sbci_ctx *c, double **out) {
    stream = c->stream;
    double *p = nullptr;
    RET(dmalloc(&p, (size_t)c->ndet));
    v.push_back(p);
    *out = p;
    return SBCI_OK;
  }
};

struct PairCoef {
  bool first;                 // first-step path (Eq. S93): basis x^a, x^b, z^a, z^b
  int nb;                     // basis vectors (4 or 6)
  double Vp[6][2];            // V' = P V, columns of the two lowest Ritz vectors
  double w[2];                // E_{t+1}^a, E_{t+1}^b
  double A[2][2], B[2][2], C[2][2], k[2];
};

// Canonical orthogonalisation, subspace eigen-problem and coefficients of one
// pair step.  S6 and T6 are the 6x6 overlap and T of (x^a, x^b, y^a, y^b, z^a,
// z^b) (rows and columns of y unused on the first path).  Returns false if the
// step is undefined on the requested path.
bool pair_step(const double *S6, const double *T6, bool first, PairCoef *pc) {
  static const int kFirst[4] = {0, 1, 4, 5}, kLater[6] = {0, 1, 2, 3, 4, 5};
  const int nb = first ? 4 : 6;
  const int *ix = first ? kFirst : kLater;
  double S[36], Hs[36], s[6], U[36];
  for (int i = 0; i < nb; ++i)
    for (int j = 0; j < nb; ++j) {
      S[i * nb + j] = S6[ix[i] * 6 + ix[j]];
      Hs[i * nb + j] = 0.5 * (T6[ix[i] * 6 + ix[j]] + T6[ix[j] * 6 + ix[i]]);
    }
  jacobi_eigh(nb, S, s, U);
  double P[36];  // nb x r
  int r = 0;
  for (int c = 0; c < nb; ++c) {
    if (!(s[c] >= 1e-14)) continue;
    const double f = 1.0 / std::sqrt(s[c]);
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
  jacobi_eigh(r, Hh, w, V);
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
  const auto &Vp = pc->Vp;
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
    if (!(std::isfinite(det) && det != 0.0)) return false;
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
  for (double v : chk)
    if (!std::isfinite(v)) return false;
  return true;
}

struct PairVecs {
  double *x[2], *X[2], *y[2], *Y[2], *z[2], *Z[2];  // z holds z' between steps
};

// Algorithm 2 lines 1-3 for the pair (alpha, alpha + 1): the start vectors
// projected against the stored states (Eqs. S77-S80), normalised, and the
// residuals z'_0 = X_0 - E_0 x_0.
sbci_status pair_start(sbci_ctx *c, VecScratch &vs, PairVecs &P, int alpha, const double E[2]) {
  Solver &s = c->s;
  const long long N = c->ndet;
  std::vector<double> r;
  const double *xc = s.xc;
  auto xcv = [&](int j) { return xc + (size_t)j * N; };
  // Algorithm 2 line 1, Eqs. S77-S80
  if (alpha > 0) {
    std::vector<const double *> u, v;
    for (int i = 0; i < 2; ++i)
      for (int j = 0; j < alpha; ++j) {
        u.push_back(xcv(j));
        v.push_back(P.x[i]);
      }
    RET(dav_dots(vs, u, v, r));
    std::vector<const double *> in{P.x[0], P.x[1], P.X[0], P.X[1]};
    for (int j = 0; j < alpha; ++j) in.push_back(xcv(j));
    std::vector<double> co(in.size() * 4, 0.0);
    for (int q = 0; q < 4; ++q) co[q * 4 + q] = 1.0;
    for (int j = 0; j < alpha; ++j)
      for (int i = 0; i < 2; ++i) {
        co[(4 + j) * 4 + i] = -r[(size_t)i * alpha + j];
        co[(4 + j) * 4 + 2 + i] = -s.Ec[j] * r[(size_t)i * alpha + j];
      }
    RET(dav_combine(vs, {P.x[0], P.x[1], P.X[0], P.X[1]}, in, co));
  }
  RET(dav_dots(vs, {P.x[0], P.x[1]}, {P.x[0], P.x[1]}, r));
  {
    const double n0 = std::sqrt(r[0]), n1 = std::sqrt(r[1]);
    std::vector<double> co(16, 0.0);
    co[0 * 4 + 0] = 1.0 / n0;
    co[1 * 4 + 1] = 1.0 / n1;
    co[2 * 4 + 2] = 1.0 / n0;
    co[3 * 4 + 3] = 1.0 / n1;
    RET(dav_combine(vs, {P.x[0], P.x[1], P.X[0], P.X[1]}, {P.x[0], P.x[1], P.X[0], P.X[1]}, co));
  }
  // line 3: z'_0 = X_0 - E_0 x_0
  return dav_combine(vs, {P.z[0], P.z[1]}, {P.x[0], P.x[1], P.X[0], P.X[1]},
                     {-E[0], 0.0, 0.0, -E[1], 1.0, 0.0, 0.0, 1.0});
}

// The lower state of the pair used its H-product budget (Q8): stored
// unconverged; the normalised upper vector becomes the next lower one.
sbci_status pair_finish_cap(sbci_ctx *c, VecScratch &vs, PairVecs &P, int alpha, double E[2], long long sigma,
                            int nstep, const int restarts[4]) {
  Solver &s = c->s;
  const long long N = c->ndet;
  std::vector<double> r;
  RET(dav_dots(vs, {P.x[0], P.x[1]}, {P.x[0], P.x[1]}, r));
  const double n0 = std::sqrt(r[0]), n1 = std::sqrt(r[1]);
  RET(dav_combine(vs, {s.xc + (size_t)alpha * N}, {P.x[0]}, {1.0 / n0}));
  s.Ec.push_back(E[0]);
  sbci_report &rep = s.rep[alpha];
  rep = sbci_report{};
  rep.energy = E[0] + c->e_core;
  rep.converged = 0;
  rep.n_sigma = rep.n_sigma_fp64 = (int)sigma;
  rep.n_step = nstep;
  for (int i = 0; i < 4; ++i) rep.n_restart[i] = restarts[i];
  s.any_unconverged = 1;
  RET(dav_combine(vs, {P.x[0], P.X[0]}, {P.x[1], P.X[1]}, {1.0 / n1, 0.0, 0.0, 1.0 / n1}));
  E[0] = E[1];
  return SBCI_OK;
}

// The lower state converged (Eq. S127) at Ritz values w, with |z'^a| = dz
// and |x^a|, |x^b| = nx: stored; the normalised upper vector becomes the next
// lower one.
sbci_status pair_finish_converged(sbci_ctx *c, VecScratch &vs, PairVecs &P, int alpha, double E[2],
                                  const double w[2], double dz, const double nx[2], long long sigma, int nstep,
                                  const int restarts[4]) {
  Solver &s = c->s;
  const long long N = c->ndet;
  RET(dav_combine(vs, {s.xc + (size_t)alpha * N}, {P.x[0]}, {1.0 / nx[0]}));
  s.Ec.push_back(w[0]);
  sbci_report &rep = s.rep[alpha];
  rep = sbci_report{};
  rep.energy = w[0] + c->e_core;
  rep.residual = dz;
  rep.converged = 1;
  rep.n_sigma = rep.n_sigma_fp64 = (int)sigma;
  rep.n_step = nstep;
  for (int i = 0; i < 4; ++i) rep.n_restart[i] = restarts[i];
  RET(dav_combine(vs, {P.x[0], P.X[0]}, {P.x[1], P.X[1]}, {1.0 / nx[1], 0.0, 0.0, 1.0 / nx[1]}));
  E[0] = w[1];
  return SBCI_OK;
}

// The pair loop driven from the host (the default): one round trip per step
// for the dots and one for the norms, the small eigen-problems on the host.
sbci_status sbci2_pair_host(sbci_ctx *c, VecScratch &vs, PairVecs &P, int alpha, double E[2], int max_cycle2) {
  Solver &s = c->s;
  const sbci_params &p = s.p;
  const long long N = c->ndet;
  std::vector<double> r;
  const double *xc = s.xc;
  auto xcv = [&](int j) { return xc + (size_t)j * N; };
  RET(pair_start(c, vs, P, alpha, E));
  bool first = true;
  int t = 0, nstep = 0, restarts[4] = {0, 0, 0, 0};
  long long sigma = 0;
  for (;;) {
    if (sigma >= p.max_sigma) return pair_finish_cap(c, vs, P, alpha, E, sigma, nstep, restarts);  // Q8
    const double E_pre = alpha == 0 ? E[0] : s.Ec[0];  // Q3
    for (int i = 0; i < 2; ++i) {  // Eqs. S81 / S101
      RET(timed(c, K_DAVP, [&] {
        return launch_dav_precond(P.z[i], P.z[i], c->d_diag, E_pre, p.guard, N, c->nsm, c->stream);
      }));
      if (p.sector) RET(timed(c, K_DAVP, [&] { return launch_symmetrize(P.z[i], c->Na, c->stream); }));
    }
    if (alpha > 0) {
      std::vector<const double *> u, v;
      for (int i = 0; i < 2; ++i)
        for (int j = 0; j < alpha; ++j) {
          u.push_back(xcv(j));
          v.push_back(P.z[i]);
        }
      RET(dav_dots(vs, u, v, r));
      std::vector<const double *> in{P.z[0], P.z[1]};
      for (int j = 0; j < alpha; ++j) in.push_back(xcv(j));
      std::vector<double> co(in.size() * 2, 0.0);
      co[0] = co[3] = 1.0;
      for (int j = 0; j < alpha; ++j)
        for (int i = 0; i < 2; ++i) co[(2 + j) * 2 + i] = -r[(size_t)i * alpha + j];
      RET(dav_combine(vs, {P.z[0], P.z[1]}, in, co));
    }
    for (int i = 0; i < 2; ++i) {  // Eqs. S82 / S102
      RET(run_sigma(c, P.z[i], P.Z[i], SBCI_FP64));
      ++sigma;
    }
    // overlap and T of the basis (x^a, x^b, y^a, y^b, z^a, z^b)
    const double *Bv[6] = {P.x[0], P.x[1], P.y[0], P.y[1], P.z[0], P.z[1]};
    const double *HB[6] = {P.X[0], P.X[1], P.Y[0], P.Y[1], P.Z[0], P.Z[1]};
    static const int kUse4[4] = {0, 1, 4, 5};
    const int nuse = first ? 4 : 6;
    std::vector<int> use;
    for (int i = 0; i < nuse; ++i) use.push_back(first ? kUse4[i] : i);
    std::vector<const double *> u, v;
    for (int a = 0; a < nuse; ++a)
      for (int b = a; b < nuse; ++b) {
        u.push_back(Bv[use[a]]);
        v.push_back(Bv[use[b]]);
      }
    const size_t ns = u.size();
    for (int a = 0; a < nuse; ++a)
      for (int b = 0; b < nuse; ++b) {
        u.push_back(Bv[use[a]]);
        v.push_back(HB[use[b]]);
      }
    RET(dav_dots(vs, u, v, r));
    double S6[36] = {0}, T6[36] = {0};
    size_t q = 0;
    for (int a = 0; a < nuse; ++a)
      for (int b = a; b < nuse; ++b, ++q) S6[use[a] * 6 + use[b]] = S6[use[b] * 6 + use[a]] = r[q];
    for (int a = 0; a < nuse; ++a)
      for (int b = 0; b < nuse; ++b, ++q) T6[use[a] * 6 + use[b]] = r[q];
    (void)ns;
    PairCoef pc;
    bool ok = false;
    if (!first) ok = pair_step(S6, T6, false, &pc);
    if (!ok) ok = pair_step(S6, T6, true, &pc);  // first step, or Q6
    if (!ok) {
      set_error("SBCI2: the pair step is undefined (subspace rank below 2)");
      return SBCI_ERR_NUMERIC;
    }
    const bool undef = pc.first && !first;
    // one combination: x, X (Q9), y, Y (Eqs. S94-S95 / S122-S123), z' (Eqs. S98, S100 / S126, S128)
    {
      std::vector<const double *> in;
      std::vector<int> basis_ix;  // position in the 6-basis of each vector input
      for (int i = 0; i < 6; ++i) {
        if (pc.first && (i == 2 || i == 3)) continue;
        basis_ix.push_back(i);
      }
      const int nb = (int)basis_ix.size();
      for (int i : basis_ix) in.push_back(Bv[i]);
      for (int i : basis_ix) in.push_back(HB[i]);
      const int nout = 10;
      std::vector<double> co((size_t)2 * nb * nout, 0.0);
      auto C = [&](int qin, int out) -> double & { return co[(size_t)qin * nout + out]; };
      auto pos = [&](int b6) {
        for (int j = 0; j < nb; ++j)
          if (basis_ix[j] == b6) return j;
        return -1;
      };
      for (int i = 0; i < 2; ++i) {
        for (int j = 0; j < nb; ++j) {
          C(j, i) = pc.k[i] * pc.Vp[j][i];            // x_{t+1}^i
          C(nb + j, 2 + i) = pc.k[i] * pc.Vp[j][i];   // X_{t+1}^i
          C(j, 8 + i) = -pc.w[i] * pc.Vp[j][i];       // z'^i = sum_j V'_{j,i} (H b_j - E b_j)
          C(nb + j, 8 + i) = pc.Vp[j][i];
        }
        // y_{t+1}^i = y_t^i - C_{i0} z^a - C_{i1} z^b + A_{i,1-i} x^{1-i}
        if (!pc.first) {
          C(pos(2 + i), 4 + i) = 1.0;
          C(nb + pos(2 + i), 6 + i) = 1.0;
        }
        for (int j = 0; j < 2; ++j) {
          C(pos(4 + j), 4 + i) = -pc.C[i][j];
          C(nb + pos(4 + j), 6 + i) = -pc.C[i][j];
        }
        C(pos(1 - i), 4 + i) = pc.A[i][1 - i];
        C(nb + pos(1 - i), 6 + i) = pc.A[i][1 - i];
      }
      RET(dav_combine(vs, {P.x[0], P.x[1], P.X[0], P.X[1], P.y[0], P.y[1], P.Y[0], P.Y[1], P.z[0], P.z[1]}, in,
                      co));
    }
    ++nstep;
    RET(dav_dots(vs, {P.z[0], P.z[1], P.x[0], P.x[1]}, {P.z[0], P.z[1], P.x[0], P.x[1]}, r));
    const double dz = std::sqrt(r[0]);
    const double nx0 = std::sqrt(r[2]), nx1 = std::sqrt(r[3]);  // |x_{t+1}| (= |k| up to rounding)
    const double dE = std::fabs(pc.w[0] - E[0]);
    sbci_trace_record rec{};
    rec.state = alpha;
    rec.t = t;
    rec.energy = pc.w[0];
    rec.b = pc.B[0][0];
    rec.c = pc.C[0][0];
    rec.k = pc.k[0];
    rec.dE = dE;
    rec.dz = dz;
    rec.event = undef ? 8 : 0;
    rec.prec = SBCI_FP64;
    const double ak0 = std::fabs(pc.k[0]), ak1 = std::fabs(pc.k[1]);
    if (dE < p.eps0 && dz < p.r0) {  // Eq. S99 / S127
      rec.event = 1;
      s.trace.push_back(rec);
      const double nx[2] = {nx0, nx1};
      return pair_finish_converged(c, vs, P, alpha, E, pc.w, dz, nx, sigma, nstep, restarts);
    }
    int cause = -1;  // Section S2.5
    if ((std::fabs(pc.B[0][0]) < p.b_th || std::fabs(pc.B[1][1]) < p.b_th) && dE < p.eps1) cause = 0;
    else if (std::min(ak0, ak1) < p.x_th1 || std::max(ak0, ak1) > p.x_th2) cause = 1;
    else if (dz > p.r1 && t > 0) cause = 2;
    else if (t + 1 >= max_cycle2) cause = 3;
    E[0] = pc.w[0];
    E[1] = pc.w[1];
    if (cause >= 0) {  // Q7
      ++restarts[cause];
      rec.event = 2 + cause;
      s.trace.push_back(rec);
      // x, X normalised; z'_0 = X_0 - E_0 x_0 = z'_{t+1} k / |x_{t+1}|
      std::vector<double> co(36, 0.0);
      const double f[6] = {1.0 / nx0, 1.0 / nx1, 1.0 / nx0, 1.0 / nx1, pc.k[0] / nx0, pc.k[1] / nx1};
      for (int q2 = 0; q2 < 6; ++q2) co[q2 * 6 + q2] = f[q2];
      RET(dav_combine(vs, {P.x[0], P.x[1], P.X[0], P.X[1], P.z[0], P.z[1]},
                      {P.x[0], P.x[1], P.X[0], P.X[1], P.z[0], P.z[1]}, co));
      first = true;
      t = 0;
      continue;
    }
    s.trace.push_back(rec);
    first = false;
    ++t;
  }
}

// ---------------------------------------------------------------------------
// The pair loop on the device: one step = preconditioner and projection of
// the residuals, two FP64 H-products, the dots of the step basis, the pair
// controller (pair_ctl.h: the 6x6 canonical orthogonalisation and subspace
// eigen-problem on one GPU thread), one combination with the coefficients it
// wrote, the norms, the controller's decision and the rescaling of a restart.
// The steps run as one CUDA-graph while-loop; the host acts only when the
// lower state converged or used its budget.  Selected by SBCI_SBCI2_DEVICE=1
// (read when a context is created).  On GB300 it is the slower loop: the two
// FP64 6x6 Jacobi solves of a step on one GPU thread (FP64 at two lanes per
// SM and clock) take longer than the host round trips they replace (H10:
// 112 ms against 52 ms per 4-state solve), so the host-driven loop is the
// default.


// Device buffers of the pair controller: its state and its trace ring.
struct PairDev {
  PairCtl *d = nullptr;
  sbci_trace_record *trace = nullptr;
  int trace_cap = 0;
  cudaStream_t stream = nullptr;
  ~PairDev() {
    if (stream) cudaStreamSynchronize(stream);  // the buffers go back to the pool
    if (d) pool_free(d);
    if (trace) pool_free(trace);
  }
};

// The kernels of one pair step (cond: the graph's loop handle, 0 outside a
// graph; timing: count and time each launch, not in a capture).
sbci_status pair_body(sbci_ctx *c, VecScratch &vs, PairVecs &P, PairCtl *d, int alpha, unsigned long long cond,
                      bool timing) {
  Solver &s = c->s;
  const sbci_params &p = s.p;
  const long long N = c->ndet;
  cudaStream_t st = c->stream;
  auto L = [&](int kid, auto &&f) -> sbci_status {
    if (timing) return timed(c, kid, f);
    CK(f());
    return SBCI_OK;
  };
  // Eqs. S81 / S101, shift Q3
  const double *shift = alpha == 0 ? &d->E[0] : &d->Ec0;
  for (int i = 0; i < 2; ++i) {
    RET(L(K_DAVP, [&] { return launch_dav_precond_dev(P.z[i], P.z[i], c->d_diag, shift, p.guard, N, c->nsm, st); }));
    if (p.sector) RET(L(K_DAVP, [&] { return launch_symmetrize(P.z[i], c->Na, st); }));
  }
  if (alpha > 0) {  // against the stored states
    std::vector<const double *> u, v, in{P.z[0], P.z[1]};
    for (int i = 0; i < 2; ++i)
      for (int j = 0; j < alpha; ++j) {
        u.push_back(s.xc + (size_t)j * N);
        v.push_back(P.z[i]);
      }
    for (int j = 0; j < alpha; ++j) in.push_back(s.xc + (size_t)j * N);
    RET(L(K_DAVD, [&] { return launch_dav_dots(u.data(), v.data(), 2 * alpha, N, vs.partials, vs.grid, st); }));
    RET(L(K_RED, [&] { return launch_reduce(vs.partials, vs.grid, 0, 2 * alpha, vs.d_res, st); }));
    RET(L(K_PAIR, [&] { return launch_pair_proj_coef(d, vs.d_res, st); }));
    double *out[2] = {P.z[0], P.z[1]};
    RET(L(K_DAVC, [&] {
      return launch_dav_combine_dev(out, 2, in.data(), (int)in.size(), d->proj, nullptr, N, c->nsm, st);
    }));
  }
  for (int i = 0; i < 2; ++i) {  // Eqs. S82 / S102
    const SigmaArgs a = plain_sigma_args(c, P.z[i], P.Z[i]);
    RET(L(gc_kid(c, SBCI_FP64), [&] { return launch_gc(c, a, SBCI_FP64); }));
    RET(L(K_SC, [&] { return launch_scatter(a, 0, st); }));
  }
  // overlap and T of the basis (x^a, x^b, y^a, y^b, z^a, z^b)
  const double *Bv[6] = {P.x[0], P.x[1], P.y[0], P.y[1], P.z[0], P.z[1]};
  const double *HB[6] = {P.X[0], P.X[1], P.Y[0], P.Y[1], P.Z[0], P.Z[1]};
  std::vector<const double *> u, v;
  for (int a = 0; a < 6; ++a)
    for (int b = a; b < 6; ++b) {
      u.push_back(Bv[a]);
      v.push_back(Bv[b]);
    }
  for (int a = 0; a < 6; ++a)
    for (int b = 0; b < 6; ++b) {
      u.push_back(Bv[a]);
      v.push_back(HB[b]);
    }
  RET(L(K_DAVD, [&] { return launch_dav_dots(u.data(), v.data(), kPairDots, N, vs.partials, vs.grid, st); }));
  RET(L(K_RED, [&] { return launch_reduce(vs.partials, vs.grid, 0, kPairDots, vs.d_res, st); }));
  RET(L(K_PAIR, [&] { return launch_pair_after_dots(d, vs.d_res, st); }));
  {  // x, X (Q9), y, Y (Eqs. S94-S95 / S122-S123), z' (Eqs. S98, S100 / S126, S128)
    const double *in[kPairIn] = {P.x[0], P.x[1], P.y[0], P.y[1], P.z[0], P.z[1],
                                 P.X[0], P.X[1], P.Y[0], P.Y[1], P.Z[0], P.Z[1]};
    double *out[kPairOut] = {P.x[0], P.x[1], P.X[0], P.X[1], P.y[0], P.y[1], P.Y[0], P.Y[1], P.z[0], P.z[1]};
    RET(L(K_DAVC, [&] {
      return launch_dav_combine_dev(out, kPairOut, in, kPairIn, d->comb, nullptr, N, c->nsm, st);
    }));
  }
  const double *nu[4] = {P.z[0], P.z[1], P.x[0], P.x[1]};
  RET(L(K_DAVD, [&] { return launch_dav_dots(nu, nu, 4, N, vs.partials, vs.grid, st); }));
  RET(L(K_RED, [&] { return launch_reduce(vs.partials, vs.grid, 0, 4, vs.d_res, st); }));
  RET(L(K_PAIR, [&] { return launch_pair_decide(d, vs.d_res, cond, st); }));
  // a restart (Q7): x, X normalised, z' scaled to k / |x|
  double *sv[6] = {P.x[0], P.x[1], P.X[0], P.X[1], P.z[0], P.z[1]};
  const double *si[6] = {P.x[0], P.x[1], P.X[0], P.X[1], P.z[0], P.z[1]};
  RET(L(K_DAVC, [&] { return launch_dav_combine_dev(sv, 6, si, 6, d->scale, &d->restart, N, c->nsm, st); }));
  return SBCI_OK;
}

// Kernels a graph-run pair step launched (the counts the timed path keeps).
void count_pair_bodies(sbci_ctx *c, int alpha, long long steps) {
  Prof &pf = c->prof;
  const long long sec = c->s.p.sector ? 2 : 0;
  pf.launches[K_DAVP] += (2 + sec) * steps;
  pf.launches[K_DAVD] += (2 + (alpha > 0)) * steps;
  pf.launches[K_RED] += (2 + (alpha > 0)) * steps;
  pf.launches[K_PAIR] += (2 + (alpha > 0)) * steps;
  pf.launches[K_DAVC] += (2 + (alpha > 0)) * steps;
  pf.launches[gc_kid(c, SBCI_FP64)] += 2 * steps;
  pf.launches[K_SC] += 2 * steps;
}

sbci_status sbci2_pair_dev(sbci_ctx *c, VecScratch &vs, PairVecs &P, int alpha, double E[2], int max_cycle2,
                           PairDev &pd) {
  Solver &s = c->s;
  const sbci_params &p = s.p;
  RET(pair_start(c, vs, P, alpha, E));
  const int none[4] = {0, 0, 0, 0};
  if (p.max_sigma <= 0) return pair_finish_cap(c, vs, P, alpha, E, 0, 0, none);  // Q8 before any step
  if (!pd.d) {
    pd.stream = c->stream;
    CK(pool_malloc((void **)&pd.d, sizeof(PairCtl)));
    pd.trace_cap = p.max_sigma / 2 + 16;  // two H-products per step
    CK(pool_malloc((void **)&pd.trace, sizeof(sbci_trace_record) * pd.trace_cap));
  }
  PairCtl h{};
  h.eps0 = p.eps0;
  h.r0 = p.r0;
  h.b_th = p.b_th;
  h.eps1 = p.eps1;
  h.x_th1 = p.x_th1;
  h.x_th2 = p.x_th2;
  h.r1 = p.r1;
  h.Ec0 = alpha > 0 ? s.Ec[0] : 0.0;
  h.alpha = alpha;
  h.max_sigma = p.max_sigma;
  h.max_cycle2 = max_cycle2;
  h.trace_cap = pd.trace_cap;
  h.E[0] = E[0];
  h.E[1] = E[1];
  h.first = 1;
  h.trace = pd.trace;
  CK(cudaMemcpyAsync(pd.d, &h, sizeof(PairCtl), cudaMemcpyHostToDevice, c->stream));
  RET(ensure_G(c, SBCI_FP64));
  if (use_graphs(c)) {
    cudaGraph_t g = nullptr;
    CK(cudaGraphCreate(&g, 0));
    cudaGraphConditionalHandle hd;
    cudaGraphExec_t ex = nullptr;
    auto fail = [&](sbci_status stt) {
      if (ex) cudaGraphExecDestroy(ex);
      cudaGraphDestroy(g);
      return stt;
    };
    if (cudaGraphConditionalHandleCreate(&hd, g, 1u, cudaGraphCondAssignDefault) != cudaSuccess)
      return fail(SBCI_ERR_CUDA);
    cudaGraphNodeParams np{};
    np.type = cudaGraphNodeTypeConditional;
    np.conditional.handle = hd;
    np.conditional.type = cudaGraphCondTypeWhile;
    np.conditional.size = 1;
    cudaGraphNode_t node;
    if (cudaGraphAddNode(&node, g, nullptr, nullptr, 0, &np) != cudaSuccess) return fail(SBCI_ERR_CUDA);
    if (cudaStreamBeginCaptureToGraph(c->stream, np.conditional.phGraph_out[0], nullptr, nullptr, 0,
                                      cudaStreamCaptureModeThreadLocal) != cudaSuccess)
      return fail(SBCI_ERR_CUDA);
    const sbci_status bst = pair_body(c, vs, P, pd.d, alpha, (unsigned long long)hd, false);
    cudaGraph_t captured = nullptr;
    const cudaError_t ce = cudaStreamEndCapture(c->stream, &captured);
    if (bst != SBCI_OK) return fail(bst);
    if (ce != cudaSuccess || cudaGraphInstantiate(&ex, g, 0) != cudaSuccess ||
        cudaGraphLaunch(ex, c->stream) != cudaSuccess) {
      set_error("SBCI2: the pair-step graph could not be built or launched");
      return fail(SBCI_ERR_CUDA);
    }
    CK(cudaMemcpyAsync(&h, pd.d, sizeof(PairCtl), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    fail(SBCI_OK);
    count_pair_bodies(c, alpha, h.nstep);
  } else {  // one step at a time (per-kernel timing)
    for (;;) {
      RET(pair_body(c, vs, P, pd.d, alpha, 0, true));
      CK(cudaMemcpyAsync(&h, pd.d, sizeof(PairCtl), cudaMemcpyDeviceToHost, c->stream));
      CK(cudaStreamSynchronize(c->stream));
      if (h.halt != PH_RUN) break;
    }
  }
  {  // a bounded MMA wait of the H-products that ran out
    int status = 0;
    CK(cudaMemcpy(&status, c->d_status, sizeof(int), cudaMemcpyDeviceToHost));
    if (status != 0) {
      set_error("a bounded device wait ran out (tensor-core MMA completion)");
      return SBCI_ERR_TIMEOUT;
    }
  }
  if (h.ntrace > 0) {
    const int n = std::min(h.ntrace, h.trace_cap);
    std::vector<sbci_trace_record> tr(n);
    CK(cudaMemcpy(tr.data(), pd.trace, sizeof(sbci_trace_record) * n, cudaMemcpyDeviceToHost));
    s.trace.insert(s.trace.end(), tr.begin(), tr.end());
  }
  E[0] = h.E[0];  // the pair's energies after its last completed step
  E[1] = h.E[1];
  switch (h.halt) {
    case PH_CONVERGED:
      return pair_finish_converged(c, vs, P, alpha, E, h.w, h.dz, h.nx, h.sigma, h.nstep, h.restarts);
    case PH_CAP:
      return pair_finish_cap(c, vs, P, alpha, E, h.sigma, h.nstep, h.restarts);
    case PH_UNDEF:
      set_error("SBCI2: the pair step is undefined (subspace rank below 2)");
      return SBCI_ERR_NUMERIC;
    case PH_BOUND:
      set_error("SBCI2: the pair loop ran past its step bound without reaching the H-product cap");
      return SBCI_ERR_NUMERIC;
    default:
      set_error("non-finite dot product in a device reduction (SBCI2)");
      return SBCI_ERR_NUMERIC;
  }
}

sbci_status sbci2_run(sbci_ctx *c, int k, int max_cycle2) {
  Solver &s = c->s;
  const sbci_params &p = s.p;
  const long long N = c->ndet;
  VecScratch vs;
  RET(scratch_init(vs, c));
  DevBuffers buf;
  // Q1, Eqs. S74-S76: start vectors and their H-images
  std::vector<Sparse> basis;
  RET(lowest_diagonal_basis(c, std::max(k, p.n_init > 0 ? p.n_init : 2), p, basis));
  const int m = (int)basis.size();
  if (m < k) {
    set_error("sbci_solve_sbci2: the space holds fewer than k start vectors");
    return SBCI_ERR_INVALID;
  }
  if (m > kDavMaxIn / 2) {
    set_error("sbci_solve_sbci2: n_init too large");
    return SBCI_ERR_INVALID;
  }
  std::vector<double *> e(m), He(m), xs(k), Xs(k);
  for (int j = 0; j < m; ++j) {
    RET(buf.get(c, &e[j]));
    RET(buf.get(c, &He[j]));
    RET(upload_sparse(c, basis[j], e[j]));
    RET(run_sigma(c, e[j], He[j], SBCI_FP64));
  }
  std::vector<double> r, A((size_t)m * m), w(m), U((size_t)m * m);
  {
    std::vector<const double *> u, v;
    for (int i = 0; i < m; ++i)
      for (int j = 0; j < m; ++j) {
        u.push_back(e[i]);
        v.push_back(He[j]);
      }
    RET(dav_dots(vs, u, v, r));
    for (int i = 0; i < m; ++i)
      for (int j = 0; j < m; ++j) A[(size_t)i * m + j] = 0.5 * (r[(size_t)i * m + j] + r[(size_t)j * m + i]);
    jacobi_eigh(m, A.data(), w.data(), U.data());
  }
  for (int i = 0; i < k; ++i) {
    RET(buf.get(c, &xs[i]));
    RET(buf.get(c, &Xs[i]));
  }
  {
    std::vector<const double *> in;
    for (int j = 0; j < m; ++j) in.push_back(e[j]);
    for (int j = 0; j < m; ++j) in.push_back(He[j]);
    for (int i0 = 0; i0 < k; i0 += kDavMaxOut / 2) {
      const int ni = std::min(kDavMaxOut / 2, k - i0);
      std::vector<double *> out;
      std::vector<double> co((size_t)2 * m * 2 * ni, 0.0);
      for (int i = 0; i < ni; ++i) out.push_back(xs[i0 + i]);
      for (int i = 0; i < ni; ++i) out.push_back(Xs[i0 + i]);
      for (int j = 0; j < m; ++j)
        for (int i = 0; i < ni; ++i) {
          co[(size_t)j * 2 * ni + i] = U[(size_t)j * m + i0 + i];
          co[(size_t)(m + j) * 2 * ni + ni + i] = U[(size_t)j * m + i0 + i];
        }
      RET(dav_combine(vs, out, in, co));
    }
  }
  PairVecs P;
  for (int i = 0; i < 2; ++i) {
    RET(buf.get(c, &P.x[i]));
    RET(buf.get(c, &P.X[i]));
    RET(buf.get(c, &P.y[i]));
    RET(buf.get(c, &P.Y[i]));
    RET(buf.get(c, &P.z[i]));
    RET(buf.get(c, &P.Z[i]));
    // y, Y enter the device loop's combination with zero coefficients on
    // first-step paths: they start as zeros, not as uninitialised memory
    CK(cudaMemsetAsync(P.y[i], 0, sizeof(double) * N, c->stream));
    CK(cudaMemsetAsync(P.Y[i], 0, sizeof(double) * N, c->stream));
  }
  const bool on_device = c->sbci2_device;
  PairDev pd;
  double E[2] = {w[0], k > 1 ? w[1] : 0.0};
  RET(dav_combine(vs, {P.x[0], P.X[0]}, {xs[0], Xs[0]}, {1.0, 0.0, 0.0, 1.0}));
  for (int alpha = 0; alpha + 1 < k; ++alpha) {
    if (alpha == 0) {
      RET(dav_combine(vs, {P.x[1], P.X[1]}, {xs[1], Xs[1]}, {1.0, 0.0, 0.0, 1.0}));
      E[1] = w[1];
    } else {  // Q2, Q10
      std::vector<const double *> u, v, in{xs[alpha + 1]};
      for (int j = 0; j < alpha; ++j) {
        u.push_back(s.xc + (size_t)j * N);
        v.push_back(xs[alpha + 1]);
      }
      RET(dav_dots(vs, u, v, r));
      std::vector<double> co{1.0};
      for (int j = 0; j < alpha; ++j) {
        in.push_back(s.xc + (size_t)j * N);
        co.push_back(-r[j]);
      }
      RET(dav_combine(vs, {P.x[1]}, in, co));
      RET(dav_dots(vs, {P.x[0]}, {P.x[1]}, r));
      RET(dav_combine(vs, {P.x[1]}, {P.x[1], P.x[0]}, {1.0, -r[0]}));
      RET(dav_dots(vs, {P.x[1]}, {P.x[1]}, r));
      RET(dav_combine(vs, {P.x[1]}, {P.x[1]}, {1.0 / std::sqrt(r[0])}));
      RET(run_sigma(c, P.x[1], P.X[1], SBCI_FP64));
      RET(dav_dots(vs, {P.x[1]}, {P.X[1]}, r));
      E[1] = r[0];
    }
    if (on_device) RET(sbci2_pair_dev(c, vs, P, alpha, E, max_cycle2, pd));
    else RET(sbci2_pair_host(c, vs, P, alpha, E, max_cycle2));
  }
  // the highest state: SBCI1 from the last pair's normalised upper vector
  // (Fig. 1B), projected against the stored states (Eqs. S4-S7)
  CK(cudaMemcpyAsync(s.x, P.x[0], sizeof(double) * N, cudaMemcpyDeviceToDevice, c->stream));
  CK(cudaMemcpyAsync(s.X, P.X[0], sizeof(double) * N, cudaMemcpyDeviceToDevice, c->stream));
  const int last = k - 1;
  if (last > 0) {
    std::vector<const double *> u, v;
    for (int i = 0; i < last; ++i) {
      u.push_back(s.xc + (size_t)i * N);
      v.push_back(s.x);
    }
    RET(dav_dots(vs, u, v, r));
    std::vector<const double *> in{s.x, s.X};
    std::vector<double> co{1.0, 0.0, 0.0, 1.0};
    for (int i = 0; i < last; ++i) {
      in.push_back(s.xc + (size_t)i * N);
      co.push_back(-r[i]);
      co.push_back(-s.Ec[i] * r[i]);
    }
    RET(dav_combine(vs, {s.x, s.X}, in, co));
  }
  RET(dav_dots(vs, {s.x}, {s.x}, r));
  const double nrm = std::sqrt(r[0]);
  RET(dav_combine(vs, {s.x, s.X}, {s.x, s.X}, {1.0 / nrm, 0.0, 0.0, 1.0 / nrm}));
  RET(start_state(c, last, E[0]));
  while (!s.done) {
    RET(run_until_halt(c));
    const sbci_status st = handle_halt(c);
    if (st != SBCI_OK && st != SBCI_ERR_NOT_CONVERGED) return st;
  }
  return SBCI_OK;
}

}  // namespace

// Asynchronous rounds of a solve, for the serving layer: launch the graph loop
// on the context stream (no wait), then, once the stream has passed it, read
// the controller and act on the halt.
sbci_status sbci::solve_round_launch(sbci_ctx *c) {
  Solver &s = c->s;
  if (!s.active || s.done) return SBCI_ERR_INVALID;
  const int prec = s.h_ctl->prec;
  if (!s.gexec[prec]) RET(build_graph(c, prec));
  CK(cudaGraphLaunch(s.gexec[prec], c->stream));
  return SBCI_OK;
}

sbci_status sbci::solve_round_read(sbci_ctx *c, int *done, bool own_graph, int *deferred) {
  Solver &s = c->s;
  *deferred = 0;
  RET(ctl_read(c));
  const long long bodies = s.h_ctl->iters;
  const int prec = s.h_ctl->prec;
  if (own_graph) count_bodies(c, prec, bodies);  // the kernels the solve's own graph ran
  s.h_ctl->iters = 0;
  CK(cudaMemsetAsync(&s.d_ctl->iters, 0, sizeof(int), c->stream));
  if (halt_needs_resync(c)) {
    RET(resync_issue(c));
    *deferred = 1;
    *done = 0;
    return SBCI_OK;
  }
  const sbci_status st = handle_halt(c);
  *done = s.done ? 1 : 0;
  return st;
}

sbci_status sbci::solve_round_complete(sbci_ctx *c, int *done) {
  Solver &s = c->s;
  double xx, xX, XX;
  RET(resync_complete(c, &xx, &xX, &XX));
  const sbci_status st = converged_after_resync(c, xx, xX, XX);
  *done = s.done ? 1 : 0;
  return st;
}

sbci_status sbci::solve_round_finish(sbci_ctx *c, int *done, bool own_graph) {
  int deferred = 0;
  RET(solve_round_read(c, done, own_graph, &deferred));
  return deferred ? solve_round_complete(c, done) : SBCI_OK;
}

cudaStream_t sbci::ctx_stream(const sbci_ctx *c) { return c->stream; }

cudaError_t sbci::ctx_fence(sbci_ctx *c, cudaStream_t waiter) {
  cudaError_t e = cudaEventRecord(c->ev_fence, c->stream);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(waiter, c->ev_fence, 0);
  return e;
}

bool sbci::ctx_batch_job(sbci_ctx *c, BatchJob *j) {
  Solver &s = c->s;
  if (!s.active || s.done || s.p.prec != SBCI_TF32X3 || s.h_ctl->prec != SBCI_TF32X3 ||
      c->npair > kBatchMaxPair)
    return false;
  uint32_t cols;
  size_t smem;
  if (!tc_dims(c->npair, &j->Kp, &j->Np, &cols, &smem)) return false;
  j->step = step_args(c, 0);
  j->sig = sigma_ctl_args(c, SBCI_TF32X3, 0);
  j->fused = use_fused(c, SBCI_TF32X3) ? 1 : 0;
  return true;
}

int sbci::ctx_step_blocks(const sbci_ctx *c) { return step_blocks(c); }
int sbci::ctx_scatter_blocks(const sbci_ctx *c) { return scatter_grid(c->ndet, c->nsm); }
int sbci::ctx_symfin_blocks(const sbci_ctx *c) { return use_symfin(c) ? symfin_grid(c->Na, c->nsm) : 0; }
long long sbci::ctx_ndet(const sbci_ctx *c) { return c->ndet; }
int sbci::ctx_device(const sbci_ctx *c) { return c->device; }

long long sbci::ctx_launch_count(const sbci_ctx *c) {
  long long n = 0;
  for (int i = 0; i < K_COUNT; ++i) n += c->prof.launches[i];
  return n;
}

size_t sbci::ctx_device_bytes(int norb, int nalpha, int nbeta, int k) {
  auto binom = [](int n, int r) {
    long long v = 1;
    for (int i = 1; i <= r; ++i) v = v * (n - r + i) / i;
    return v;
  };
  const long long na = binom(norb, nalpha), nb = binom(norb, nbeta), nd = na * nb;
  const long long npair = norb * (norb + 1) / 2;
  const long long vec = (10LL + k) * nd * 8 + nd * 4;  // x X y Y w z0 z1 Z0 Z1 pinv + stored states + FP32 z
  const long long G = npair * nd * 8;            // sigma scratch (FP64 size, shared by FP32 modes)
  const long long tab = (na * nalpha * (norb - nalpha + 1) + nb * nbeta * (norb - nbeta + 1)) * 4;
  return (size_t)(vec + G + tab + nd * 8 + (1 << 20));
}

bool sbci::ctx_sigma_args(const sbci_ctx *c, SigmaArgs *a, cudaStream_t *stream) {
  if (!c) return false;
  *a = SigmaArgs{};
  a->link_a = c->d_link_a;
  a->link_b = c->d_link_b;
  a->link_bT = c->d_link_bT;
  a->W = c->d_W;
  a->Wf = c->d_Wf;
  a->Wtc = c->d_Wtc;
  a->fc_link_a = c->d_fc_link_a;
  a->na = c->Na;
  a->nb = c->Nb;
  a->nlink_a = c->sa.nlink;
  a->nlink_b = c->sb.nlink;
  a->npair = c->npair;
  a->npair_pad = c->npair_pad;
  a->ndet = c->ndet;
  a->grid = c->grid;
  if (stream) *stream = c->stream;
  return true;
}

// ===========================================================================
extern "C" {

const char *sbci_last_error(void) { return g_err.c_str(); }

sbci_status sbci_params_init(sbci_params *p) {
  if (!p) {
    set_error("sbci_params_init: NULL");
    return SBCI_ERR_INVALID;
  }
  p->eps0 = 1e-10;
  p->r0 = 1e-5;
  p->b_th = 1e-2;
  p->eps1 = 1e-7;
  p->x_th1 = 0.1;
  p->x_th2 = 1.2;
  p->r1 = 1.0;
  p->max_cycle = 20;
  p->max_sigma = 1000;
  p->guard = 1e-8;
  p->gs_tol = 1e-14;
  p->sector = 0;
  p->n_init = 0;
  p->init = 0;
  p->prec = SBCI_FP64;
  p->mixed_eps = 1e-8;
  p->mixed_r = 1e-4;
  p->refine_max_sigma = 300;
  p->start_noise = 0.0;
  p->noise_seed = 0;
  p->init_stage = 0;
  return SBCI_OK;
}

sbci_status sbci_pool_stats(size_t *cached_bytes, long long *hits, long long *misses) {
  pool_stats(cached_bytes, hits, misses);
  return SBCI_OK;
}

sbci_status sbci_pool_trim(void) {
  const cudaError_t e = pool_trim();
  if (e != cudaSuccess) {
    set_error(std::string("sbci_pool_trim: ") + cudaGetErrorString(e));
    return SBCI_ERR_CUDA;
  }
  return SBCI_OK;
}

void sbci_destroy(sbci_ctx *c) {
  if (!c) return;
  if (c->stream) cudaStreamSynchronize(c->stream);  // its buffers go back to the pool
  free_solver(c);
  for (cudaEvent_t e : c->prof.pool) cudaEventDestroy(e);
  void *ptrs[] = {c->d_link_a, c->d_link_bT, c->d_mask_b, c->d_W, c->d_Wf, c->d_Wtc, c->d_Wbf, c->d_fc_link_a, c->d_Wos, c->d_fexp, c->d_cf,
                  c->d_diag, c->d_ea, c->d_eb, c->d_ja, c->d_G, c->d_partials, c->d_result, c->d_tmp_in,
                  c->d_tmp_out, c->d_lrUt64, c->d_lrUL64, c->d_Wtclr};
  for (void *p : ptrs)
    if (p) pool_free(p);
  if (c->d_link_b && c->d_link_b != c->d_link_a) pool_free(c->d_link_b);
  if (c->ev_fence) cudaEventDestroy(c->ev_fence);
  if (c->h_result) pool_free_host(c->h_result);
  if (c->h_status) pool_free_host(c->h_status);
  if (c->d_status) pool_free(c->d_status);
  if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
  delete c;
}

sbci_status sbci_init_integrals(sbci_ctx **out, int norb, int nalpha, int nbeta, const double *h1,
                                const double *eri, double e_core, void *cuda_stream) {
  if (!out || !h1 || !eri) {
    set_error("sbci_init_integrals: NULL argument");
    return SBCI_ERR_INVALID;
  }
  *out = nullptr;
  if (norb < 1 || norb > kMaxOrb || nalpha < 0 || nbeta < 0 || nalpha > norb || nbeta > norb ||
      nalpha + nbeta < 1) {
    set_error("sbci_init_integrals: need 1 <= norb <= 16, 0 <= nalpha, nbeta <= norb, nalpha+nbeta >= 1");
    return SBCI_ERR_INVALID;
  }
  const int n = norb;
  const size_t n2 = (size_t)n * n, n4 = n2 * n2;
  RET(check_finite(h1, n2, "h1"));
  RET(check_finite(eri, n4, "eri"));
  if (!std::isfinite(e_core)) {
    set_error("non-finite e_core");
    return SBCI_ERR_NUMERIC;
  }
  // the packed contraction relies on h = h^T and the 8-fold symmetry of (ij|kl)
  double scale = 0.0;
  for (size_t i = 0; i < n4; ++i) scale = std::max(scale, std::fabs(eri[i]));
  for (size_t i = 0; i < n2; ++i) scale = std::max(scale, std::fabs(h1[i]));
  const double tol = 1e-10 * (scale > 0 ? scale : 1.0);
  auto E4 = [&](int i, int j, int k, int l) { return eri[(((size_t)i * n + j) * n + k) * n + l]; };
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) {
      if (std::fabs(h1[i * n + j] - h1[j * n + i]) > tol) {
        set_error("h1 is not symmetric");
        return SBCI_ERR_INVALID;
      }
      for (int k = 0; k < n; ++k)
        for (int l = 0; l < n; ++l) {
          const double v = E4(i, j, k, l);
          if (std::fabs(v - E4(j, i, k, l)) > tol || std::fabs(v - E4(i, j, l, k)) > tol ||
              std::fabs(v - E4(k, l, i, j)) > tol) {
            set_error("eri lacks the 8-fold symmetry of real-orbital (ij|kl)");
            return SBCI_ERR_INVALID;
          }
        }
    }
  sbci_ctx *c = new sbci_ctx();
  c->n = n;
  c->ne_a = nalpha;
  c->ne_b = nbeta;
  c->e_core = e_core;
  build_strings(n, nalpha, c->sa);
  build_strings(n, nbeta, c->sb);
  c->Na = c->sa.nstr;
  c->Nb = c->sb.nstr;
  c->ndet = (long long)c->Na * c->Nb;
  c->npair = n * (n + 1) / 2;
  c->npair_pad = (c->npair + 7) / 8 * 8;
  if (cuda_stream) {
    c->stream = (cudaStream_t)cuda_stream;
  } else {
    cudaError_t e = cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
      set_error(std::string("cudaStreamCreate: ") + cudaGetErrorString(e));
      delete c;
      return SBCI_ERR_CUDA;
    }
    c->own_stream = true;
  }
  int dev = 0, nsm = 0;
  sbci_status st = SBCI_OK;
#define TRY(x)                  \
  do {                          \
    st = (x);                   \
    if (st != SBCI_OK) {        \
      sbci_destroy(c);          \
      return st;                \
    }                           \
  } while (0)
  auto cuda_ok = [&](cudaError_t e, const char *what) -> sbci_status {
    if (e == cudaSuccess) return SBCI_OK;
    set_error(std::string(what) + ": " + cudaGetErrorString(e));
    return e == cudaErrorMemoryAllocation ? SBCI_ERR_NOMEM : SBCI_ERR_CUDA;
  };
  TRY(cuda_ok(cudaGetDevice(&dev), "cudaGetDevice"));
  TRY(cuda_ok(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev), "attr"));
  c->nsm = std::max(nsm, 1);
  c->device = dev;
  c->grid = 8 * c->nsm;  // upper bound of every kernel's block count that writes partials
  TRY(cuda_ok(prepare_sigma_kernels(), "kernel attributes"));
  // packed operator W[P][Q], P = (i>=j), Q = (k>=l):
  //   W = 1/2 (ij|kl) + (k_ij d_kl + d_ij k_kl) / (2N),  k_ij = h_ij - 1/2 sum_m (im|mj)
  const int N = nalpha + nbeta;
  std::vector<double> kmat(n2);
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) {
      double s = h1[i * n + j];
      for (int m = 0; m < n; ++m) s -= 0.5 * E4(i, m, m, j);
      kmat[i * n + j] = s;
    }
  c->W_host.assign((size_t)c->npair_pad * c->npair, 0.0);
  for (int i = 0, P = 0; i < n; ++i)
    for (int j = 0; j <= i; ++j, ++P)
      for (int k = 0, Q = 0; k < n; ++k)
        for (int l = 0; l <= k; ++l, ++Q) {
          double v = 0.5 * E4(i, j, k, l);
          if (k == l) v += kmat[i * n + j] / (2.0 * N);
          if (i == j) v += kmat[k * n + l] / (2.0 * N);
          c->W_host[(size_t)P * c->npair + Q] = v;
        }
  std::vector<float> Wf(c->W_host.begin(), c->W_host.end());
  // per-string diagonal pieces
  std::vector<double> ea(c->Na), eb(c->Nb), ja((size_t)c->Na * n);
  auto string_energy = [&](uint32_t m) {
    double e = 0.0;
    for (int p = 0; p < n; ++p) {
      if (!(m >> p & 1u)) continue;
      e += h1[p * n + p];
      for (int q = 0; q < n; ++q)
        if (m >> q & 1u) e += 0.5 * (E4(p, p, q, q) - E4(p, q, q, p));
    }
    return e;
  };
  for (int a = 0; a < c->Na; ++a) {
    ea[a] = string_energy(c->sa.masks[a]);
    for (int q = 0; q < n; ++q) {
      double s = 0.0;
      for (int p = 0; p < n; ++p)
        if (c->sa.masks[a] >> p & 1u) s += E4(p, p, q, q);
      ja[(size_t)a * n + q] = s;
    }
  }
  for (int b = 0; b < c->Nb; ++b) eb[b] = string_energy(c->sb.masks[b]);
  // device uploads
  auto up = [&](void **dst, const void *src, size_t bytes) -> sbci_status {
    sbci_status r = cuda_ok(pool_malloc(dst, bytes ? bytes : 1), "cudaMalloc");
    if (r != SBCI_OK) return r;
    return cuda_ok(cudaMemcpyAsync(*dst, src, bytes, cudaMemcpyHostToDevice, c->stream), "H2D");
  };
  TRY(up((void **)&c->d_link_a, c->sa.links.data(), c->sa.links.size() * 4));
  if (nbeta == nalpha) c->d_link_b = c->d_link_a;
  else TRY(up((void **)&c->d_link_b, c->sb.links.data(), c->sb.links.size() * 4));
  {
    std::vector<uint32_t> bT((size_t)c->sb.nlink * c->Nb);
    for (int e = 0; e < c->sb.nlink; ++e)
      for (int ib = 0; ib < c->Nb; ++ib) bT[(size_t)e * c->Nb + ib] = c->sb.links[(size_t)ib * c->sb.nlink + e];
    TRY(up((void **)&c->d_link_bT, bT.data(), bT.size() * 4));
  }
  TRY(up((void **)&c->d_mask_b, c->sb.masks.data(), c->sb.masks.size() * 4));
  TRY(up((void **)&c->d_W, c->W_host.data(), c->W_host.size() * 8));
  TRY(up((void **)&c->d_Wf, Wf.data(), Wf.size() * 4));
  TRY(up((void **)&c->d_ea, ea.data(), ea.size() * 8));
  TRY(up((void **)&c->d_eb, eb.data(), eb.size() * 8));
  TRY(up((void **)&c->d_ja, ja.data(), ja.size() * 8));
  TRY(cuda_ok(pool_malloc((void **)&c->d_diag, sizeof(double) * c->ndet), "cudaMalloc diag"));
  TRY(cuda_ok(pool_malloc((void **)&c->d_partials, sizeof(double) * S_COUNT * c->grid), "cudaMalloc"));
  TRY(cuda_ok(cudaMemsetAsync(c->d_partials, 0, sizeof(double) * S_COUNT * c->grid, c->stream), "memset"));
  TRY(cuda_ok(pool_malloc((void **)&c->d_result, sizeof(double) * S_COUNT), "cudaMalloc"));
  TRY(cuda_ok(pool_malloc_host((void **)&c->h_result, sizeof(double) * S_COUNT), "cudaMallocHost"));
  TRY(cuda_ok(pool_malloc_host((void **)&c->h_status, sizeof(int)), "cudaMallocHost"));
  *c->h_status = 0;
  TRY(cuda_ok(pool_malloc((void **)&c->d_status, sizeof(int)), "cudaMalloc"));
  TRY(cuda_ok(cudaEventCreateWithFlags(&c->ev_fence, cudaEventDisableTiming), "cudaEventCreate"));
  TRY(cuda_ok(cudaMemsetAsync(c->d_status, 0, sizeof(int), c->stream), "memset"));
  c->tc_grid = tc_grid(c->npair, c->ndet, c->nsm);
  {
    const char *e = std::getenv("SBCI_SBCI2_DEVICE");
    c->sbci2_device = e && std::strcmp(e, "1") == 0;
  }
  {  // the pipelined form of the tensor-core kernel where the plain one runs
     // one CTA per SM (its operands take more than half of shared memory:
     // npair > 55); SBCI_TC_PIPE=0 keeps the plain kernel, 1 takes the
     // pipelined one for every size
    const char *e = std::getenv("SBCI_TC_PIPE");
    const bool off = e && std::strcmp(e, "0") == 0, all = e && std::strcmp(e, "1") == 0;
    int Kp, Np;
    uint32_t cols;
    size_t smem = 0;
    const bool one_cta = tc_dims(c->npair, &Kp, &Np, &cols, &smem) && smem > 113 * 1024;
    if (c->tc_grid > 0 && !off && (one_cta || all)) c->tcp_grid = tcp_grid(c->npair, c->ndet, c->nsm);
  }
  {  // SBCI_FUSED=0 keeps the tile kernel + scatter for singlet-sector TF32x3 steps
    const char *e = std::getenv("SBCI_FUSED");
    c->fc_grid = (e && e[0] == '0') ? 0 : fc_grid(c->npair, c->Na, c->Nb, c->sb.nlink, c->nsm);
    if (c->fc_grid > 0) {  // (fc_dims holds J <= 255 and pair <= 127 for these spaces)
      std::vector<uint16_t> w(c->sa.links.size());
      for (size_t i = 0; i < w.size(); ++i) {
        const uint32_t v = c->sa.links[i];
        w[i] = (uint16_t)((uint32_t)link_J(v) | (uint32_t)link_pair(v) << 8 | (link_neg(v) ? 0x8000u : 0u));
      }
      TRY(up((void **)&c->d_fc_link_a, w.data(), w.size() * sizeof(uint16_t)));
    }
  }
  {
    int Kp, Np;
    uint32_t cols;
    size_t smem;
    if (tc_dims(c->npair, &Kp, &Np, &cols, &smem)) {
      TRY(cuda_ok(pool_malloc((void **)&c->d_Wtc, sizeof(uint32_t) * 2 * Np * Kp), "cudaMalloc"));
      TRY(cuda_ok(launch_split_W(c->d_W, c->npair, Kp, Np, c->d_Wtc, c->stream), "split kernel"));
    }
  }
  if (bf_W_elems(c->npair) > 0) {  // BF16x3 operand B and the kernel's launch shape
    TRY(cuda_ok(pool_malloc((void **)&c->d_Wbf, sizeof(uint16_t) * bf_W_elems(c->npair)), "cudaMalloc"));
    TRY(cuda_ok(launch_split_W_bf(c->d_W, c->npair, c->d_Wbf, c->stream), "split kernel"));
    c->bf_grid = bf_grid(c->npair, c->ndet, c->nsm);
  }
  // low-rank form of W for the FP64 SIMT contraction (lowrank.h, df_factor)
  const char *lr_mode = std::getenv("SBCI_LOWRANK");  // "0": keep the full contraction
  const bool lr_off = lr_mode && std::strcmp(lr_mode, "0") == 0;
  if (!lr_off && c->npair > 55) {
    const int np = c->npair;
    std::vector<double> V((size_t)np * np), kap(np), del(np);
    for (int i = 0, P = 0; i < n; ++i)
      for (int j = 0; j <= i; ++j, ++P) {
        kap[P] = kmat[i * n + j];
        del[P] = (i == j) ? 1.0 : 0.0;
        for (int k = 0, Q = 0; k < n; ++k)
          for (int l = 0; l <= k; ++l, ++Q) V[(size_t)P * np + Q] = E4(i, j, k, l);
      }
    std::vector<double> Ut, UL;
    const int rr = df_factor(np, V.data(), kap.data(), del.data(), N, Ut, UL);
    if (rr > 0) {
      TRY(up(&c->d_lrUt64, Ut.data(), Ut.size() * 8));
      TRY(up(&c->d_lrUL64, UL.data(), UL.size() * 8));
      c->lr_rank = rr;
      // the factored TF32x3 contraction on the tensor cores where the full
      // form's operands do not fit shared memory (n = 15) and its own do; at
      // n = 14 the full form is faster (the factor saves 14 % of the tensor
      // work of a gather-bound kernel and adds a TMEM round trip).
      // SBCI_TC_LOWRANK=1 takes the factored form wherever it fits, 0 never.
      const char *tlr = std::getenv("SBCI_TC_LOWRANK");
      c->tclr_first = tlr && std::strcmp(tlr, "1") == 0;
      const size_t words = tclr_W_words(np, rr);
      if (!(tlr && std::strcmp(tlr, "0") == 0) && words > 0) {
        const int g = tclr_grid(np, rr, c->ndet, c->nsm);
        if (g > 0) {
          TRY(cuda_ok(pool_malloc((void **)&c->d_Wtclr, sizeof(uint32_t) * words), "cudaMalloc"));
          TRY(cuda_ok(launch_split_lr_tc(static_cast<const double *>(c->d_lrUt64),
                                         static_cast<const double *>(c->d_lrUL64), rr, np, c->d_Wtclr, c->stream),
                      "split kernel"));
          c->tclr_grid = g;
        }
      }
    }
  }
  {
    // FP64 contraction on the tensor cores by exact slices where the operands
    // fit (npair <= 55); SBCI_FP64_CONTRACTION=dfma keeps the FP64 FMA kernel
    const char *mode = std::getenv("SBCI_FP64_CONTRACTION");
    const bool dfma = mode && std::strcmp(mode, "dfma") == 0;
    if (!dfma && os_supported(c->npair) && prepare_os_kernel(c->npair) == cudaSuccess) {
      TRY(cuda_ok(pool_malloc(&c->d_Wos, os_W_bytes()), "cudaMalloc"));
      TRY(cuda_ok(pool_malloc((void **)&c->d_fexp, sizeof(int) * 64), "cudaMalloc"));
      TRY(cuda_ok(launch_split_W_os(c->d_W, c->npair, c->d_Wos, c->d_fexp, c->stream), "slice kernel"));
      c->os_grid = os_grid(c->ndet, c->nsm);
    }
  }
  TRY(cuda_ok(launch_diagonal(c->d_diag, c->d_ea, c->d_eb, c->d_ja, c->d_mask_b, c->Na, c->Nb, n,
                              c->stream), "diagonal kernel"));
  TRY(cuda_ok(cudaStreamSynchronize(c->stream), "sync"));
#undef TRY
  *out = c;
  return SBCI_OK;
}

sbci_status sbci_dims(const sbci_ctx *c, long long *ndet, int *na, int *nb, int *nlink_a,
                      int *nlink_b, int *npair) {
  if (!c) {
    set_error("sbci_dims: NULL context");
    return SBCI_ERR_INVALID;
  }
  if (ndet) *ndet = c->ndet;
  if (na) *na = c->Na;
  if (nb) *nb = c->Nb;
  if (nlink_a) *nlink_a = c->sa.nlink;
  if (nlink_b) *nlink_b = c->sb.nlink;
  if (npair) *npair = c->npair;
  return SBCI_OK;
}

sbci_status sbci_string_table(const sbci_ctx *c, int spin, int *out) {
  if (!c || !out || (spin != 0 && spin != 1)) {
    set_error("sbci_string_table: bad argument");
    return SBCI_ERR_INVALID;
  }
  const StringSet &S = spin == 0 ? c->sa : c->sb;
  std::vector<uint32_t> buf((size_t)S.nstr * S.nlink);
  CK(cudaMemcpy(buf.data(), spin == 0 ? c->d_link_a : c->d_link_b, buf.size() * 4,
                cudaMemcpyDeviceToHost));
  for (size_t i = 0; i < buf.size(); ++i) {
    out[3 * i + 0] = link_pair(buf[i]);
    out[3 * i + 1] = link_J(buf[i]);
    out[3 * i + 2] = link_neg(buf[i]) ? -1 : 1;
  }
  return SBCI_OK;
}

sbci_status sbci_diagonal(sbci_ctx *c, double *out, int on_device) {
  if (!c || !out) {
    set_error("sbci_diagonal: NULL argument");
    return SBCI_ERR_INVALID;
  }
  CK(cudaMemcpyAsync(out, c->d_diag, sizeof(double) * c->ndet,
                     on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  return SBCI_OK;
}

sbci_status sbci_sigma(sbci_ctx *c, const double *in, double *out, int nvec, int prec, int on_device) {
  if (!c || !in || !out || nvec < 0) {
    set_error("sbci_sigma: bad argument");
    return SBCI_ERR_INVALID;
  }
  RET(check_prec(c, prec));
  const size_t n = (size_t)c->ndet;
  if (!on_device) {
    RET(check_finite(in, n * nvec, "c"));
    if (c->tmp_elems < n) {
      if (c->d_tmp_in) CK(cudaStreamSynchronize(c->stream));
      if (c->d_tmp_in) pool_free(c->d_tmp_in);
      if (c->d_tmp_out) pool_free(c->d_tmp_out);
      c->d_tmp_in = c->d_tmp_out = nullptr;
      c->tmp_elems = 0;
      RET(dmalloc(&c->d_tmp_in, n));
      RET(dmalloc(&c->d_tmp_out, n));
      c->tmp_elems = n;
    }
  }
  for (int v = 0; v < nvec; ++v) {
    const double *src = in + v * n;
    double *dst = out + v * n;
    if (!on_device) {
      CK(cudaMemcpyAsync(c->d_tmp_in, src, n * 8, cudaMemcpyHostToDevice, c->stream));
      RET(run_sigma(c, c->d_tmp_in, c->d_tmp_out, prec));
      CK(cudaMemcpyAsync(dst, c->d_tmp_out, n * 8, cudaMemcpyDeviceToHost, c->stream));
    } else {
      RET(run_sigma(c, src, dst, prec));
    }
  }
  CK(cudaMemcpyAsync(c->h_status, c->d_status, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  if (*c->h_status != 0) {
    set_error("a bounded device wait ran out (tensor-core MMA completion)");
    return SBCI_ERR_TIMEOUT;
  }
  return SBCI_OK;
}

sbci_status sbci_begin(sbci_ctx *c, int k, const sbci_params *params, const double *c0) {
  if (c && params && params->init == 1 && !c0) {
    set_error("init = 1 needs c0");
    return SBCI_ERR_INVALID;
  }
  RET(begin_common(c, k, params, "sbci_begin"));
  Solver &s = c->s;
  double E0 = 0.0;
  if (s.p.init == 1) RET(init_from_vector(c, c0, &E0));
  else RET(initial_guess(c, k, &E0));
  if (s.p.start_noise > 0.0) {
    RET(mix_noise(c, 0, &E0));
    RET(gen_dots(c, {s.x}, {s.x}));  // x0 must be a unit vector
    const double nx = std::sqrt(c->h_result[S_GEN0]);
    RET(lincomb(c, s.x, {s.x}, {1.0 / nx}));
    RET(lincomb(c, s.X, {s.X}, {1.0 / nx}));
  }
  return start_state(c, 0, E0);
}


sbci_status sbci_step(sbci_ctx *c, sbci_trace_record *rec, int *done) {
  if (!c || !c->s.active) {
    set_error("sbci_step: no active solve (call sbci_begin)");
    return SBCI_ERR_INVALID;
  }
  Solver &s = c->s;
  if (done) *done = s.done ? 1 : 0;
  if (s.done) return SBCI_OK;
  const size_t n0 = s.trace.size();
  sbci_status ret = SBCI_OK;
  // bodies until one SB step has been recorded (the first body after a
  // (re)start only prepares the first subspace solve)
  for (int guard = 0; guard < 4 && s.trace.size() == n0 && !s.done; ++guard) {
    RET(launch_body(c, s.h_ctl->prec, 0, true));
    RET(ctl_read(c));
    if (s.h_ctl->halt) {
      ret = handle_halt(c);
      if (ret != SBCI_OK && ret != SBCI_ERR_NOT_CONVERGED) return ret;
    }
  }
  if (rec && s.trace.size() > n0) *rec = s.trace.back();
  if (done) *done = s.done ? 1 : 0;
  return ret;
}

sbci_status sbci_finish(sbci_ctx *c, double *energies, double *vecs, sbci_report *rep) {
  if (!c || !c->s.active) {
    set_error("sbci_finish: no active solve");
    return SBCI_ERR_INVALID;
  }
  Solver &s = c->s;
  const int nst = (int)s.Ec.size();
  for (int i = 0; i < nst; ++i) {
    if (energies) energies[i] = s.Ec[i] + c->e_core;
    if (rep) rep[i] = s.rep[i];
  }
  if (vecs && nst > 0)
    CK(cudaMemcpyAsync(vecs, s.xc, sizeof(double) * (size_t)nst * c->ndet, cudaMemcpyDeviceToHost,
                       c->stream));
  CK(cudaStreamSynchronize(c->stream));
  if (nst < s.k) {
    set_error("sbci_finish: solve not finished");
    return SBCI_ERR_INVALID;
  }
  return s.any_unconverged ? SBCI_ERR_NOT_CONVERGED : SBCI_OK;
}

sbci_status sbci_solve(sbci_ctx *c, int k, const sbci_params *params, const double *c0,
                       double *energies, double *vecs, sbci_report *rep) {
  RET(sbci_begin(c, k, params, c0));
  Solver &s = c->s;
  while (!s.done) {
    RET(run_until_halt(c));
    const sbci_status st = handle_halt(c);
    if (st != SBCI_OK && st != SBCI_ERR_NOT_CONVERGED) return st;
  }
  return sbci_finish(c, energies, vecs, rep);
}

sbci_status sbci_solve_sbci2(sbci_ctx *c, int k, const sbci_params *params, int max_cycle2, double *energies,
                             double *vecs, sbci_report *rep) {
  if (params && (params->prec != SBCI_FP64 || params->init != 0 || params->start_noise > 0.0)) {
    set_error("sbci_solve_sbci2: needs prec = SBCI_FP64, init = 0 and start_noise = 0");
    return SBCI_ERR_INVALID;
  }
  if (max_cycle2 < 0) {
    set_error("sbci_solve_sbci2: max_cycle2 must be >= 0");
    return SBCI_ERR_INVALID;
  }
  RET(begin_common(c, k, params, "sbci_solve_sbci2"));
  const sbci_status st = sbci2_run(c, k, max_cycle2 > 0 ? max_cycle2 : 10);
  if (st != SBCI_OK) {
    c->s.active = false;
    return st;
  }
  return sbci_finish(c, energies, vecs, rep);
}

sbci_status sbci_davidson(sbci_ctx *c, int k, const sbci_params *params, int max_space, double *energies,
                          double *vecs, sbci_report *rep, long long *vector_bytes) {
  if (!c || k < 1 || k > kMaxStates || !energies) {
    set_error("sbci_davidson: need a context, 1 <= k <= 8 and energies");
    return SBCI_ERR_INVALID;
  }
  sbci_params p;
  if (params) p = *params;
  else sbci_params_init(&p);
  if (max_space == 0) max_space = std::max(12, 4 * k);
  if (max_space < 2 * k || max_space > kDavMaxSpace) {
    set_error("sbci_davidson: need 2k <= max_space <= 64");
    return SBCI_ERR_INVALID;
  }
  if (p.sector && c->ne_a != c->ne_b) {
    set_error("sector = 1 needs nalpha == nbeta");
    return SBCI_ERR_INVALID;
  }
  if ((long long)k > c->ndet) {
    set_error("sbci_davidson: more states than determinants");
    return SBCI_ERR_INVALID;
  }
  RET(ensure_G(c, SBCI_FP64));
  return davidson_run(c, k, p, max_space, energies, vecs, rep, vector_bytes);
}

sbci_status sbci_trace(const sbci_ctx *c, sbci_trace_record *buf, int cap, int *n) {
  if (!c) {
    set_error("sbci_trace: NULL context");
    return SBCI_ERR_INVALID;
  }
  const int m = (int)c->s.trace.size();
  if (n) *n = m;
  if (buf)
    for (int i = 0; i < m && i < cap; ++i) buf[i] = c->s.trace[i];
  return SBCI_OK;
}

sbci_status sbci_profile(sbci_ctx *c, int enable) {
  if (!c) {
    set_error("sbci_profile: NULL context");
    return SBCI_ERR_INVALID;
  }
  RET(prof_flush(c));
  Prof &p = c->prof;
  for (int i = 0; i < K_COUNT; ++i) {
    p.launches[i] = 0;
    p.ms[i] = 0.0;
  }
  p.on = enable != 0;
  return SBCI_OK;
}

sbci_status sbci_profile_read(sbci_ctx *c, sbci_kernel_stat *out, int cap, int *n) {
  if (!c) {
    set_error("sbci_profile_read: NULL context");
    return SBCI_ERR_INVALID;
  }
  RET(prof_flush(c));
  if (n) *n = K_COUNT;
  for (int i = 0; i < K_COUNT && out && i < cap; ++i) {
    std::memset(out[i].name, 0, sizeof(out[i].name));
    std::strncpy(out[i].name, kKidName[i], sizeof(out[i].name) - 1);
    out[i].launches = c->prof.launches[i];
    out[i].total_ms = c->prof.ms[i];
  }
  return SBCI_OK;
}

}  // extern "C"
