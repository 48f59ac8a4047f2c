// Serving layer: continuous batching of SBCI solves on one GPU.
//
// Requests (an active space, k states, parameters) wait in a FIFO queue and
// are admitted into slots while a slot is free and the device-memory
// footprint of the request fits the budget.  Each admitted solve keeps its
// vectors, excitation tables and controller state resident on the GPU and
// runs its SB steps as a CUDA-graph loop on its own stream, so solves that
// arrive while others are running overlap on the device.  sbci_server_progress
// is non-blocking: it admits what fits, and for every slot whose stream has
// reached the end of its graph round it handles the controller event (state
// converged, stage switch, cap) and launches the next round, or retires the
// finished solve and frees its slot and memory.
//
// Batched mode (the default): solves that can share the batched persistent
// kernels (TF32x3 sigma, n <= 12) do not get a graph each; the server keeps a
// device job table of them and runs ONE graph while-loop whose four step
// kernels walk the table as a work queue, so a single launch of each kernel
// advances every batched solve.  The loop ends when any solve's controller
// halts; the server then acts on those solves, rebuilds the table (new
// arrivals join, finished solves leave) and launches the next round.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cstdlib>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/sbci.h"
#include "batch.h"
#include "host_pool.h"
#include "sbci_internal.h"

using namespace sbci;

namespace {

double now_s() {
  using namespace std::chrono;
  return duration<double>(steady_clock::now().time_since_epoch()).count();
}

struct Request {
  long long ticket = 0;
  int norb = 0, nalpha = 0, nbeta = 0, k = 1;
  std::vector<double> h1, eri;
  double e_core = 0.0;
  sbci_params p{};
  double t_submit = 0.0;
  size_t bytes = 0;
};

struct SolveSlot {
  bool used = false;
  Request req;
  sbci_ctx *ctx = nullptr;
  cudaEvent_t ev = nullptr;
  bool in_flight = false;
  bool batched = false;  // advanced by the batch graph instead of its own graph
  bool host_pending = false;  // halted: its host work runs while the next round computes
  double t_admit = 0.0;
};

// Online autotuner of the batched kernels' launch shapes (CTAs per kernel),
// one per operand class.  The first bodies of a class run one kernel at a
// time bracketed by CUDA events, each kernel with the next of its candidate
// CTA counts; once every candidate has kTuneSamples timings, the one with the
// lowest median is kept for each kernel and the class's graph is built with
// it.  CTA counts never change a solve's arithmetic (its virtual blocks and
// tiles are fixed by the solve), so tuning changes timing only.
constexpr int kTuneSamples = 3;

struct ClassGraph {
  BatchConfig cfg{};
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  bool tuned = false;
  std::vector<int> cand[BK_COUNT];
  std::vector<std::vector<float>> ms[BK_COUNT];
  long long tune_bodies = 0;
};

void tune_init(ClassGraph &g, int nsm) {
  g.cand[BK_UPDATE] = {nsm, 2 * nsm, 4 * nsm};
  g.cand[BK_PROJECT] = {nsm, 2 * nsm, 4 * nsm, 8 * nsm};
  for (int k = 1; k <= g.cfg.tc_per_sm_max; ++k) g.cand[BK_TC].push_back(k * nsm);
  for (int k = 1; k <= g.cfg.fc_per_sm_max; ++k) g.cand[BK_FUSED].push_back(k * nsm);
  g.cand[BK_SCATTER] = {nsm, 2 * nsm, 3 * nsm, 6 * nsm};
  g.cand[BK_SYMFIN] = {nsm, 2 * nsm, 4 * nsm};
  g.cand[BK_END] = {1};
  for (int k = 0; k < BK_COUNT; ++k) {
    if (!(g.cfg.mask & (1u << k))) g.cand[k] = {g.cfg.ctas[k]};  // not launched in this class
    g.ms[k].assign(g.cand[k].size(), std::vector<float>());
  }
}

bool launched(const ClassGraph &g, int k) { return (g.cfg.mask & (1u << k)) != 0; }

bool tune_complete(const ClassGraph &g) {
  for (int k = 0; k < BK_COUNT; ++k)
    if (launched(g, k))
      for (const auto &v : g.ms[k])
        if ((int)v.size() < kTuneSamples) return false;
  return true;
}

void tune_choose(ClassGraph &g) {
  for (int k = 0; k < BK_COUNT; ++k) {
    if (!launched(g, k)) continue;
    int best = 0;
    float best_t = 0.f;
    for (size_t c = 0; c < g.cand[k].size(); ++c) {
      std::vector<float> v = g.ms[k][c];
      std::sort(v.begin(), v.end());
      const float med = v[v.size() / 2];
      if (c == 0 || med < best_t) {
        best = (int)c;
        best_t = med;
      }
    }
    g.cfg.ctas[k] = g.cand[k][best];
  }
  g.tuned = true;
}

// Kernels per loop body of a class.
int body_kernels(const ClassGraph &g) {
  int n = 0;
  for (int k = 0; k < BK_COUNT; ++k) n += launched(g, k) ? 1 : 0;
  return n;
}

// Event timing of single launches (kernel timing and tuning).
struct KernelStats {
  bool on = false;
  long long launches[BK_COUNT] = {};
  double ms[BK_COUNT] = {};
  long long host_events = 0;  // halted solves handled between rounds
  double host_ms = 0.0;       // host wall time of that handling
};

struct GraphCache {
  std::map<std::vector<int>, ClassGraph> m;
  cudaEvent_t ev[2 * BK_COUNT] = {};
  int *h_stop = nullptr;  // pinned
  ClassGraph *get(const BatchClass &k, int nsm) {
    const std::vector<int> key = {k.Kp, k.Np, k.fKp, k.fNp, (int)k.mask};
    auto it = m.find(key);
    if (it != m.end()) return &it->second;
    ClassGraph g;
    if (batch_config(nsm, k, &g.cfg) != cudaSuccess) return nullptr;
    tune_init(g, nsm);
    return &(m[key] = g);
  }
  void destroy() {
    for (auto &kv : m) {
      if (kv.second.exec) cudaGraphExecDestroy(kv.second.exec);
      if (kv.second.graph) cudaGraphDestroy(kv.second.graph);
    }
    m.clear();
    for (cudaEvent_t &e : ev)
      if (e) cudaEventDestroy(e), e = nullptr;
    if (h_stop) cudaFreeHost(h_stop);
    h_stop = nullptr;
  }
};

// One batch round of class cg on stream s: the class's graph loop once it is
// tuned (unless kernel timing is on or SBCI_NO_GRAPH=1, for profilers that do
// not follow graph loops); otherwise the same bodies launched kernel by
// kernel, each bracketed by events, until a body ends with a halted solve.
cudaError_t run_round(GraphCache &gc, ClassGraph &cg, BatchTable *d_table, int *d_status, cudaStream_t s,
                      KernelStats *stats) {
  const char *env = std::getenv("SBCI_NO_GRAPH");
  const bool no_graph = env && env[0] == '1';
  const bool timing = stats && stats->on;
  cudaError_t e = cudaSuccess;
  if (cg.tuned && !cg.exec && (e = build_batch_graph(cg.cfg, d_table, d_status, s, &cg.graph, &cg.exec)) != cudaSuccess)
    return e;
  if (cg.tuned && !timing && !no_graph) return cudaGraphLaunch(cg.exec, s);
  for (cudaEvent_t &x : gc.ev)
    if (!x && (e = cudaEventCreate(&x)) != cudaSuccess) return e;
  if (!gc.h_stop && (e = cudaMallocHost((void **)&gc.h_stop, sizeof(int))) != cudaSuccess) return e;
  for (;;) {
    BatchConfig cfg = cg.cfg;
    int ci[BK_COUNT];
    for (int k = 0; k < BK_COUNT; ++k) {
      ci[k] = cg.tuned ? -1 : (int)(cg.tune_bodies % (long long)cg.cand[k].size());
      if (ci[k] >= 0) cfg.ctas[k] = cg.cand[k][ci[k]];
    }
    for (int k = 0; k < BK_COUNT; ++k) {
      if (!launched(cg, k)) continue;
      if ((e = cudaEventRecord(gc.ev[2 * k], s)) != cudaSuccess) return e;
      if ((e = launch_batch_kernel(k, cfg, d_table, d_status, 0ull, s)) != cudaSuccess) return e;
      if ((e = cudaEventRecord(gc.ev[2 * k + 1], s)) != cudaSuccess) return e;
    }
    if ((e = cudaMemcpyAsync(gc.h_stop, &d_table->stop, sizeof(int), cudaMemcpyDeviceToHost, s)) != cudaSuccess ||
        (e = cudaStreamSynchronize(s)) != cudaSuccess)
      return e;
    for (int k = 0; k < BK_COUNT; ++k) {
      if (!launched(cg, k)) continue;
      float t = 0.f;
      if ((e = cudaEventElapsedTime(&t, gc.ev[2 * k], gc.ev[2 * k + 1])) != cudaSuccess) return e;
      if (ci[k] >= 0) cg.ms[k][ci[k]].push_back(t);
      if (timing) {
        stats->launches[k] += 1;
        stats->ms[k] += t;
      }
    }
    if (!cg.tuned) {
      cg.tune_bodies += 1;
      if (tune_complete(cg)) tune_choose(cg);
    }
    if (*gc.h_stop) return cudaSuccess;
  }
}

}  // namespace

// Operand class of a table: the largest Kp and Np of its tile-kernel jobs and
// of its column-kernel jobs, and the kernels its jobs need.
BatchClass sbci::table_class(const BatchTable &t) {
  BatchClass k{8, 16, 8, 16, 0u};
  for (int j = 0; j < t.njobs; ++j) {
    const BatchJob &b = t.job[j];
    if (b.fused) {
      k.mask |= 1u << BK_FUSED;
      k.fKp = std::max(k.fKp, b.Kp);
      k.fNp = std::max(k.fNp, b.Np);
    } else {
      k.mask |= (1u << BK_TC) | (1u << BK_SCATTER);
      k.Kp = std::max(k.Kp, b.Kp);
      k.Np = std::max(k.Np, b.Np);
    }
    if (b.sig.symA) k.mask |= 1u << BK_SYMFIN;
  }
  return k;
}

namespace {

struct Result {
  int done = 0;
  sbci_status status = SBCI_OK;
  std::vector<double> energies;
  std::vector<sbci_report> rep;
  double t_submit = 0.0, t_admit = 0.0, t_done = 0.0;
  std::string error;  // the library's message when status is an error
};

}  // namespace

struct sbci_server {
  size_t budget = 0, used = 0;
  int max_slots = 1;
  int mode = 1;  // 1: batched persistent kernels for eligible solves; 0: a graph per solve
  std::deque<Request> queue;
  std::vector<SolveSlot> slots;
  std::map<long long, Result> results;
  long long next_ticket = 1;
  // batch engine
  cudaStream_t stream = nullptr;
  cudaEvent_t batch_ev = nullptr;
  BatchTable *d_table = nullptr, *h_table = nullptr;
  int *d_status = nullptr;
  GraphCache graphs;
  bool batch_ok = false;  // the batch engine could be set up
  bool batch_in_flight = false;
  std::vector<int> batch_slots;  // table row -> slot index
  int nsm = 1;
};

namespace {

sbci_status retire(sbci_server *sv, SolveSlot &sl, sbci_status st) {
  Result &r = sv->results[sl.req.ticket];
  r.status = st;
  if (st != SBCI_OK) r.error = sbci_last_error();
  r.energies.assign(sl.req.k, 0.0);
  r.rep.assign(sl.req.k, sbci_report{});
  if (st == SBCI_OK || st == SBCI_ERR_NOT_CONVERGED) {
    const sbci_status fs = sbci_finish(sl.ctx, r.energies.data(), nullptr, r.rep.data());
    if (fs != SBCI_OK && fs != SBCI_ERR_NOT_CONVERGED) r.status = fs;
  }
  r.done = 1;
  r.t_done = now_s();
  sbci_destroy(sl.ctx);
  sl.ctx = nullptr;
  sl.used = false;
  sl.in_flight = false;
  sv->used -= sl.req.bytes;
  sl.req = Request{};
  return SBCI_OK;
}

sbci_status launch_round(SolveSlot &sl) {
  sbci_status st = solve_round_launch(sl.ctx);
  if (st != SBCI_OK) return st;
  if (cudaEventRecord(sl.ev, ctx_stream(sl.ctx)) != cudaSuccess) {
    set_error("server: cudaEventRecord failed");
    return SBCI_ERR_CUDA;
  }
  sl.in_flight = true;
  return SBCI_OK;
}

// Admits queued requests while a slot and the memory budget allow.
sbci_status admit(sbci_server *sv) {
  while (!sv->queue.empty()) {
    Request &q = sv->queue.front();
    if (sv->used + q.bytes > sv->budget) break;
    int free_slot = -1;
    for (int i = 0; i < (int)sv->slots.size(); ++i)
      if (!sv->slots[i].used) {
        free_slot = i;
        break;
      }
    if (free_slot < 0) break;
    SolveSlot &sl = sv->slots[free_slot];
    sl.req = std::move(q);
    sv->queue.pop_front();
    sl.used = true;
    sl.t_admit = now_s();
    sv->results[sl.req.ticket].t_admit = sl.t_admit;
    sv->used += sl.req.bytes;
    sbci_status st = sbci_init_integrals(&sl.ctx, sl.req.norb, sl.req.nalpha, sl.req.nbeta,
                                         sl.req.h1.data(), sl.req.eri.data(), sl.req.e_core, nullptr);
    if (st == SBCI_OK) st = sbci_begin(sl.ctx, sl.req.k, &sl.req.p, nullptr);
    if (st == SBCI_OK) {
      BatchJob probe;
      sl.batched = sv->mode == 1 && sv->batch_ok && ctx_batch_job(sl.ctx, &probe);
      if (!sl.batched) st = launch_round(sl);
    }
    if (st != SBCI_OK) {
      if (sl.ctx) {
        retire(sv, sl, st);
      } else {
        Result &r = sv->results[sl.req.ticket];
        r.status = st;
        r.done = 1;
        r.t_done = now_s();
        sv->used -= sl.req.bytes;
        sl.used = false;
        sl.req = Request{};
      }
    }
  }
  return SBCI_OK;
}

}  // namespace

namespace {

// Work-item offsets of job nj (just filled by ctx_batch_job) in every kernel
// of the body: a column-fused job has columns and no tiles or scatter blocks.
void table_offsets(BatchTable &t, int nj, const sbci_ctx *c) {
  const BatchJob &b = t.job[nj];
  t.off_step[nj + 1] = t.off_step[nj] + ctx_step_blocks(c);
  t.off_sc[nj + 1] = t.off_sc[nj] + (b.fused ? 0 : ctx_scatter_blocks(c));
  t.off_tc[nj + 1] = t.off_tc[nj] + (b.fused ? 0 : (int)((ctx_ndet(c) + 127) / 128));
  t.off_fc[nj + 1] = t.off_fc[nj] + (b.fused ? b.sig.nb : 0);
  t.off_sf[nj + 1] = t.off_sf[nj] + ctx_symfin_blocks(c);
}

// Rebuilds the job table from the batched slots and launches one round.
sbci_status launch_batch_round(sbci_server *sv) {
  BatchTable &t = *sv->h_table;
  sv->batch_slots.clear();
  int nj = 0;
  t.off_step[0] = t.off_sc[0] = t.off_tc[0] = t.off_sf[0] = t.off_fc[0] = 0;
  for (int i = 0; i < (int)sv->slots.size(); ++i) {
    SolveSlot &sl = sv->slots[i];
    if (!sl.used || !sl.batched || sl.host_pending || nj >= kMaxBatch) continue;
    if (!ctx_batch_job(sl.ctx, &t.job[nj])) {
      // no longer batchable (its state fell back to FP64 sigma): own graph loop from now on
      sl.batched = false;
      const sbci_status st = launch_round(sl);
      if (st != SBCI_OK) retire(sv, sl, st);
      continue;
    }
    table_offsets(t, nj, sl.ctx);
    if (ctx_fence(sl.ctx, sv->stream) != cudaSuccess) {
      set_error("server: stream ordering failed");
      return SBCI_ERR_CUDA;
    }
    t.halted[nj] = 0;
    sv->batch_slots.push_back(i);
    ++nj;
  }
  t.njobs = nj;
  t.tc_next = 0;
  if (nj == 0) return SBCI_OK;
  ClassGraph *cg = sv->graphs.get(table_class(t), sv->nsm);
  if (!cg) {
    set_error("server: no batch configuration for this operand class");
    return SBCI_ERR_CUDA;
  }
  // (a round of a class still being tuned runs host-driven and returns when done)
  if (cudaMemcpyAsync(sv->d_table, sv->h_table, sizeof(BatchTable), cudaMemcpyHostToDevice, sv->stream) !=
          cudaSuccess ||
      run_round(sv->graphs, *cg, sv->d_table, sv->d_status, sv->stream, nullptr) != cudaSuccess ||
      cudaEventRecord(sv->batch_ev, sv->stream) != cudaSuccess) {
    set_error("server: batch launch failed");
    return SBCI_ERR_CUDA;
  }
  sv->batch_in_flight = true;
  return SBCI_OK;
}

// After a batch round: act on every halted solve, then launch the next round.
sbci_status progress_batch(sbci_server *sv) {
  if (sv->batch_in_flight) {
    const cudaError_t q = cudaEventQuery(sv->batch_ev);
    if (q == cudaErrorNotReady) return SBCI_OK;
    sv->batch_in_flight = false;
    if (q != cudaSuccess) {
      set_error(std::string("server: ") + cudaGetErrorString(q));
      return SBCI_ERR_CUDA;
    }
    int status = 0;
    if (cudaMemcpy(&status, sv->d_status, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess ||
        cudaMemcpy(sv->h_table->halted, sv->d_table->halted, sizeof(int) * kMaxBatch,
                   cudaMemcpyDeviceToHost) != cudaSuccess) {
      set_error("server: reading the batch table failed");
      return SBCI_ERR_CUDA;
    }
    if (status) {
      set_error("a bounded device wait ran out (batched tensor-core kernel)");
      return SBCI_ERR_TIMEOUT;
    }
    // the halted solves sit out one round: the round of the others is launched
    // first, and their host work (FP64 re-syncs, verification, next state)
    // runs on their own streams while it computes
    std::vector<int> halted;
    for (int j = 0; j < (int)sv->batch_slots.size(); ++j)
      if (sv->h_table->halted[j]) {
        halted.push_back(sv->batch_slots[j]);
        sv->slots[sv->batch_slots[j]].host_pending = true;
      }
    sbci_status lst = launch_batch_round(sv);
    // their host work in parallel (each solve on its own stream), then the
    // retirements in slot order on this thread
    const int nh = (int)halted.size();
    std::vector<sbci_status> hs(nh, SBCI_OK);
    std::vector<int> hd(nh, 0);
    std::vector<std::string> hm(nh);
    host_parallel_for(nh, [&](int q) {
      SolveSlot &sl = sv->slots[halted[q]];
      cudaSetDevice(ctx_device(sl.ctx));
      hs[q] = solve_round_finish(sl.ctx, &hd[q], false);
      if (hs[q] != SBCI_OK && hs[q] != SBCI_ERR_NOT_CONVERGED) hm[q] = last_error();
    });
    for (int q = 0; q < nh; ++q) {
      SolveSlot &sl = sv->slots[halted[q]];
      sl.host_pending = false;
      if (hs[q] != SBCI_OK && hs[q] != SBCI_ERR_NOT_CONVERGED) {
        set_error(hm[q]);
        retire(sv, sl, hs[q]);
        continue;
      }
      if (hd[q]) retire(sv, sl, SBCI_OK);
    }
    if (lst != SBCI_OK) return lst;
    if (!sv->batch_in_flight) return launch_batch_round(sv);  // every solve had halted
    return SBCI_OK;
  }
  return launch_batch_round(sv);
}

// The batch engine of sbci_solve_batch: one per device, made on first use and
// kept (stream, job table, per-class graphs and tuning), so that a call pays
// no set-up; calls on one device are serialised by its mutex.
struct Engine {
  std::mutex mu;
  bool ready = false;
  int nsm = 1;
  cudaStream_t stream = nullptr;
  BatchTable *d_table = nullptr, *h_table = nullptr;
  int *d_status = nullptr;
  GraphCache graphs;
  KernelStats prof;  // sbci_batch_profile
};

constexpr int kMaxDevices = 64;
Engine g_engines[kMaxDevices];
const char *const kBatchKernelName[BK_COUNT] = {"batch_update", "batch_project", "batch_gather_contract_tc",
                                                "batch_fused_column", "batch_scatter", "batch_symfinish",
                                                "batch_end"};

cudaError_t engine_setup(Engine &eng, int dev) {
  if (eng.ready) return cudaSuccess;
  cudaError_t e = cudaDeviceGetAttribute(&eng.nsm, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess && !eng.stream) e = cudaStreamCreateWithFlags(&eng.stream, cudaStreamNonBlocking);
  if (e == cudaSuccess && !eng.d_table) e = cudaMalloc((void **)&eng.d_table, sizeof(BatchTable));
  if (e == cudaSuccess && !eng.h_table) e = cudaMallocHost((void **)&eng.h_table, sizeof(BatchTable));
  if (e == cudaSuccess && !eng.d_status) e = cudaMalloc((void **)&eng.d_status, sizeof(int));
  if (e == cudaSuccess) e = cudaMemset(eng.d_status, 0, sizeof(int));
  eng.ready = e == cudaSuccess;
  return e;
}

cudaError_t engine_round(Engine &eng, int *kernels_per_body) {
  ClassGraph *cg = eng.graphs.get(table_class(*eng.h_table), eng.nsm);
  if (!cg) return cudaErrorInvalidValue;
  *kernels_per_body = body_kernels(*cg);
  return run_round(eng.graphs, *cg, eng.d_table, eng.d_status, eng.stream, &eng.prof);
}

Engine *current_engine(std::string *why) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    *why = "no usable CUDA device";
    return nullptr;
  }
  return &g_engines[dev];
}

}  // namespace

extern "C" {

sbci_status sbci_solve_batch(sbci_ctx **ctx, int n, int k, const sbci_params *params, double *energies,
                             sbci_report *rep, long long *launches) {
  if (!ctx || n < 1 || n > kMaxBatch || k < 1 || !energies) {
    set_error("sbci_solve_batch: need 1 <= n <= 64 contexts, k >= 1 and energies");
    return SBCI_ERR_INVALID;
  }
  std::string why;
  Engine *pe = current_engine(&why);
  int dev = 0;
  if (!pe || cudaGetDevice(&dev) != cudaSuccess) {
    set_error("sbci_solve_batch: " + why);
    return SBCI_ERR_CUDA;
  }
  Engine &eng = *pe;
  std::lock_guard<std::mutex> lock(eng.mu);
  if (engine_setup(eng, dev) != cudaSuccess) {
    set_error("sbci_solve_batch: CUDA set-up failed");
    return SBCI_ERR_CUDA;
  }
  std::vector<int> done(n, 0);
  long long host_launches0 = 0;
  for (int i = 0; i < n; ++i) host_launches0 += ctx_launch_count(ctx[i]);
  {  // the solves' initial guesses in parallel (each on its own stream)
    std::vector<sbci_status> bs(n, SBCI_OK);
    std::vector<std::string> bm(n);
    host_parallel_for(n, [&](int i) {
      cudaSetDevice(ctx_device(ctx[i]));
      bs[i] = sbci_begin(ctx[i], k, params, nullptr);
      if (bs[i] != SBCI_OK) bm[i] = last_error();
    });
    for (int i = 0; i < n; ++i)
      if (bs[i] != SBCI_OK) {
        set_error(bm[i]);
        return bs[i];
      }
  }
  std::memset(eng.h_table, 0, sizeof(BatchTable));
  if (cudaMemsetAsync(eng.d_status, 0, sizeof(int), eng.stream) != cudaSuccess) {
    set_error("sbci_solve_batch: CUDA set-up failed");
    return SBCI_ERR_CUDA;
  }
  unsigned long long bodies = 0;  // kernels the batch rounds launched (bodies x kernels per body)
  sbci_status worst = SBCI_OK;
  // a solve that halted sits out the next round: that round is launched first
  // and the solve's host work (FP64 re-syncs, verification, next state) runs on
  // its own stream while the others compute
  std::vector<int> pending;
  std::vector<char> is_pending(n, 0);
  for (;;) {
    BatchTable &t = *eng.h_table;
    std::vector<int> row;
    int nj = 0;
    t.off_step[0] = t.off_sc[0] = t.off_tc[0] = t.off_sf[0] = t.off_fc[0] = 0;
    for (int i = 0; i < n; ++i) {
      if (done[i] || is_pending[i]) continue;
      if (!ctx_batch_job(ctx[i], &t.job[nj])) {  // not batchable: solve it on its own
        double *E = energies + (size_t)i * k;
        sbci_status st = SBCI_OK;
        while (!done[i]) {
          st = solve_round_launch(ctx[i]);
          if (st != SBCI_OK) return st;
          st = solve_round_finish(ctx[i], &done[i]);
          if (st != SBCI_OK && st != SBCI_ERR_NOT_CONVERGED) return st;
        }
        st = sbci_finish(ctx[i], E, nullptr, rep ? rep + (size_t)i * k : nullptr);
        if (st != SBCI_OK) worst = st;
        continue;
      }
      table_offsets(t, nj, ctx[i]);
      if (ctx_fence(ctx[i], eng.stream) != cudaSuccess) {
        set_error("sbci_solve_batch: stream ordering failed");
        return SBCI_ERR_CUDA;
      }
      t.halted[nj] = 0;
      row.push_back(i);
      ++nj;
    }
    if (nj == 0 && pending.empty()) break;
    t.njobs = nj;
    t.tc_next = 0;
    t.bodies = 0;
    int status = 0;
    unsigned long long round_bodies = 0;
    int per_body = 0;
    if (nj > 0 &&
        (cudaMemcpyAsync(eng.d_table, eng.h_table, sizeof(BatchTable), cudaMemcpyHostToDevice, eng.stream) !=
             cudaSuccess ||
         engine_round(eng, &per_body) != cudaSuccess ||
         cudaMemcpyAsync(t.halted, eng.d_table->halted, sizeof(int) * kMaxBatch, cudaMemcpyDeviceToHost,
                         eng.stream) != cudaSuccess ||
         cudaMemcpyAsync(&status, eng.d_status, sizeof(int), cudaMemcpyDeviceToHost, eng.stream) != cudaSuccess ||
         cudaMemcpyAsync(&round_bodies, &eng.d_table->bodies, sizeof(round_bodies), cudaMemcpyDeviceToHost,
                         eng.stream) != cudaSuccess)) {
      cudaStreamSynchronize(eng.stream);
      set_error("sbci_solve_batch: batch round failed");
      return SBCI_ERR_CUDA;
    }
    sbci_status host_st = SBCI_OK;
    const double th0 = now_s();
    const long long nhalted = (long long)pending.size();
    // the halted solves' host work (FP64 re-syncs, verification, next state)
    // in parallel: each solve on its own stream, so their launches and waits
    // overlap; statuses and messages are collected in solve order
    {
      const int np = (int)pending.size();
      std::vector<sbci_status> rs(np, SBCI_OK), fs(np, SBCI_OK);
      std::vector<std::string> rm(np), fm(np);
      host_parallel_for(np, [&](int q) {
        const int i = pending[q];
        cudaSetDevice(ctx_device(ctx[i]));
        rs[q] = solve_round_finish(ctx[i], &done[i], false);
        if (rs[q] != SBCI_OK && rs[q] != SBCI_ERR_NOT_CONVERGED) {
          rm[q] = last_error();
          return;
        }
        if (done[i]) {
          fs[q] = sbci_finish(ctx[i], energies + (size_t)i * k, nullptr, rep ? rep + (size_t)i * k : nullptr);
          if (fs[q] != SBCI_OK) fm[q] = last_error();
        }
      });
      for (int q = 0; q < np; ++q) {
        is_pending[pending[q]] = 0;
        if (rs[q] != SBCI_OK && rs[q] != SBCI_ERR_NOT_CONVERGED) {
          if (host_st == SBCI_OK) {
            host_st = rs[q];
            set_error(rm[q]);
          }
          continue;
        }
        if (fs[q] != SBCI_OK) {
          worst = fs[q];
          if (host_st == SBCI_OK) set_error(fm[q]);
        }
      }
    }
    pending.clear();
    if (eng.prof.on && nhalted > 0) {
      eng.prof.host_events += nhalted;
      eng.prof.host_ms += 1e3 * (now_s() - th0);
    }
    if (nj > 0 && cudaStreamSynchronize(eng.stream) != cudaSuccess) {
      set_error("sbci_solve_batch: batch round failed");
      return SBCI_ERR_CUDA;
    }
    if (host_st != SBCI_OK) return host_st;
    bodies += round_bodies * (unsigned long long)per_body;
    if (status) {
      set_error("a bounded device wait ran out (batched tensor-core kernel)");
      return SBCI_ERR_TIMEOUT;
    }
    for (int j = 0; j < nj; ++j) {
      if (!t.halted[j]) continue;
      pending.push_back(row[j]);
      is_pending[row[j]] = 1;
    }
  }
  if (launches) {
    long long host_launches1 = 0;
    for (int i = 0; i < n; ++i) host_launches1 += ctx_launch_count(ctx[i]);
    *launches = (long long)bodies + (host_launches1 - host_launches0);
  }
  return worst;
}

sbci_status sbci_init_integrals_many(sbci_ctx **out, int n, int norb, int nalpha, int nbeta, const double *h1,
                                     const double *eri, double e_core, void *const *cuda_streams) {
  if (!out || n < 0) {
    set_error("sbci_init_integrals_many: NULL output or n < 0");
    return SBCI_ERR_INVALID;
  }
  for (int i = 0; i < n; ++i) out[i] = nullptr;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    set_error("sbci_init_integrals_many: cudaGetDevice failed");
    return SBCI_ERR_CUDA;
  }
  std::vector<sbci_status> st(n, SBCI_OK);
  std::vector<std::string> msg(n);
  host_parallel_for(n, [&](int i) {
    cudaSetDevice(dev);
    st[i] = sbci_init_integrals(&out[i], norb, nalpha, nbeta, h1, eri, e_core,
                                cuda_streams ? cuda_streams[i] : nullptr);
    if (st[i] != SBCI_OK) msg[i] = last_error();
  });
  for (int i = 0; i < n; ++i)
    if (st[i] != SBCI_OK) {
      for (int j = 0; j < n; ++j) {
        sbci_destroy(out[j]);
        out[j] = nullptr;
      }
      set_error(msg[i]);
      return st[i];
    }
  return SBCI_OK;
}

sbci_status sbci_batch_profile(int enable) {
  std::string why;
  Engine *pe = current_engine(&why);
  if (!pe) {
    set_error("sbci_batch_profile: " + why);
    return SBCI_ERR_CUDA;
  }
  std::lock_guard<std::mutex> lock(pe->mu);
  for (int k = 0; k < BK_COUNT; ++k) {
    pe->prof.launches[k] = 0;
    pe->prof.ms[k] = 0.0;
  }
  pe->prof.host_events = 0;
  pe->prof.host_ms = 0.0;
  pe->prof.on = enable != 0;
  return SBCI_OK;
}

sbci_status sbci_batch_profile_read(sbci_kernel_stat *out, int cap, int *n) {
  std::string why;
  Engine *pe = current_engine(&why);
  if (!pe) {
    set_error("sbci_batch_profile_read: " + why);
    return SBCI_ERR_CUDA;
  }
  std::lock_guard<std::mutex> lock(pe->mu);
  if (n) *n = BK_COUNT + 1;
  for (int k = 0; k < BK_COUNT && out && k < cap; ++k) {
    std::memset(out[k].name, 0, sizeof(out[k].name));
    std::strncpy(out[k].name, kBatchKernelName[k], sizeof(out[k].name) - 1);
    out[k].launches = pe->prof.launches[k];
    out[k].total_ms = pe->prof.ms[k];
  }
  if (out && BK_COUNT < cap) {
    sbci_kernel_stat &h = out[BK_COUNT];
    std::memset(h.name, 0, sizeof(h.name));
    std::strncpy(h.name, "batch_host_halted", sizeof(h.name) - 1);
    h.launches = pe->prof.host_events;
    h.total_ms = pe->prof.host_ms;
  }
  return SBCI_OK;
}

sbci_status sbci_batch_classes(sbci_batch_class *out, int cap, int *n) {
  std::string why;
  Engine *pe = current_engine(&why);
  if (!pe) {
    set_error("sbci_batch_classes: " + why);
    return SBCI_ERR_CUDA;
  }
  std::lock_guard<std::mutex> lock(pe->mu);
  int i = 0;
  for (const auto &kv : pe->graphs.m) {
    if (out && i < cap) {
      const ClassGraph &g = kv.second;
      sbci_batch_class &r = out[i];
      r.Kp = g.cfg.Kp;
      r.Np = g.cfg.Np;
      r.smem_bytes = (int)g.cfg.smem;
      r.tc_per_sm_max = g.cfg.tc_per_sm_max;
      r.fKp = g.cfg.fKp;
      r.fNp = g.cfg.fNp;
      r.fused_smem_bytes = (int)g.cfg.fsmem;
      r.kernels = (int)g.cfg.mask;
      r.tuned = g.tuned ? 1 : 0;
      for (int k = 0; k < BK_COUNT; ++k) r.ctas[k] = g.cfg.ctas[k];
    }
    ++i;
  }
  if (n) *n = i;
  return SBCI_OK;
}

sbci_status sbci_server_create(sbci_server **out, size_t mem_budget_bytes, int max_slots) {
  if (!out || max_slots < 1 || max_slots > 1024) {
    set_error("sbci_server_create: need out and 1 <= max_slots <= 1024");
    return SBCI_ERR_INVALID;
  }
  sbci_server *sv = new sbci_server();
  sv->budget = mem_budget_bytes;
  sv->max_slots = max_slots;
  sv->slots.resize(max_slots);
  int dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sv->nsm, cudaDevAttrMultiProcessorCount, dev);
  if (cudaStreamCreateWithFlags(&sv->stream, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&sv->batch_ev, cudaEventDisableTiming) != cudaSuccess ||
      cudaMalloc((void **)&sv->d_table, sizeof(BatchTable)) != cudaSuccess ||
      cudaMallocHost((void **)&sv->h_table, sizeof(BatchTable)) != cudaSuccess ||
      cudaMalloc((void **)&sv->d_status, sizeof(int)) != cudaSuccess ||
      cudaMemset(sv->d_table, 0, sizeof(BatchTable)) != cudaSuccess ||
      cudaMemset(sv->d_status, 0, sizeof(int)) != cudaSuccess) {
    set_error("sbci_server_create: CUDA allocation failed");
    sbci_server_destroy(sv);
    return SBCI_ERR_CUDA;
  }
  std::memset(sv->h_table, 0, sizeof(BatchTable));
  // the class of the largest batchable solve: checks that the engine can be set up
  {
    int Kp, Np;
    uint32_t cols;
    size_t smem;
    sv->batch_ok = tc_dims(kBatchMaxPair, &Kp, &Np, &cols, &smem) &&
                   sv->graphs.get(BatchClass{Kp, Np, 8, 16, (1u << BK_TC) | (1u << BK_SCATTER)}, sv->nsm) != nullptr;
    // and the largest column-fused class (10 orbitals, 252 strings per spin)
    int fKp, fNp;
    if (sv->batch_ok && fc_dims(55, 252, 252, 30, &fKp, &fNp, &cols, &smem))
      sv->batch_ok = sv->graphs.get(BatchClass{8, 16, fKp, fNp, (1u << BK_FUSED) | (1u << BK_SYMFIN)}, sv->nsm) !=
                     nullptr;
  }
  if (!sv->batch_ok) {
    set_error("sbci_server_create: building the batch graph failed");
    sbci_server_destroy(sv);
    return SBCI_ERR_CUDA;
  }
  for (SolveSlot &sl : sv->slots) {
    if (cudaEventCreateWithFlags(&sl.ev, cudaEventDisableTiming) != cudaSuccess) {
      set_error("sbci_server_create: cudaEventCreate failed");
      sbci_server_destroy(sv);
      return SBCI_ERR_CUDA;
    }
  }
  *out = sv;
  return SBCI_OK;
}

sbci_status sbci_server_submit(sbci_server *sv, int norb, int nalpha, int nbeta, const double *h1,
                               const double *eri, double e_core, int k, const sbci_params *params,
                               long long *ticket) {
  if (!sv || !h1 || !eri || !ticket || k < 1 || k > 8 || norb < 1 || norb > 16) {
    set_error("sbci_server_submit: bad argument");
    return SBCI_ERR_INVALID;
  }
  Request q;
  q.ticket = sv->next_ticket++;
  q.norb = norb;
  q.nalpha = nalpha;
  q.nbeta = nbeta;
  q.k = k;
  q.h1.assign(h1, h1 + (size_t)norb * norb);
  q.eri.assign(eri, eri + (size_t)norb * norb * norb * norb);
  q.e_core = e_core;
  if (params) q.p = *params;
  else sbci_params_init(&q.p);
  q.t_submit = now_s();
  q.bytes = ctx_device_bytes(norb, nalpha, nbeta, k);
  if (q.bytes > sv->budget) {
    set_error("sbci_server_submit: the request alone exceeds the memory budget");
    return SBCI_ERR_NOMEM;
  }
  Result &r = sv->results[q.ticket];
  r.t_submit = q.t_submit;
  *ticket = q.ticket;
  sv->queue.push_back(std::move(q));
  return SBCI_OK;
}

sbci_status sbci_server_progress(sbci_server *sv, int *n_active, int *n_queued) {
  if (!sv) {
    set_error("sbci_server_progress: NULL server");
    return SBCI_ERR_INVALID;
  }
  sbci_status st = admit(sv);
  if (st != SBCI_OK) return st;
  for (SolveSlot &sl : sv->slots) {
    if (!sl.used || sl.batched || !sl.in_flight) continue;
    const cudaError_t q = cudaEventQuery(sl.ev);
    if (q == cudaErrorNotReady) continue;
    sl.in_flight = false;
    if (q != cudaSuccess) {
      set_error(std::string("server: ") + cudaGetErrorString(q));
      retire(sv, sl, SBCI_ERR_CUDA);
      continue;
    }
    int done = 0;
    st = solve_round_finish(sl.ctx, &done);
    if (st != SBCI_OK && st != SBCI_ERR_NOT_CONVERGED) {
      retire(sv, sl, st);
      continue;
    }
    if (done) {
      retire(sv, sl, SBCI_OK);
      continue;
    }
    st = launch_round(sl);
    if (st != SBCI_OK) retire(sv, sl, st);
  }
  st = admit(sv);  // slots freed above
  if (st != SBCI_OK) return st;
  if (sv->mode == 1) {
    st = progress_batch(sv);
    if (st != SBCI_OK) return st;
  }
  int act = 0;
  for (const SolveSlot &sl : sv->slots) act += sl.used ? 1 : 0;
  if (n_active) *n_active = act;
  if (n_queued) *n_queued = (int)sv->queue.size();
  return SBCI_OK;
}

sbci_status sbci_server_poll(sbci_server *sv, long long ticket, int *done, double *energies,
                             sbci_report *rep, double *times) {
  if (!sv || !done) {
    set_error("sbci_server_poll: bad argument");
    return SBCI_ERR_INVALID;
  }
  auto it = sv->results.find(ticket);
  if (it == sv->results.end()) {
    set_error("sbci_server_poll: unknown ticket");
    return SBCI_ERR_INVALID;
  }
  const Result &r = it->second;
  *done = r.done;
  if (!r.done) return SBCI_OK;
  for (size_t i = 0; i < r.energies.size(); ++i) {
    if (energies) energies[i] = r.energies[i];
    if (rep) rep[i] = r.rep[i];
  }
  if (times) {
    times[0] = r.t_admit - r.t_submit;  // queueing
    times[1] = r.t_done - r.t_submit;   // latency
  }
  if (r.status != SBCI_OK) set_error(r.error);
  return r.status;
}

sbci_status sbci_server_set_batching(sbci_server *sv, int on) {
  if (!sv) {
    set_error("sbci_server_set_batching: NULL server");
    return SBCI_ERR_INVALID;
  }
  for (const SolveSlot &sl : sv->slots)
    if (sl.used) {
      set_error("sbci_server_set_batching: only while no solve is admitted");
      return SBCI_ERR_INVALID;
    }
  sv->mode = on ? 1 : 0;
  return SBCI_OK;
}

void sbci_server_destroy(sbci_server *sv) {
  if (!sv) return;
  if (sv->stream) cudaStreamSynchronize(sv->stream);
  for (SolveSlot &sl : sv->slots) {
    if (sl.ctx) {
      cudaStreamSynchronize(ctx_stream(sl.ctx));
      sbci_destroy(sl.ctx);
    }
    if (sl.ev) cudaEventDestroy(sl.ev);
  }
  sv->graphs.destroy();
  if (sv->d_table) cudaFree(sv->d_table);
  if (sv->h_table) cudaFreeHost(sv->h_table);
  if (sv->d_status) cudaFree(sv->d_status);
  if (sv->batch_ev) cudaEventDestroy(sv->batch_ev);
  if (sv->stream) cudaStreamDestroy(sv->stream);
  delete sv;
}

}  // extern "C"
