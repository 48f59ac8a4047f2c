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
#include <cuda_runtime.h>

#include <chrono>
#include <cstring>
#include <deque>
#include <map>
#include <string>
#include <vector>

#include "../../include/sbci.h"
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
  double t_admit = 0.0;
};

struct Result {
  int done = 0;
  sbci_status status = SBCI_OK;
  std::vector<double> energies;
  std::vector<sbci_report> rep;
  double t_submit = 0.0, t_admit = 0.0, t_done = 0.0;
};

}  // namespace

struct sbci_server {
  size_t budget = 0, used = 0;
  int max_slots = 1;
  std::deque<Request> queue;
  std::vector<SolveSlot> slots;
  std::map<long long, Result> results;
  long long next_ticket = 1;
};

namespace {

sbci_status retire(sbci_server *sv, SolveSlot &sl, sbci_status st) {
  Result &r = sv->results[sl.req.ticket];
  r.status = st;
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
    if (st == SBCI_OK) st = launch_round(sl);
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

extern "C" {

sbci_status sbci_server_create(sbci_server **out, size_t mem_budget_bytes, int max_slots) {
  if (!out || max_slots < 1 || max_slots > 1024) {
    set_error("sbci_server_create: need out and 1 <= max_slots <= 1024");
    return SBCI_ERR_INVALID;
  }
  sbci_server *sv = new sbci_server();
  sv->budget = mem_budget_bytes;
  sv->max_slots = max_slots;
  sv->slots.resize(max_slots);
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
    if (!sl.used || !sl.in_flight) continue;
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
  return r.status;
}

void sbci_server_destroy(sbci_server *sv) {
  if (!sv) return;
  for (SolveSlot &sl : sv->slots) {
    if (sl.ctx) {
      cudaStreamSynchronize(ctx_stream(sl.ctx));
      sbci_destroy(sl.ctx);
    }
    if (sl.ev) cudaEventDestroy(sl.ev);
  }
  delete sv;
}

}  // extern "C"
