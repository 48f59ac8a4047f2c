// Body of the gather-form scatter of the sigma build, shared by the
// one-solve kernel and the persistent batched kernel (kernels_loop.cu, the
// only translation unit that includes this header, compiled without implicit
// multiply-add contraction, so both kernels round identically):
//   sigma[I] = sum over the links of I of sign * G[pair, J]
// with the dots of sigma against up to three vectors; in device-controlled
// mode the solve's last virtual block finishes the dots and runs the subspace
// solve (ctl.h).  Processes virtual block vb of nvb; returns true when this
// call ran the last block and the controller halted.
#pragma once

#include <cuda_runtime.h>

#include "ctl.h"
#include "devreduce.cuh"
#include "sbci_internal.h"

namespace sbci {

constexpr int kScTile = 256;  // determinants per tile of the scatter

template <typename AccT>
__device__ __forceinline__ bool scatter_body(const SigmaArgs &a, int vb, int nvb) {
  double *sig = a.sigma;
  const double *du[3] = {a.dot_u[0], a.dot_u[1], a.dot_u[2]};
  if (a.ctl) {
    if (a.ctl->halt) return false;
    sig = a.ctl->Zn;
    du[2] = a.ctl->zn;
  }
  const int tid = threadIdx.x;
  const long long ntiles = (a.ndet + kScTile - 1) / kScTile;
  const AccT *G = reinterpret_cast<const AccT *>(a.G);
  double dots[3] = {0.0, 0.0, 0.0};
  for (long long tile = vb; tile < ntiles; tile += nvb) {
    const long long I = tile * kScTile + tid;
    if (I >= a.ndet) continue;
    const int ia = (int)(I / a.nb), ib = (int)(I - (long long)ia * a.nb);
    AccT acc = (AccT)0;
    const uint32_t *la = a.link_a + (size_t)ia * a.nlink_a;
    const AccT *gcol = G + ib;
    for_links<8, AccT>(
        la, a.nlink_a, 1,
        [&](uint32_t v) { return __ldg(gcol + (size_t)link_pair(v) * a.ndet + (size_t)link_J(v) * a.nb); },
        [&](uint32_t v, AccT g) { acc += link_neg(v) ? -g : g; });
    const uint32_t *lb = a.link_bT + ib;
    const AccT *grow = G + (size_t)ia * a.nb;
    for_links<8, AccT>(
        lb, a.nlink_b, a.nb, [&](uint32_t v) { return __ldg(grow + (size_t)link_pair(v) * a.ndet + link_J(v)); },
        [&](uint32_t v, AccT g) { acc += link_neg(v) ? -g : g; });
    const double sv = (double)acc;
    sig[I] = sv;
#pragma unroll
    for (int j = 0; j < 3; ++j)
      if (du[j]) dots[j] = fma(du[j][I], sv, dots[j]);
  }
  if (!du[0] && !du[1] && !du[2]) return false;
  int slots[3];
#pragma unroll
  for (int j = 0; j < 3; ++j) slots[j] = du[j] ? a.dot_slot[j] : -1;
  block_partials<3, kScTile>(dots, slots, a.partials, nvb, vb);
  if (!a.ctl) return false;  // host mode: the host reduces the partials
  if (!last_block(a.counter, nvb)) return false;
  finish_slots(a.partials, nvb, a.dot_slot, 3, a.ctl->dots, a.counter);
  __shared__ int s_halt;
  if (threadIdx.x == 0) {
    ctl_solve(*a.ctl);
    s_halt = a.ctl->halt;
  }
  __syncthreads();
  return s_halt != 0;
}

}  // namespace sbci
