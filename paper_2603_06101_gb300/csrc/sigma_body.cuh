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
  AccT *symA = reinterpret_cast<AccT *>(a.symA);
  for (long long tile = vb; tile < ntiles; tile += nvb) {
    const long long I = tile * kScTile + tid;
    if (I >= a.ndet) continue;
    int ia, ib;
    split_det(I, a.nb, ia, ib);
    AccT acc = (AccT)0;
    const uint32_t *la = a.link_a + (size_t)ia * a.nlink_a;
    const AccT *gcol = G + ib;
    for_links<8, AccT>(
        la, a.nlink_a, 1,
        [&](uint32_t v) { return __ldg(gcol + (size_t)link_pair(v) * a.ndet + (size_t)link_J(v) * a.nb); },
        [&](uint32_t v, AccT g) { acc += link_neg(v) ? -g : g; });
    if (symA) {  // singlet sector: the beta part is the transpose of the alpha part
      symA[I] = acc;
      continue;
    }
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
  if (symA || (!du[0] && !du[1] && !du[2])) return false;
  int slots[3];
#pragma unroll
  for (int j = 0; j < 3; ++j) slots[j] = du[j] ? a.dot_slot[j] : -1;
  block_partials<3, kScTile>(dots, slots, a.partials, nvb, vb);
  if (!a.ctl) return false;  // host mode: the host reduces the partials
  if (!last_block(a.counter, nvb)) return false;
  finish_slots(a.partials, nvb, a.dot_slot, 3, a.ctl->dots, a.counter);
  return ctl_run_shadowed(a.ctl, [](CtlHead &h) { ctl_solve(h); }) != 0;
}

// Symmetric finish of a singlet-sector sigma (device-controlled mode): with
// c = c^T (and the same strings for both spins) the beta part of sigma is the
// transpose of the alpha part A, so sigma = A + A^T.  Work unit: a pair of
// 32 x 32 tiles (ti, tj), ti >= tj, of A, both read coalesced into shared
// memory; it writes the two sigma tiles (one on the diagonal), takes the dots
// of sigma against x, y and z over tile (ti, tj) (weight 2 off the diagonal:
// all four are symmetric matrices), and the last block runs the subspace
// solve.
constexpr int kSfT = 32;


template <typename AccT>
__device__ __forceinline__ bool symfin_body(const SigmaArgs &a, int vb, int nvb) {
  CtlState *ctl = a.ctl;
  if (ctl->halt) return false;
  __shared__ AccT tA[kSfT][kSfT + 1], tB[kSfT][kSfT + 1];
  const AccT *A = reinterpret_cast<const AccT *>(a.symA);
  double *sig = ctl->Zn;
  const double *du[3] = {a.dot_u[0], a.dot_u[1], ctl->zn};
  const int n = a.na, T = (n + kSfT - 1) / kSfT, units = T * (T + 1) / 2;
  const int tid = threadIdx.x;
  double dots[3] = {0.0, 0.0, 0.0};
  for (int u = vb; u < units; u += nvb) {
    int ti, tj;
    tri_unit(u, &ti, &tj);
    double ud[3] = {0.0, 0.0, 0.0};  // this unit's dots over tile (ti, tj)
    __syncthreads();  // the previous unit's readers are done
    for (int k = tid; k < kSfT * kSfT; k += blockDim.x) {
      const int r = k / kSfT, c = k - r * kSfT;
      const int i1 = ti * kSfT + r, j1 = tj * kSfT + c, i2 = tj * kSfT + r, j2 = ti * kSfT + c;
      tA[r][c] = (i1 < n && j1 < n) ? A[(size_t)i1 * n + j1] : (AccT)0;
      tB[r][c] = (i2 < n && j2 < n) ? A[(size_t)i2 * n + j2] : (AccT)0;
    }
    __syncthreads();
    for (int k = tid; k < kSfT * kSfT; k += blockDim.x) {
      const int r = k / kSfT, c = k - r * kSfT;
      // tile (ti, tj): sigma[i][j] = A[i][j] + A[j][i]
      const int i1 = ti * kSfT + r, j1 = tj * kSfT + c;
      if (i1 < n && j1 < n) {
        const size_t I = (size_t)i1 * n + j1;
        const double sv = (double)(tA[r][c] + tB[c][r]);
        sig[I] = sv;
#pragma unroll
        for (int j = 0; j < 3; ++j) ud[j] = fma(du[j][I], sv, ud[j]);
      }
      // tile (tj, ti), off the diagonal: the transpose of tile (ti, tj), since
      // sigma, x, y and z are symmetric matrices (the same values; the dots of
      // the pair count tile (ti, tj) twice)
      const int i2 = tj * kSfT + r, j2 = ti * kSfT + c;
      if (ti != tj && i2 < n && j2 < n) sig[(size_t)i2 * n + j2] = (double)(tB[r][c] + tA[c][r]);
    }
    const double wgt = (ti != tj) ? 2.0 : 1.0;
#pragma unroll
    for (int j = 0; j < 3; ++j) dots[j] = fma(wgt, ud[j], dots[j]);
  }
  block_partials<3, kScTile>(dots, a.dot_slot, a.partials, nvb, vb);
  if (!last_block(a.counter, nvb)) return false;
  finish_slots(a.partials, nvb, a.dot_slot, 3, ctl->dots, a.counter);
  return ctl_run_shadowed(ctl, [](CtlHead &h) { ctl_solve(h); }) != 0;
}

}  // namespace sbci
