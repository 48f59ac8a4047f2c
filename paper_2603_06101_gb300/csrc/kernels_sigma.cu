// Sigma build sigma = H c over alpha/beta strings (the H-product of Eq. S9 and
// Eq. S32), in two kernels:
//
//  1. gather + contract:   D[Q, I] = sum_{links of I} sign * c[J]   (both spins)
//                          G[P, I] = sum_Q W[P, Q] D[Q, I]
//  2. gather-form scatter: sigma[I] = sum_{links of I} sign * G[pair, J]
//     with the dot products of sigma against up to three vectors fused in.
//
// H = sum_{ij,kl} W_{ij,kl} E_ij E_kl with the one-electron part absorbed
// into W (see api.cpp); D and G are over packed pairs P = (i >= j).  Both
// phases read the excitation list of the determinant's own strings, using
// <I|E_kl|J> = <J|E_lk|I>, so neither phase needs atomics and the result is
// bitwise reproducible.  G is the only scratch, [npair][Ndet].
#include <cuda_runtime.h>

#include "ctl.h"
#include "devreduce.cuh"
#include "sbci_internal.h"

namespace sbci {

constexpr int kTile = 64;   // determinants per tile = threads per block (gather + contract)
constexpr int kScTile = 256;  // determinants per tile of the scatter
constexpr int kRows = 8;    // W rows per register block of the contraction

// Phase 1.  One thread per determinant; the thread's D column lives in shared
// memory (npair values), so no block-level synchronisation is needed.
template <typename AccT>
__global__ void __launch_bounds__(kTile) k_gather_contract(SigmaArgs a) {
  extern __shared__ unsigned char smem_raw[];
  AccT *sD = reinterpret_cast<AccT *>(smem_raw);  // [npair][kTile]
  const int tid = threadIdx.x;
  const double *cin = a.c;
  if (a.ctl) {
    if (a.ctl->halt) return;
    cin = a.ctl->zn;
  }
  const long long ntiles = (a.ndet + kTile - 1) / kTile;
  AccT *G = reinterpret_cast<AccT *>(a.G);
  for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const long long I = tile * kTile + tid;
    if (I >= a.ndet) continue;
    for (int q = 0; q < a.npair; ++q) sD[q * kTile + tid] = (AccT)0;
    const int ia = (int)(I / a.nb), ib = (int)(I - (long long)ia * a.nb);
    const uint32_t *la = a.link_a + (size_t)ia * a.nlink_a;
    const double *ccol = cin + ib;
    for_links<8, double>(
        la, a.nlink_a, [&](uint32_t v) { return __ldg(ccol + (size_t)link_J(v) * a.nb); },
        [&](uint32_t v, double cv) {
          AccT &d = sD[link_pair(v) * kTile + tid];
          d += link_neg(v) ? (AccT)(-cv) : (AccT)cv;
        });
    const uint32_t *lb = a.link_b + (size_t)ib * a.nlink_b;
    const double *crow = cin + (size_t)ia * a.nb;
    for_links<8, double>(
        lb, a.nlink_b, [&](uint32_t v) { return __ldg(crow + link_J(v)); },
        [&](uint32_t v, double cv) {
          AccT &d = sD[link_pair(v) * kTile + tid];
          d += link_neg(v) ? (AccT)(-cv) : (AccT)cv;
        });
    const AccT *W = nullptr;
    if constexpr (sizeof(AccT) == 8) W = reinterpret_cast<const AccT *>(a.W);
    else W = reinterpret_cast<const AccT *>(a.Wf);
    for (int P0 = 0; P0 < a.npair; P0 += kRows) {
      AccT acc[kRows];
#pragma unroll
      for (int r = 0; r < kRows; ++r) acc[r] = (AccT)0;
      for (int q = 0; q < a.npair; ++q) {
        const AccT d = sD[q * kTile + tid];
#pragma unroll
        for (int r = 0; r < kRows; ++r) acc[r] = fma(__ldg(W + (size_t)(P0 + r) * a.npair + q), d, acc[r]);
      }
#pragma unroll
      for (int r = 0; r < kRows; ++r)
        if (P0 + r < a.npair) G[(size_t)(P0 + r) * a.ndet + I] = acc[r];
    }
  }
}

// Phase 2.  sigma[I] = sum over the links of I of sign * G[pair, J], with the
// dots of sigma against up to three vectors; in device-controlled mode the
// last block finishes the dots and runs the subspace solve (ctl.h).
template <typename AccT>
__global__ void __launch_bounds__(kScTile) k_scatter(SigmaArgs a) {
  double *sig = a.sigma;
  const double *du[3] = {a.dot_u[0], a.dot_u[1], a.dot_u[2]};
  if (a.ctl) {
    if (a.ctl->halt) {
      if (a.cond && blockIdx.x == 0 && threadIdx.x == 0)
        cudaGraphSetConditional((cudaGraphConditionalHandle)a.cond, 0u);
      return;
    }
    sig = a.ctl->Zn;
    du[2] = a.ctl->zn;
  }
  const int tid = threadIdx.x;
  const long long ntiles = (a.ndet + kScTile - 1) / kScTile;
  const AccT *G = reinterpret_cast<const AccT *>(a.G);
  double dots[3] = {0.0, 0.0, 0.0};
  for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const long long I = tile * kScTile + tid;
    if (I >= a.ndet) continue;
    const int ia = (int)(I / a.nb), ib = (int)(I - (long long)ia * a.nb);
    AccT acc = (AccT)0;
    const uint32_t *la = a.link_a + (size_t)ia * a.nlink_a;
    const AccT *gcol = G + ib;
    for_links<8, AccT>(
        la, a.nlink_a,
        [&](uint32_t v) { return __ldg(gcol + (size_t)link_pair(v) * a.ndet + (size_t)link_J(v) * a.nb); },
        [&](uint32_t v, AccT g) { acc += link_neg(v) ? -g : g; });
    const uint32_t *lb = a.link_b + (size_t)ib * a.nlink_b;
    const AccT *grow = G + (size_t)ia * a.nb;
    for_links<8, AccT>(
        lb, a.nlink_b, [&](uint32_t v) { return __ldg(grow + (size_t)link_pair(v) * a.ndet + link_J(v)); },
        [&](uint32_t v, AccT g) { acc += link_neg(v) ? -g : g; });
    const double sv = (double)acc;
    sig[I] = sv;
#pragma unroll
    for (int j = 0; j < 3; ++j)
      if (du[j]) dots[j] += du[j][I] * sv;
  }
  if (!du[0] && !du[1] && !du[2]) return;
  int slots[3];
#pragma unroll
  for (int j = 0; j < 3; ++j) slots[j] = du[j] ? a.dot_slot[j] : -1;
  block_partials<3, kScTile>(dots, slots, a.partials, gridDim.x);
  if (!a.ctl) return;  // host mode: the host reduces the partials
  if (!last_block(a.counter)) return;
  finish_slots(a.partials, gridDim.x, a.dot_slot, 3, a.ctl->dots, a.counter);
  if (threadIdx.x == 0) {
    ctl_solve(*a.ctl);
    if (a.ctl->halt && a.cond) cudaGraphSetConditional((cudaGraphConditionalHandle)a.cond, 0u);
  }
}

size_t sigma_scratch_bytes(int npair, long long ndet, int prec) {
  const size_t el = (prec == 0) ? sizeof(double) : sizeof(float);
  return el * (size_t)npair * (size_t)ndet;
}

template <typename AccT>
static cudaError_t launch_gc_t(const SigmaArgs &a, cudaStream_t s) {
  const long long ntiles = (a.ndet + kTile - 1) / kTile;
  const int grid1 = (int)(ntiles < 65535LL * 16 ? ntiles : 65535LL * 16);
  const size_t smem = sizeof(AccT) * (size_t)a.npair * kTile;
  k_gather_contract<AccT><<<grid1, kTile, smem, s>>>(a);
  return cudaGetLastError();
}

int scatter_grid(long long ndet, int nsm) {
  long long g = (ndet + kScTile - 1) / kScTile;
  if (g > 8LL * nsm) g = 8LL * nsm;
  if (g < 1) g = 1;
  return (int)g;
}

template <typename AccT>
static cudaError_t launch_sc_t(const SigmaArgs &a, cudaStream_t s) {
  k_scatter<AccT><<<a.grid, kScTile, 0, s>>>(a);
  return cudaGetLastError();
}

// Opts the gather+contract kernels into large dynamic shared memory (once per
// process, outside any stream capture).
cudaError_t prepare_sigma_kernels() {
  const int big = 227 * 1024;
  cudaError_t e = cudaFuncSetAttribute(k_gather_contract<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(k_gather_contract<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
}

cudaError_t launch_gather_contract(const SigmaArgs &a, int prec, cudaStream_t s) {
  return prec == 0 ? launch_gc_t<double>(a, s) : launch_gc_t<float>(a, s);
}
cudaError_t launch_scatter(const SigmaArgs &a, int prec, cudaStream_t s) {
  return prec == 0 ? launch_sc_t<double>(a, s) : launch_sc_t<float>(a, s);
}

}  // namespace sbci
