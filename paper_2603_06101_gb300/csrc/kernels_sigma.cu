// Sigma build sigma = H c over alpha/beta strings (the H-product of Eq. S9 and
// Eq. S32), in two kernels (the SIMT gather + contract here; the scatter, with
// the other kernels of the SB step loop, in kernels_loop.cu):
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
#include "lowrank.h"
#include "sbci_internal.h"

namespace sbci {

constexpr int kTile = 64;   // determinants per tile = threads per block (gather + contract)
constexpr int kRows = 8;    // W rows per register block of the contraction

// D column of determinant I (both spins) into shared memory; cin is the input
// vector in FP64 or, for the FP32 accumulation, its FP32 copy (the same
// values after the conversion, so the same D).
template <typename AccT, typename T>
__device__ __forceinline__ void simt_gather(const SigmaArgs &a, const T *cin, long long I, int tid, AccT *sD) {
  for (int q = 0; q < a.npair; ++q) sD[q * kTile + tid] = (AccT)0;
  int ia, ib;
    split_det(I, a.nb, ia, ib);
  const uint32_t *la = a.link_a + (size_t)ia * a.nlink_a;
  const T *ccol = cin + ib;
  for_links<8, T>(
      la, a.nlink_a, 1, [&](uint32_t v) { return __ldg(ccol + (size_t)link_J(v) * a.nb); },
      [&](uint32_t v, T cv) {
        AccT &d = sD[link_pair(v) * kTile + tid];
        d += link_neg(v) ? (AccT)(-cv) : (AccT)cv;
      });
  const uint32_t *lb = a.link_bT + ib;
  const T *crow = cin + (size_t)ia * a.nb;
  for_links<8, T>(
      lb, a.nlink_b, a.nb, [&](uint32_t v) { return __ldg(crow + link_J(v)); },
      [&](uint32_t v, T cv) {
        AccT &d = sD[link_pair(v) * kTile + tid];
        d += link_neg(v) ? (AccT)(-cv) : (AccT)cv;
      });
}

// Phase 1.  One thread per determinant; the thread's D column lives in shared
// memory (npair values), so no block-level synchronisation is needed.
template <typename AccT>
__global__ void __launch_bounds__(kTile) k_gather_contract(SigmaArgs a) {
  extern __shared__ unsigned char smem_raw[];
  AccT *sD = reinterpret_cast<AccT *>(smem_raw);  // [npair][kTile]
  const int tid = threadIdx.x;
  const double *cin = a.c;
  const float *cinf = nullptr;
  if (a.ctl) {
    if (a.ctl->halt) return;
    cin = a.ctl->zn;
    if constexpr (sizeof(AccT) == 4) cinf = a.ctl->zf;
  }
  const long long ntiles = (a.ndet + kTile - 1) / kTile;
  AccT *G = reinterpret_cast<AccT *>(a.G);
  for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const long long I = tile * kTile + tid;
    if (I >= a.ndet) continue;
    if (cinf) simt_gather<AccT, float>(a, cinf, I, tid, sD);
    else simt_gather<AccT, double>(a, cin, I, tid, sD);
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

// Phase 1 in the low-rank form of W (lowrank.h): t = F^T D into shared
// memory after the D column, then G = (F M) t.  Same gather.
template <typename AccT>
__global__ void __launch_bounds__(kTile) k_gather_contract_lr(SigmaArgs a, const AccT *Ut, const AccT *UL, int r) {
  extern __shared__ unsigned char smem_raw[];
  AccT *sD = reinterpret_cast<AccT *>(smem_raw);  // [npair][kTile]
  AccT *sT = sD + (size_t)a.npair * kTile;        // [r][kTile]
  const int tid = threadIdx.x;
  const double *cin = a.c;
  const float *cinf = nullptr;
  if (a.ctl) {
    if (a.ctl->halt) return;
    cin = a.ctl->zn;
    if constexpr (sizeof(AccT) == 4) cinf = a.ctl->zf;
  }
  const long long ntiles = (a.ndet + kTile - 1) / kTile;
  AccT *G = reinterpret_cast<AccT *>(a.G);
  for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const long long I = tile * kTile + tid;
    if (I >= a.ndet) continue;
    if (cinf) simt_gather<AccT, float>(a, cinf, I, tid, sD);
    else simt_gather<AccT, double>(a, cin, I, tid, sD);
    for (int R0 = 0; R0 < r; R0 += kRows) {
      AccT acc[kRows];
#pragma unroll
      for (int k = 0; k < kRows; ++k) acc[k] = (AccT)0;
      for (int q = 0; q < a.npair; ++q) {
        const AccT d = sD[q * kTile + tid];
#pragma unroll
        for (int k = 0; k < kRows; ++k)
          if (R0 + k < r) acc[k] = fma(__ldg(Ut + (size_t)(R0 + k) * a.npair + q), d, acc[k]);
      }
#pragma unroll
      for (int k = 0; k < kRows; ++k)
        if (R0 + k < r) sT[(R0 + k) * kTile + tid] = acc[k];
    }
    for (int P0 = 0; P0 < a.npair; P0 += kRows) {
      AccT acc[kRows];
#pragma unroll
      for (int k = 0; k < kRows; ++k) acc[k] = (AccT)0;
      for (int q = 0; q < r; ++q) {
        const AccT t = sT[q * kTile + tid];
#pragma unroll
        for (int k = 0; k < kRows; ++k)
          if (P0 + k < a.npair) acc[k] = fma(__ldg(UL + (size_t)(P0 + k) * r + q), t, acc[k]);
      }
#pragma unroll
      for (int k = 0; k < kRows; ++k)
        if (P0 + k < a.npair) G[(size_t)(P0 + k) * a.ndet + I] = acc[k];
    }
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

// Opts the gather+contract kernels into large dynamic shared memory (once per
// process, outside any stream capture).
cudaError_t prepare_sigma_kernels() {
  const int big = 227 * 1024;
  cudaError_t e = cudaFuncSetAttribute(k_gather_contract<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_gather_contract<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_gather_contract_lr<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_gather_contract_lr<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
  return e;
}

template <typename AccT>
static cudaError_t launch_lr_t(const SigmaArgs &a, const AccT *Ut, const AccT *UL, int r, cudaStream_t s) {
  const long long ntiles = (a.ndet + kTile - 1) / kTile;
  const int grid1 = (int)(ntiles < 65535LL * 16 ? ntiles : 65535LL * 16);
  const size_t smem = sizeof(AccT) * (size_t)(a.npair + r) * kTile;
  k_gather_contract_lr<AccT><<<grid1, kTile, smem, s>>>(a, Ut, UL, r);
  return cudaGetLastError();
}

cudaError_t launch_gather_contract_lr(const SigmaArgs &a, int prec, const void *Ut, const void *UL, int r,
                                      cudaStream_t s) {
  if (r < 1) return cudaErrorInvalidValue;
  return prec == 0 ? launch_lr_t<double>(a, (const double *)Ut, (const double *)UL, r, s)
                   : launch_lr_t<float>(a, (const float *)Ut, (const float *)UL, r, s);
}

cudaError_t launch_gather_contract(const SigmaArgs &a, int prec, cudaStream_t s) {
  return prec == 0 ? launch_gc_t<double>(a, s) : launch_gc_t<float>(a, s);
}

}  // namespace sbci
