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

#include "sbci_internal.h"

namespace sbci {

constexpr int kTile = 64;   // determinants per tile = threads per block
constexpr int kRows = 8;    // W rows per register block of the contraction

// Phase 1.  One thread per determinant; the thread's D column lives in shared
// memory (npair values), so no block-level synchronisation is needed.
template <typename AccT>
__global__ void __launch_bounds__(kTile) k_gather_contract(SigmaArgs a) {
  extern __shared__ unsigned char smem_raw[];
  AccT *sD = reinterpret_cast<AccT *>(smem_raw);  // [npair][kTile]
  const int tid = threadIdx.x;
  const long long ntiles = (a.ndet + kTile - 1) / kTile;
  AccT *G = reinterpret_cast<AccT *>(a.G);
  for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const long long I = tile * kTile + tid;
    if (I >= a.ndet) continue;
    for (int q = 0; q < a.npair; ++q) sD[q * kTile + tid] = (AccT)0;
    const int ia = (int)(I / a.nb), ib = (int)(I - (long long)ia * a.nb);
    const uint32_t *la = a.link_a + (size_t)ia * a.nlink_a;
    for (int e = 0; e < a.nlink_a; ++e) {
      const uint32_t v = __ldg(la + e);
      const double cv = __ldg(a.c + (size_t)link_J(v) * a.nb + ib);
      AccT &d = sD[link_pair(v) * kTile + tid];
      d += link_neg(v) ? (AccT)(-cv) : (AccT)cv;
    }
    const uint32_t *lb = a.link_b + (size_t)ib * a.nlink_b;
    const double *crow = a.c + (size_t)ia * a.nb;
    for (int e = 0; e < a.nlink_b; ++e) {
      const uint32_t v = __ldg(lb + e);
      const double cv = __ldg(crow + link_J(v));
      AccT &d = sD[link_pair(v) * kTile + tid];
      d += link_neg(v) ? (AccT)(-cv) : (AccT)cv;
    }
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

__device__ __forceinline__ double block_sum(double v, double *red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) red[wid] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x == 0)
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) s += red[i];
  return s;
}

// Phase 2.  sigma[I] = sum over the links of I of sign * G[pair, J].
template <typename AccT>
__global__ void __launch_bounds__(kTile) k_scatter(SigmaArgs a) {
  __shared__ double red[kTile / 32];
  const int tid = threadIdx.x;
  const long long ntiles = (a.ndet + kTile - 1) / kTile;
  const AccT *G = reinterpret_cast<const AccT *>(a.G);
  double dots[3] = {0.0, 0.0, 0.0};
  for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const long long I = tile * kTile + tid;
    if (I >= a.ndet) continue;
    const int ia = (int)(I / a.nb), ib = (int)(I - (long long)ia * a.nb);
    AccT acc = (AccT)0;
    const uint32_t *la = a.link_a + (size_t)ia * a.nlink_a;
    for (int e = 0; e < a.nlink_a; ++e) {
      const uint32_t v = __ldg(la + e);
      const AccT g = __ldg(G + (size_t)link_pair(v) * a.ndet + (size_t)link_J(v) * a.nb + ib);
      acc += link_neg(v) ? -g : g;
    }
    const uint32_t *lb = a.link_b + (size_t)ib * a.nlink_b;
    const size_t rowoff = (size_t)ia * a.nb;
    for (int e = 0; e < a.nlink_b; ++e) {
      const uint32_t v = __ldg(lb + e);
      const AccT g = __ldg(G + (size_t)link_pair(v) * a.ndet + rowoff + link_J(v));
      acc += link_neg(v) ? -g : g;
    }
    const double s = (double)acc;
    a.sigma[I] = s;
#pragma unroll
    for (int j = 0; j < 3; ++j)
      if (a.dot_u[j]) dots[j] += a.dot_u[j][I] * s;
  }
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    if (!a.dot_u[j]) continue;
    const double t = block_sum(dots[j], red);
    if (tid == 0) a.partials[(size_t)a.dot_slot[j] * a.grid + blockIdx.x] = t;
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
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(k_gather_contract<AccT>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  k_gather_contract<AccT><<<grid1, kTile, smem, s>>>(a);
  return cudaGetLastError();
}

template <typename AccT>
static cudaError_t launch_sc_t(const SigmaArgs &a, cudaStream_t s) {
  k_scatter<AccT><<<a.grid, kTile, 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_gather_contract(const SigmaArgs &a, int prec, cudaStream_t s) {
  return prec == 0 ? launch_gc_t<double>(a, s) : launch_gc_t<float>(a, s);
}
cudaError_t launch_scatter(const SigmaArgs &a, int prec, cudaStream_t s) {
  return prec == 0 ? launch_sc_t<double>(a, s) : launch_sc_t<float>(a, s);
}

}  // namespace sbci
