// FP64 helper kernels: linear combinations and dot products for the rare
// host-driven events (initial guess, state transitions), the diagonal of H,
// and deterministic reductions.
//
// Every dot product is reduced in two fixed-order stages (block partials,
// then one pass per slot), so results do not depend on scheduling.
#include <cuda_runtime.h>

#include "sbci_internal.h"

namespace sbci {

constexpr int kVecThreads = 256;

__device__ __forceinline__ double warp_sum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

// Block reduction of NV values per thread; thread 0 writes partials.
template <int NV>
__device__ __forceinline__ void block_store(double (&v)[NV], const int *slots, double *partials,
                                            int grid) {
  __shared__ double red[NV][kVecThreads / 32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int j = 0; j < NV; ++j) {
    const double s = warp_sum(v[j]);
    if (lane == 0) red[j][wid] = s;
  }
  __syncthreads();
  if (threadIdx.x < NV) {
    const int j = threadIdx.x;
    double s = 0.0;
    for (int i = 0; i < kVecThreads / 32; ++i) s += red[j][i];
    if (slots[j] >= 0) partials[(size_t)slots[j] * grid + blockIdx.x] = s;
  }
}

struct LinComb {
  const double *in[8];
  double coef[8];
  int nin;
};

__global__ void k_lincomb(double *out, LinComb L, long long n) {
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    double s = 0.0;
    for (int j = 0; j < L.nin; ++j) s += L.coef[j] * L.in[j][i];
    out[i] = s;
  }
}

struct DotList {
  const double *u[16];
  const double *v[16];
  int n;
};

__global__ void __launch_bounds__(kVecThreads) k_dots(DotList L, long long n, double *partials, int grid) {
  double acc[16];
#pragma unroll
  for (int j = 0; j < 16; ++j) acc[j] = 0.0;
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
#pragma unroll
    for (int j = 0; j < 16; ++j)
      if (j < L.n) acc[j] += L.u[j][i] * L.v[j][i];
  }
  int slots[16];
  for (int j = 0; j < 16; ++j) slots[j] = (j < L.n) ? S_GEN0 + j : -1;
  block_store<16>(acc, slots, partials, grid);
}

__global__ void k_reduce(const double *partials, int grid, int s0, double *result) {
  __shared__ double red[kVecThreads / 32];
  const int slot = s0 + blockIdx.x;
  double v = 0.0;
  for (int i = threadIdx.x; i < grid; i += blockDim.x) v += partials[(size_t)slot * grid + i];
  v = warp_sum(v);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) s += red[i];
    result[slot] = s;
  }
}

// D_I = ea[Ia] + eb[Ib] + sum_{q in occ(Ib)} ja[Ia][q]
__global__ void k_diagonal(double *diag, const double *ea, const double *eb, const double *ja,
                           const uint32_t *mask_b, int na, int nb, int norb) {
  const long long n = (long long)na * nb;
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    const int ia = (int)(i / nb), ib = (int)(i - (long long)ia * nb);
    double s = ea[ia] + eb[ib];
    uint32_t m = mask_b[ib];
    while (m) {
      const int q = __ffs(m) - 1;
      s += ja[(size_t)ia * norb + q];
      m &= m - 1u;
    }
    diag[i] = s;
  }
}

__global__ void k_symmetrize(double *v, int n) {
  const long long total = (long long)n * n;
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += stride) {
    const int a = (int)(i / n), b = (int)(i - (long long)a * n);
    if (a < b) {
      const double s = 0.5 * (v[i] + v[(size_t)b * n + a]);
      v[i] = s;
      v[(size_t)b * n + a] = s;
    }
  }
}

// SplitMix64 output function (Steele, Lea & Flood 2014) on a counter.
__device__ __forceinline__ unsigned long long splitmix(unsigned long long z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

__global__ void k_splitmix(double *r, long long n, unsigned long long seed, int alpha) {
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    const unsigned long long ctr = ((unsigned long long)alpha << 40) + (unsigned long long)i + 1ull;
    const unsigned long long z = splitmix(seed + 0x9E3779B97F4A7C15ull * ctr);
    r[i] = 2.0 * ((double)(z >> 11) * 0x1.0p-53) - 1.0;
  }
}

static int grid_for(long long n, int cap) {
  long long g = (n + kVecThreads - 1) / kVecThreads;
  if (g > cap) g = cap;
  if (g < 1) g = 1;
  return (int)g;
}

cudaError_t launch_lincomb(double *out, const double *const *in, const double *coef, int nin,
                           long long n, cudaStream_t s) {
  LinComb L{};
  L.nin = nin;
  for (int j = 0; j < nin && j < 8; ++j) {
    L.in[j] = in[j];
    L.coef[j] = coef[j];
  }
  k_lincomb<<<grid_for(n, 4096), kVecThreads, 0, s>>>(out, L, n);
  return cudaGetLastError();
}

cudaError_t launch_dots(const double *const *u, const double *const *v, int npairs, long long n,
                        double *partials, int grid, cudaStream_t s) {
  DotList L{};
  L.n = npairs;
  for (int j = 0; j < npairs && j < 16; ++j) {
    L.u[j] = u[j];
    L.v[j] = v[j];
  }
  k_dots<<<grid, kVecThreads, 0, s>>>(L, n, partials, grid);
  return cudaGetLastError();
}

__global__ void k_sparse_set(double *dst, const double *pairs, int n) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q < n) dst[(long long)pairs[2 * q]] = pairs[2 * q + 1];
}

__global__ void k_gather_at(const double *src, const double *offs, int n, double *out) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q < n) out[q] = src[(long long)offs[q]];
}

cudaError_t launch_sparse_set(double *dst, const double *pairs, int n, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  k_sparse_set<<<(n + 255) / 256, 256, 0, s>>>(dst, pairs, n);
  return cudaGetLastError();
}

cudaError_t launch_gather_at(const double *src, const double *offs, int n, double *out, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  k_gather_at<<<(n + 255) / 256, 256, 0, s>>>(src, offs, n, out);
  return cudaGetLastError();
}

cudaError_t launch_reduce(const double *partials, int grid, int s0, int s1, double *result,
                          cudaStream_t s) {
  if (s1 <= s0) return cudaSuccess;
  k_reduce<<<s1 - s0, kVecThreads, 0, s>>>(partials, grid, s0, result);
  return cudaGetLastError();
}

cudaError_t launch_diagonal(double *diag, const double *ea, const double *eb, const double *ja,
                            const uint32_t *mask_b, int na, int nb, int norb, cudaStream_t s) {
  k_diagonal<<<grid_for((long long)na * nb, 8192), kVecThreads, 0, s>>>(diag, ea, eb, ja, mask_b,
                                                                        na, nb, norb);
  return cudaGetLastError();
}

__global__ void k_to_float(const double *in, float *out, long long n) {
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) out[i] = (float)in[i];
}

cudaError_t launch_to_float(const double *in, float *out, long long n, cudaStream_t s) {
  k_to_float<<<grid_for(n, 8192), kVecThreads, 0, s>>>(in, out, n);
  return cudaGetLastError();
}

cudaError_t launch_splitmix(double *r, long long n, unsigned long long seed, int alpha, cudaStream_t s) {
  k_splitmix<<<grid_for(n, 8192), kVecThreads, 0, s>>>(r, n, seed, alpha);
  return cudaGetLastError();
}

cudaError_t launch_symmetrize(double *v, int n, cudaStream_t s) {
  k_symmetrize<<<grid_for((long long)n * n, 8192), kVecThreads, 0, s>>>(v, n);
  return cudaGetLastError();
}

}  // namespace sbci
