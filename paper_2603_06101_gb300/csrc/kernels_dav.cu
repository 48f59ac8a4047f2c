// Kernels of the host-driven solvers: the block Davidson-Liu solver
// (Davidson 1975; Liu 1978), the method the paper compares SBCI with, and the
// SBCI2 pair steps (Algorithm 2).  Dot products over lists of vector pairs,
// linear combinations of whole vectors, and the diagonal preconditioner
// (D - theta)^-1.  For Davidson these are the "inner products and
// matrix-product constructions" over the stored subspace that SBCI avoids
// (Introduction); each is one streaming pass over its vectors.
//
// Dot products are reduced in two fixed-order stages (block partials, then
// one pass per slot in k_reduce), so results do not depend on scheduling.
#include <cuda_runtime.h>

#include "sbci_internal.h"

namespace sbci {

namespace {

constexpr int kDavThreads = 256;
constexpr int kDavGroup = 8;  // pairs accumulated per pass over the vectors

struct DavDots {
  const double *u[kDavMaxPairs];
  const double *v[kDavMaxPairs];
  int n;
};

struct DavComb {
  const double *in[kDavMaxIn];
  double *out[kDavMaxOut];
  double coef[kDavMaxIn * kDavMaxOut];  // [input][output]
  int nin, nout;
};

__device__ __forceinline__ double dav_warp_sum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

// partials[p * grid + block] = this block's part of u_p . v_p, pairs in
// groups of kDavGroup per pass (the vectors of a group are read once).
__global__ void __launch_bounds__(kDavThreads) k_dav_dots(const __grid_constant__ DavDots L, long long n,
                                                          double *partials, int grid) {
  __shared__ double red[kDavGroup][kDavThreads / 32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (int g0 = 0; g0 < L.n; g0 += kDavGroup) {
    const int ng = min(kDavGroup, L.n - g0);
    double acc[kDavGroup];
#pragma unroll
    for (int j = 0; j < kDavGroup; ++j) acc[j] = 0.0;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
#pragma unroll
      for (int j = 0; j < kDavGroup; ++j)
        if (j < ng) acc[j] += L.u[g0 + j][i] * L.v[g0 + j][i];
    }
#pragma unroll
    for (int j = 0; j < kDavGroup; ++j) {
      const double s = dav_warp_sum(acc[j]);
      if (lane == 0) red[j][wid] = s;
    }
    __syncthreads();
    if (threadIdx.x < ng) {
      double s = 0.0;
      for (int w = 0; w < kDavThreads / 32; ++w) s += red[threadIdx.x][w];
      partials[(size_t)(g0 + threadIdx.x) * grid + blockIdx.x] = s;
    }
    __syncthreads();  // red[] is reused by the next group
  }
}

// out_j[i] = sum_q coef[q][j] in_q[i].  A thread reads every input at index i
// before it writes any output there, so an output may be one of the inputs
// (in-place collapse and projection).
__global__ void __launch_bounds__(kDavThreads) k_dav_combine(const __grid_constant__ DavComb C, long long n) {
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    double acc[kDavMaxOut];
#pragma unroll
    for (int j = 0; j < kDavMaxOut; ++j) acc[j] = 0.0;
    for (int q = 0; q < C.nin; ++q) {
      const double x = C.in[q][i];
#pragma unroll
      for (int j = 0; j < kDavMaxOut; ++j)
        if (j < C.nout) acc[j] += C.coef[q * kDavMaxOut + j] * x;
    }
#pragma unroll
    for (int j = 0; j < kDavMaxOut; ++j)
      if (j < C.nout) C.out[j][i] = acc[j];
  }
}

// out_i = in_i / d_i, d_i = D_i - shift with |d_i| < guard replaced by
// sign(d_i) guard (d_i = 0 -> +guard), the guard SBCI uses (Eqs. 6-7).
// out may be in.
__global__ void k_dav_precond(double *out, const double *in, const double *diag, double shift, double guard,
                              long long n) {
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    double d = diag[i] - shift;
    if (fabs(d) < guard) d = d < 0.0 ? -guard : guard;
    out[i] = in[i] / d;
  }
}

// The combination with its coefficients in device memory (coef[q * kDavMaxOut
// + j], written by a controller kernel), skipped when *active == 0: the same
// per-element arithmetic as k_dav_combine.
struct DavCombDev {
  const double *in[kDavMaxIn];
  double *out[kDavMaxOut];
  int nin, nout;
};

__global__ void __launch_bounds__(kDavThreads) k_dav_combine_dev(const __grid_constant__ DavCombDev C,
                                                                 const double *coef, const int *active,
                                                                 long long n) {
  if (active && *active == 0) return;
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    double acc[kDavMaxOut];
#pragma unroll
    for (int j = 0; j < kDavMaxOut; ++j) acc[j] = 0.0;
    for (int q = 0; q < C.nin; ++q) {
      const double x = C.in[q][i];
#pragma unroll
      for (int j = 0; j < kDavMaxOut; ++j)
        if (j < C.nout) acc[j] += coef[q * kDavMaxOut + j] * x;
    }
#pragma unroll
    for (int j = 0; j < kDavMaxOut; ++j)
      if (j < C.nout) C.out[j][i] = acc[j];
  }
}

// k_dav_precond with the shift read from device memory.
__global__ void k_dav_precond_dev(double *out, const double *in, const double *diag, const double *shift,
                                  double guard, long long n) {
  const double sh = *shift;
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    double d = diag[i] - sh;
    if (fabs(d) < guard) d = d < 0.0 ? -guard : guard;
    out[i] = in[i] / d;
  }
}

int dav_grid(long long n, int cap) {
  long long g = (n + kDavThreads - 1) / kDavThreads;
  if (g > cap) g = cap;
  if (g < 1) g = 1;
  return (int)g;
}

}  // namespace

int dav_dots_grid(long long n, int nsm) {
  // about eight elements per thread, at most four blocks per SM
  long long g = (n + 8LL * kDavThreads - 1) / (8LL * kDavThreads);
  if (g > 4LL * nsm) g = 4LL * nsm;
  if (g < 1) g = 1;
  return (int)g;
}

cudaError_t launch_dav_dots(const double *const *u, const double *const *v, int npairs, long long n,
                            double *partials, int grid, cudaStream_t s) {
  if (npairs < 1 || npairs > kDavMaxPairs) return cudaErrorInvalidValue;
  DavDots L{};
  L.n = npairs;
  for (int p = 0; p < npairs; ++p) {
    L.u[p] = u[p];
    L.v[p] = v[p];
  }
  k_dav_dots<<<grid, kDavThreads, 0, s>>>(L, n, partials, grid);
  return cudaGetLastError();
}

cudaError_t launch_dav_combine(double *const *out, int nout, const double *const *in, int nin,
                               const double *coef, long long n, int nsm, cudaStream_t s) {
  if (nin < 1 || nin > kDavMaxIn || nout < 1 || nout > kDavMaxOut) return cudaErrorInvalidValue;
  DavComb C{};
  C.nin = nin;
  C.nout = nout;
  for (int q = 0; q < nin; ++q) {
    C.in[q] = in[q];
    for (int j = 0; j < nout; ++j) C.coef[q * kDavMaxOut + j] = coef[q * nout + j];
  }
  for (int j = 0; j < nout; ++j) C.out[j] = out[j];
  k_dav_combine<<<dav_grid(n, 8 * nsm), kDavThreads, 0, s>>>(C, n);
  return cudaGetLastError();
}

cudaError_t launch_dav_precond(double *out, const double *in, const double *diag, double shift, double guard,
                               long long n, int nsm, cudaStream_t s) {
  k_dav_precond<<<dav_grid(n, 8 * nsm), kDavThreads, 0, s>>>(out, in, diag, shift, guard, n);
  return cudaGetLastError();
}

cudaError_t launch_dav_combine_dev(double *const *out, int nout, const double *const *in, int nin,
                                   const double *coef, const int *active, long long n, int nsm, cudaStream_t s) {
  if (nin < 1 || nin > kDavMaxIn || nout < 1 || nout > kDavMaxOut) return cudaErrorInvalidValue;
  DavCombDev C{};
  C.nin = nin;
  C.nout = nout;
  for (int q = 0; q < nin; ++q) C.in[q] = in[q];
  for (int j = 0; j < nout; ++j) C.out[j] = out[j];
  k_dav_combine_dev<<<dav_grid(n, 8 * nsm), kDavThreads, 0, s>>>(C, coef, active, n);
  return cudaGetLastError();
}

cudaError_t launch_dav_precond_dev(double *out, const double *in, const double *diag, const double *shift,
                                   double guard, long long n, int nsm, cudaStream_t s) {
  k_dav_precond_dev<<<dav_grid(n, 8 * nsm), kDavThreads, 0, s>>>(out, in, diag, shift, guard, n);
  return cudaGetLastError();
}

}  // namespace sbci
