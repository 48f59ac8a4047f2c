// Deterministic FP64 reductions for kernels whose last block finishes a
// global sum.  GB300 runs FP64 at a small fraction of its FP32 rate, so the
// block stage avoids shuffle trees over many values: each warp transposes its
// values through shared memory and one lane per value adds the 32 entries in
// order.  The grid stage sums the per-block partials in a fixed order.
#pragma once

#include <cuda_runtime.h>

namespace sbci {

// Block partials of NV values per thread -> partials[slot * grid + block]
// (slots[j] < 0: value j unused).  NT = threads per block; block is the
// (virtual) block index within its grid of size grid; buf: shared memory of
// [NT / 32][NV][33] doubles; scale (optional): a factor per value applied to
// the block's sum.
template <int NV, int NT>
__device__ __forceinline__ void block_partials_in(const double (&v)[NV], const int (&slots)[NV],
                                                  double *partials, int grid, int block, double (*buf)[NV][33],
                                                  const double *scale = nullptr) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  __syncthreads();  // a persistent block may come back with the buffer still in use
#pragma unroll
  for (int j = 0; j < NV; ++j) buf[wid][j][lane] = v[j];
  __syncwarp();
  double ws = 0.0;
  if (lane < NV)
    for (int i = 0; i < 32; ++i) ws += buf[wid][lane][i];
  __syncwarp();
  if (lane < NV) buf[wid][lane][32] = ws;
  __syncthreads();
  if (threadIdx.x < NV) {
    const int j = threadIdx.x;
    double s = 0.0;
    for (int w = 0; w < NT / 32; ++w) s += buf[w][j][32];
    if (scale) s *= scale[j];  // a block sum's weight (exact for powers of two)
    if (slots[j] >= 0) partials[(size_t)slots[j] * grid + block] = s;
  }
}

// The same with the block's own shared buffer.
template <int NV, int NT>
__device__ __forceinline__ void block_partials(const double (&v)[NV], const int (&slots)[NV],
                                               double *partials, int grid, int block) {
  __shared__ double buf[NT / 32][NV][33];
  block_partials_in<NV, NT>(v, slots, partials, grid, block, buf);
}

// Bytes of the caller-provided buffer of block_partials_in.
template <int NV, int NT>
constexpr size_t block_partials_bytes() {
  return sizeof(double) * (NT / 32) * NV * 33;
}

// Returns true in exactly one of nblocks (virtual) blocks: the last one to
// arrive.  Its threads then see every other block's partials.
__device__ __forceinline__ bool last_block(unsigned int *counter, int nblocks) {
  __shared__ unsigned int s_last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) s_last = (atomicAdd(counter, 1u) == (unsigned int)nblocks - 1u) ? 1u : 0u;
  __syncthreads();
  if (s_last) __threadfence();
  return s_last != 0u;
}

// In the last block: out[slot] = sum_b partials[slot * grid + b] in a fixed
// order (lane-strided sums, then a fixed shuffle tree), one warp per slot;
// resets the counter for the next launch.
__device__ __forceinline__ void finish_slots(const double *partials, int grid, const int *slots,
                                             int nslots, double *out, unsigned int *counter) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int j = wid; j < nslots; j += nw) {
    const int slot = slots[j];
    double s = 0.0;
    for (int b = lane; b < grid; b += 32) s += __ldcg(partials + (size_t)slot * grid + b);
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if (lane == 0) out[slot] = s;
  }
  __syncthreads();
  if (threadIdx.x == 0) *counter = 0u;
}

}  // namespace sbci
