// Pipelined TF32x3 gather + contract on the tensor cores (one sigma call or
// one device-controlled solve; the tile arithmetic of tc_body.cuh).
//
// The plain tile kernel runs gather, split, MMAs, wait and epilogue of a tile
// one after the other in a CTA of 8 warps.  Here 4 more warps own the
// epilogue, and TMEM holds two accumulators, so the epilogue of tile i
// (tcgen05.ld, G stores to global) runs while the 8 gather warps build and
// contract tile i + 1:
//   gather warps  wait for MMA(i - 1) (it reads the A buffers), gather and
//                 split tile i (named barrier 1, 256 threads); thread 0 waits
//                 until the epilogue of tile i - 2 has drained accumulator
//                 i % 2, issues the MMAs of tile i into it and commits to
//                 mma_bar[i % 2];
//   epilogue warps wait on mma_bar[i % 2], read their lane quadrant of the
//                 accumulator, store G and arrive on free_bar[i % 2].
// mma_bar[j] completes once per tile i with i % 2 = j, so tile i waits on
// parity (i / 2) % 2; free_bar[j] (128 arrivals) likewise.  Every wait is
// bounded: a wait that runs out makes its group leave the tile loop (the
// other group's waits then run out too), raises bit 0 of *status, and the
// CTA waits once more (bounded) for its last MMAs before freeing TMEM.  The
// D operand, the split, the MMAs and the G values are those of the plain
// kernel.
#include <cuda_runtime.h>
#include <stdint.h>

#include "ctl.h"
#include "sbci_internal.h"
#include "tc_body.cuh"

namespace sbci {

namespace {

constexpr int kTpThreads = 384;  // 8 gather warps + 4 epilogue warps

// TMEM column offset of the second accumulator (a 32-column boundary).
__host__ __device__ constexpr int tp_stride(int Np) {
  return Np <= 32 ? 32 : Np <= 64 ? 64 : Np <= 128 ? 128 : 256;
}

// AND of pred over the n threads of named barrier id.
template <int kId, int kN>
__device__ __forceinline__ bool bar_and(bool pred) {
  uint32_t r;
  asm volatile(
      "{\n\t.reg .pred p, q;\n\t"
      "setp.ne.u32 q, %1, 0;\n\t"
      "bar.red.and.pred p, %2, %3, q;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}\n"
      : "=r"(r)
      : "r"((uint32_t)pred), "n"(kId), "n"(kN)
      : "memory");
  return r != 0;
}

__device__ __forceinline__ void mbar_arrive(uint32_t addr) {
  asm volatile(
      "{\n\t.reg .b64 st;\n\t"
      "mbarrier.arrive.shared::cta.b64 st, [%0];\n\t}\n" ::"r"(addr)
      : "memory");
}

__global__ void __launch_bounds__(kTpThreads, 1)
    k_gather_contract_tcp(SigmaArgs a, int Kp, int Np, uint32_t tmem_cols, int *status) {
  extern __shared__ __align__(128) unsigned char smem[];
  TcSmem sm;
  sm.A = reinterpret_cast<float *>(smem);
  sm.Alo = sm.A + kTcM * Kp;
  sm.Bhi = reinterpret_cast<uint32_t *>(sm.Alo + kTcM * Kp);
  sm.Blo = sm.Bhi + Np * Kp;
  uint64_t *bars = reinterpret_cast<uint64_t *>(sm.Blo + Np * Kp);  // mma_bar[2], free_bar[2]
  uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(bars + 4);
  sm.sA = smem_u32(sm.A);
  sm.sAlo = smem_u32(sm.Alo);
  sm.sBhi = smem_u32(sm.Bhi);
  sm.sBlo = smem_u32(sm.Blo);
  sm.sbar = smem_u32(bars);  // (unused by the helpers called here)
  const uint32_t mma_bar0 = smem_u32(bars), free_bar0 = smem_u32(bars + 2);
  const int tid = threadIdx.x, warp = tid >> 5;
  const float *cin = a.cf;
  if (a.ctl) {
    if (a.ctl->halt) return;  // uniform: before any TMEM allocation or barrier
    cin = a.ctl->zf;
  }
  if (!cin) {  // no FP32 input: refuse (uniform, before any allocation)
    if (tid == 0) atomicOr(status, 4);
    return;
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(
                     smem_u32(tmem_slot)),
                 "r"(tmem_cols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
  }
  if (tid == 0) {
    for (int j = 0; j < 2; ++j) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(mma_bar0 + 8 * j) : "memory");
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 128;\n" ::"r"(free_bar0 + 8 * j) : "memory");
    }
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  tc_load_B(a, Kp, Np, sm);  // (ends with a barrier of the whole CTA)
  const uint32_t tmem = *tmem_slot;
  const uint32_t stride = (uint32_t)tp_stride(Np);
  const long long ntiles = (a.ndet + kTcM - 1) / kTcM;
  bool ok = true;
  long long issued = 0;  // MMA groups committed (thread 0)
  if (tid < 2 * kTcM) {
    // gather warps
    const uint32_t idesc = idesc_tf32(kTcM, Np);
    const uint32_t LBO = 128, SBO = (uint32_t)Kp * 32;
    long long i = 0;
    for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++i) {
      if (i >= 1) {  // MMA(i - 1) has finished reading A / Alo
        bool w = mbar_wait(mma_bar0 + 8 * (uint32_t)((i - 1) & 1), (uint32_t)(((i - 1) >> 1) & 1), kWaitIters);
        w = bar_and<1, 2 * kTcM>(w);
        if (!w) {
          ok = false;
          break;
        }
        fence_after();
      }
      const long long I = tile * kTcM + (tid & (kTcM - 1));
      tc_gather_split<false>(a, cin, I, I < a.ndet, Kp, sm);
      if (tid == 0) {
        bool f = true;
        if (i >= 2) f = mbar_wait(free_bar0 + 8 * (uint32_t)(i & 1), (uint32_t)(((i - 2) >> 1) & 1), kWaitIters);
        if (f) {
          fence_after();
          const uint32_t acc = tmem + (uint32_t)(i & 1) * stride;
          for (int kk = 0; kk < Kp / 8; ++kk) {
            const uint32_t koff = (uint32_t)kk * 256;  // two K-adjacent core matrices
            const uint64_t ah = smem_desc(sm.sA + koff, LBO, SBO), al = smem_desc(sm.sAlo + koff, LBO, SBO);
            const uint64_t bh = smem_desc(sm.sBhi + koff, LBO, SBO), bl = smem_desc(sm.sBlo + koff, LBO, SBO);
            mma_tf32(acc, ah, bh, idesc, kk > 0 ? 1u : 0u);
            mma_tf32(acc, ah, bl, idesc, 1u);
            mma_tf32(acc, al, bh, idesc, 1u);
          }
          asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
                           mma_bar0 + 8 * (uint32_t)(i & 1))
                       : "memory");
          issued = i + 1;
        } else {
          ok = false;  // the others run out of their next wait
        }
      }
    }
  } else {
    // epilogue warps: lane quadrant warp % 4
    const int q = warp & 3;
    const int lane_row = q * 32 + (tid & 31);
    float *G = reinterpret_cast<float *>(a.G);
    long long i = 0;
    for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++i) {
      bool w = mbar_wait(mma_bar0 + 8 * (uint32_t)(i & 1), (uint32_t)((i >> 1) & 1), kWaitIters);
      w = bar_and<2, kTcM>(w);
      if (!w) {
        ok = false;
        break;
      }
      fence_after();
      const uint32_t lane_addr = tmem + (uint32_t)(i & 1) * stride + ((uint32_t)(q * 32) << 16);
      const long long I = tile * kTcM + lane_row;
      const bool valid = I < a.ndet;
      for (int c0 = 0; c0 < Np; c0 += 32) {
        uint32_t r[32];
        tmem_ld16_nowait(lane_addr + (uint32_t)c0, r);
        if (c0 + 16 < Np) tmem_ld16_nowait(lane_addr + (uint32_t)(c0 + 16), r + 16);
        asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
        if (valid) {
#pragma unroll
          for (int j = 0; j < 32; ++j)
            if (c0 + j < a.npair) G[(size_t)(c0 + j) * a.ndet + I] = __uint_as_float(r[j]);
        }
      }
      fence_before();
      mbar_arrive(free_bar0 + 8 * (uint32_t)(i & 1));
    }
  }
  const bool all_ok = __syncthreads_and(ok) != 0;
  if (!all_ok) {
    if (tid == 0) {
      atomicOr(status, 1);
      if (issued > 0)  // let the last MMAs drain (bounded)
        mbar_wait(mma_bar0 + 8 * (uint32_t)((issued - 1) & 1), (uint32_t)(((issued - 1) >> 1) & 1), kWaitIters);
    }
  }
  fence_before();
  __syncthreads();
  fence_after();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(tmem_cols)
                 : "memory");
}

bool tcp_dims(int npair, int *Kp, int *Np, uint32_t *cols, size_t *smem) {
  uint32_t c1;
  size_t s1;
  if (!tc_dims(npair, Kp, Np, &c1, &s1)) return false;
  *cols = 2u * (uint32_t)tp_stride(*Np);
  *smem = s1 + 32;  // four mbarriers and the TMEM slot (48 bytes) in place of one and the slot (16)
  return *cols <= 512 && *smem <= 227 * 1024;
}

}  // namespace

int tcp_grid(int npair, long long ndet, int num_sms) {
  int Kp, Np;
  uint32_t cols;
  size_t smem;
  if (!tcp_dims(npair, &Kp, &Np, &cols, &smem)) return 0;
  const void *f = (const void *)k_gather_contract_tcp;
  int optin = 0;
  if (max_dynamic_smem(f, &optin) != cudaSuccess || (int)smem > optin ||
      cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, optin) != cudaSuccess ||
      cudaFuncSetAttribute(f, cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared) !=
          cudaSuccess)
    return 0;
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, f, kTpThreads, smem) != cudaSuccess) return 0;
  if ((uint32_t)per_sm * cols > 512) per_sm = (int)(512 / cols);
  if (per_sm < 1) return 0;
  const long long ntiles = (ndet + kTcM - 1) / kTcM;
  long long grid = (long long)num_sms * per_sm;
  if (grid > ntiles) grid = ntiles;
  if (grid < 1) grid = 1;
  return (int)grid;
}

cudaError_t launch_gather_contract_tcp(const SigmaArgs &a, int *status, int grid, cudaStream_t s) {
  int Kp, Np;
  uint32_t cols;
  size_t smem;
  if (!tcp_dims(a.npair, &Kp, &Np, &cols, &smem) || grid < 1) return cudaErrorInvalidValue;
  k_gather_contract_tcp<<<grid, kTpThreads, smem, s>>>(a, Kp, Np, cols, status);
  return cudaGetLastError();
}

}  // namespace sbci
