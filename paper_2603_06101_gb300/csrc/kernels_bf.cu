// Tensor-core gather + contract in 3-term BF16 split precision (SBCI_BF16X3),
// for every orbital count up to n = 16 (npair <= 136):
//
//   G^T = D_hi W_hi + D_hi W_lo + D_lo W_hi,   X_hi = bf16(X), X_lo = bf16(X - X_hi)
//
// by tcgen05.mma kind::f16 with BF16 operands and an FP32 accumulator in TMEM.
// A BF16 element is half a TF32 one, so the operands of the largest space
// (Kp = Np = 144 at n = 16) fit shared memory where the TF32 ones do not.
// The dropped D_lo W_lo term and the BF16 rounding of the lo parts leave a
// relative error of about 2^-17 per product (TF32x3: 2^-21).
//
// Per tile of 128 determinants (persistent CTAs of 256 threads):
//   1. gather   thread r adds the alpha links of row r, thread r + 128 the beta
//               links, into one FP32 row of D in shared memory (row stride
//               Kp + 1 words).  A pair receives at most one alpha and one beta
//               term, and one FP32 addition is commutative, so the shared-memory
//               atomic adds give the same D in any order;
//   2. split    each thread reads half a row into registers; after a barrier
//               it writes the BF16 hi and lo halves of that half row over the
//               same bytes, as the K-major no-swizzle canonical operand A;
//   3. MMA      three BF16 products per K step of 16, one issuing thread;
//   4. epilogue tcgen05.ld of the accumulator -> G[P][I] (FP32) in global,
//               read by the FP32 scatter.
// Operand B (W split into BF16 hi / lo in the operand layout) is made once
// per context and copied into shared memory when a CTA starts.  Every wait on
// the MMA-completion mbarrier is bounded; on timeout the kernel raises bit 0
// of *status, waits once more (bounded) for its MMAs, frees its TMEM and
// returns.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "ctl.h"
#include "sbci_internal.h"
#include "tc_body.cuh"

namespace sbci {

namespace {

constexpr int kBfThreads = 256;

// Instruction descriptor of kind::f16 with BF16 A and B (format 1 at bits 7-9
// and 10-12), F32 D (bits 4-5 = 1), both K-major, N >> 3 at bits 17-22,
// M >> 4 at bits 24-28.
__host__ __device__ constexpr uint32_t idesc_bf16x(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16x(uint32_t tmem, uint64_t ad, uint64_t bd, uint32_t idesc,
                                          uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem),
      "l"(ad), "l"(bd), "r"(idesc), "r"(accumulate)
      : "memory");
}

// BF16 element offset of (r, q) in a K-major no-swizzle operand with Kp
// columns: core matrix (r/8, q/8) of 8 rows x 8 BF16 (128 bytes), K-adjacent
// core matrices 128 bytes apart (LBO), 8-row groups Kp*16 bytes apart (SBO).
__device__ __forceinline__ int op16(int r, int q, int Kp) {
  return (r >> 3) * (Kp * 8) + (q >> 3) * 64 + (r & 7) * 8 + (q & 7);
}

__device__ __forceinline__ void split_bf16(float v, uint16_t *hi, uint16_t *lo) {
  const __nv_bfloat16 h = __float2bfloat16_rn(v);
  const __nv_bfloat16 l = __float2bfloat16_rn(v - __bfloat162float(h));  // v - h is exact in FP32
  *hi = __bfloat16_as_ushort(h);
  *lo = __bfloat16_as_ushort(l);
}

__global__ void k_split_W_bf(const double *W, int npair, int Kp, int Np, uint16_t *out) {
  const int nb = Np * Kp;
  for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < nb; idx += gridDim.x * blockDim.x) {
    const int n = idx / Kp, k = idx - n * Kp;
    const double w = (n < npair && k < npair) ? W[(size_t)n * npair + k] : 0.0;
    const __nv_bfloat16 h = __double2bfloat16(w);
    const __nv_bfloat16 l = __double2bfloat16(w - (double)__bfloat162float(h));
    out[op16(n, k, Kp)] = __bfloat16_as_ushort(h);
    out[nb + op16(n, k, Kp)] = __bfloat16_as_ushort(l);
  }
}

// Half a row of D held in registers during the in-place split (Kp <= 144).
constexpr int kBfHalfMax = 72;

__global__ void __launch_bounds__(kBfThreads, 1)
    k_gather_contract_bf(SigmaArgs a, const uint16_t *Wbf, int Kp, int Np, uint32_t tmem_cols, int *status) {
  extern __shared__ __align__(128) unsigned char smem[];
  const int S = Kp + 1;                          // FP32 row stride of the gather buffer
  float *Dst = reinterpret_cast<float *>(smem);  // 128 x S FP32, then the BF16 operand A (hi, lo)
  uint16_t *Ahi = reinterpret_cast<uint16_t *>(smem);
  uint16_t *Alo = Ahi + kTcM * Kp;
  const size_t region = (size_t)kTcM * S * 4;  // >= 2 * 128 * Kp * 2 bytes of the operand
  uint16_t *Bhi = reinterpret_cast<uint16_t *>(smem + region);
  uint16_t *Blo = Bhi + Np * Kp;
  uint64_t *mbar = reinterpret_cast<uint64_t *>(Blo + Np * Kp);
  uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(mbar + 1);
  const uint32_t sAhi = smem_u32(Ahi), sAlo = smem_u32(Alo), sBhi = smem_u32(Bhi), sBlo = smem_u32(Blo);
  const uint32_t sbar = smem_u32(mbar);
  const int tid = threadIdx.x, warp = tid >> 5;
  const float *cin = a.cf;
  if (a.ctl) {
    if (a.ctl->halt) return;  // uniform: before any TMEM allocation or barrier
    cin = a.ctl->zf;
  }
  if (!cin || !Wbf) {  // no FP32 input or no operand B: refuse (uniform, before any allocation)
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
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(sbar) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  {  // operand B: a copy of the pre-split W (16-byte loads)
    const int nb = Np * Kp;  // BF16 elements per half, a multiple of 8
    const uint4 *src = reinterpret_cast<const uint4 *>(Wbf);
    uint4 *dst = reinterpret_cast<uint4 *>(Bhi);
    for (int i = tid; i < nb / 4; i += blockDim.x) dst[i] = __ldg(src + i);  // hi and lo halves
  }
  fence_async_smem();
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = *tmem_slot;
  const uint32_t idesc = idesc_bf16x(kTcM, Np);
  const uint32_t LBO = 128, SBO = (uint32_t)Kp * 16;
  float *G = reinterpret_cast<float *>(a.G);
  const int npair = a.npair;
  const int r = tid & (kTcM - 1), half = tid >> 7;
  const int hq = Kp / 2;  // a multiple of 8
  const int q0 = half * hq;
  const long long ntiles = (a.ndet + kTcM - 1) / kTcM;
  uint32_t phase = 0;
  bool ok = true;
  for (long long tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x) {
    const long long I = tile * kTcM + r;
    const bool valid = I < a.ndet;
    // 1. zero the FP32 rows (each thread half a row), then gather with atomic adds
    for (int q = q0; q < q0 + hq; ++q) Dst[r * S + q] = 0.f;
    if (half == 0 && r == 0) Dst[kTcM * S - 1] = 0.f;  // (the padding word past the last row's Kp)
    __syncthreads();
    if (valid) {
      int ia, ib;
      split_det(I, a.nb, ia, ib);
      float *row = Dst + r * S;
      if (half == 0) {
        const float *ccol = cin + ib;
        for_links_pipelined<8, float>(
            a.link_a + (size_t)ia * a.nlink_a, a.nlink_a, 1,
            [&](uint32_t v) { return __ldg(ccol + (size_t)link_J(v) * a.nb); },
            [&](uint32_t v, float f) { atomicAdd(row + link_pair(v), link_neg(v) ? -f : f); });
      } else {
        const float *crow = cin + (size_t)ia * a.nb;
        for_links_pipelined<8, float>(
            a.link_bT + ib, a.nlink_b, a.nb, [&](uint32_t v) { return __ldg(crow + link_J(v)); },
            [&](uint32_t v, float f) { atomicAdd(row + link_pair(v), link_neg(v) ? -f : f); });
      }
    }
    __syncthreads();
    // 2. in-place split: half a row into registers, barrier, BF16 hi / lo over the same bytes
    float v[kBfHalfMax];
#pragma unroll
    for (int j = 0; j < kBfHalfMax; ++j)
      if (j < hq) v[j] = Dst[r * S + q0 + j];
    __syncthreads();
#pragma unroll
    for (int j = 0; j < kBfHalfMax; j += 8) {
      if (j < hq) {
        uint16_t h[8], l[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) split_bf16(v[j + u], &h[u], &l[u]);
        const int off = op16(r, q0 + j, Kp);  // 8 consecutive K of one core-matrix row: 16 bytes
        *reinterpret_cast<uint4 *>(Ahi + off) =
            make_uint4(h[0] | (uint32_t)h[1] << 16, h[2] | (uint32_t)h[3] << 16, h[4] | (uint32_t)h[5] << 16,
                       h[6] | (uint32_t)h[7] << 16);
        *reinterpret_cast<uint4 *>(Alo + off) =
            make_uint4(l[0] | (uint32_t)l[1] << 16, l[2] | (uint32_t)l[3] << 16, l[4] | (uint32_t)l[5] << 16,
                       l[6] | (uint32_t)l[7] << 16);
      }
    }
    fence_async_smem();
    fence_before();
    __syncthreads();
    fence_after();
    // 3. three products per K step of 16, one issuing thread
    if (tid == 0) {
      for (int kk = 0; kk < Kp / 16; ++kk) {
        const uint32_t koff = (uint32_t)kk * 256;  // two K-adjacent core matrices of 8 BF16
        const uint64_t ah = smem_desc(sAhi + koff, LBO, SBO), al = smem_desc(sAlo + koff, LBO, SBO);
        const uint64_t bh = smem_desc(sBhi + koff, LBO, SBO), bl = smem_desc(sBlo + koff, LBO, SBO);
        mma_bf16x(tmem, ah, bh, idesc, kk > 0 ? 1u : 0u);
        mma_bf16x(tmem, ah, bl, idesc, 1u);
        mma_bf16x(tmem, al, bh, idesc, 1u);
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(sbar)
                   : "memory");
    }
    ok = mbar_wait(sbar, phase, kWaitIters);
    ok = __syncthreads_and(ok) != 0;
    if (!ok) break;
    phase ^= 1u;
    fence_after();
    // 4. epilogue: warp w reads lane quadrant w % 4, half of the columns
    const uint32_t lane_addr = tmem + ((uint32_t)((warp & 3) * 32) << 16);
    const int ncol16 = Np / 16;
    const int c_begin = (warp >> 2) * ((ncol16 + 1) / 2) * 16;
    const int c_end = (warp >> 2) ? Np : ((ncol16 + 1) / 2) * 16;
    const long long Ie = tile * kTcM + (warp & 3) * 32 + (tid & 31);
    for (int c0 = c_begin; c0 < c_end; c0 += 32) {
      uint32_t rr[32];
      tmem_ld16_nowait(lane_addr + (uint32_t)c0, rr);
      if (c0 + 16 < c_end) tmem_ld16_nowait(lane_addr + (uint32_t)(c0 + 16), rr + 16);
      asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
      if (Ie < a.ndet) {
#pragma unroll
        for (int j = 0; j < 32; ++j)
          if (c0 + j < c_end && c0 + j < npair) G[(size_t)(c0 + j) * a.ndet + Ie] = __uint_as_float(rr[j]);
      }
    }
    fence_before();
    __syncthreads();
    fence_after();
  }
  if (!ok) {
    if (tid == 0) atomicOr(status, 1);
    mbar_wait(sbar, phase, kWaitIters);  // let the outstanding MMAs drain (bounded)
  }
  fence_before();
  __syncthreads();
  fence_after();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(tmem_cols)
                 : "memory");
}

}  // namespace

bool bf_dims(int npair, int *Kp, int *Np, uint32_t *cols, size_t *smem) {
  const int kp = (npair + 15) / 16 * 16;
  const int np = (npair + 15) / 16 * 16;
  uint32_t c = 32;
  while (c < (uint32_t)np) c <<= 1;
  const size_t region = (size_t)kTcM * (kp + 1) * 4;
  const size_t bytes = region + (size_t)2 * np * kp * 2 + 16;
  *Kp = kp;
  *Np = np;
  *cols = c;
  *smem = bytes;
  return npair >= 1 && kp / 2 <= kBfHalfMax && np <= 256 && c <= 512 && bytes <= 227 * 1024;
}

int bf_grid(int npair, long long ndet, int num_sms) {
  int Kp, Np;
  uint32_t cols;
  size_t smem;
  if (!bf_dims(npair, &Kp, &Np, &cols, &smem)) return 0;
  int optin = 0;
  if (max_dynamic_smem((const void *)k_gather_contract_bf, &optin) != cudaSuccess || (int)smem > optin ||
      cudaFuncSetAttribute(k_gather_contract_bf, cudaFuncAttributeMaxDynamicSharedMemorySize, optin) !=
          cudaSuccess ||
      cudaFuncSetAttribute(k_gather_contract_bf, cudaFuncAttributePreferredSharedMemoryCarveout,
                           cudaSharedmemCarveoutMaxShared) != cudaSuccess)
    return 0;
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_gather_contract_bf, kBfThreads, smem) !=
          cudaSuccess ||
      per_sm < 1)
    per_sm = 1;
  if ((uint32_t)per_sm * cols > 512) per_sm = (int)(512 / cols);
  const long long ntiles = (ndet + kTcM - 1) / kTcM;
  long long grid = (long long)num_sms * per_sm;
  if (grid > ntiles) grid = ntiles;
  if (grid < 1) grid = 1;
  return (int)grid;
}

size_t bf_W_elems(int npair) {
  int Kp, Np;
  uint32_t cols;
  size_t smem;
  if (!bf_dims(npair, &Kp, &Np, &cols, &smem)) return 0;
  return (size_t)2 * Np * Kp;
}

cudaError_t launch_split_W_bf(const double *W, int npair, uint16_t *out, cudaStream_t s) {
  int Kp, Np;
  uint32_t cols;
  size_t smem;
  if (!bf_dims(npair, &Kp, &Np, &cols, &smem)) return cudaErrorInvalidValue;
  const int nb = Np * Kp;
  k_split_W_bf<<<(nb + 255) / 256, 256, 0, s>>>(W, npair, Kp, Np, out);
  return cudaGetLastError();
}

cudaError_t launch_gather_contract_bf(const SigmaArgs &a, const uint16_t *Wbf, int *status, int grid,
                                      cudaStream_t s) {
  int Kp, Np;
  uint32_t cols;
  size_t smem;
  if (!bf_dims(a.npair, &Kp, &Np, &cols, &smem) || grid < 1) return cudaErrorInvalidValue;
  k_gather_contract_bf<<<grid, kBfThreads, smem, s>>>(a, Wbf, Kp, Np, cols, status);
  return cudaGetLastError();
}

}  // namespace sbci
