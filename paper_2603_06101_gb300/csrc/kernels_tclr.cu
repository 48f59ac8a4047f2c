// Density-fitted (factored) TF32x3 gather + contract on the tensor cores.
//
// With density-fitted two-electron integrals the packed operator factors as
// W = F M F^T (lowrank.h: F = [L | kappa | delta] from a pivoted Cholesky of
// the pair matrix plus the one-electron part, rank r + 2), so a tile's
// G = D W is two chained products (the density-fitted contraction written as
// GEMMs, T = D F then G = T (F M)^T, M symmetric):
//   1. D gathered and split into TF32 hi / lo exactly as in the full-form
//      kernel (tc_gather_split);
//   2. T = D F, (128 x Kp) x (Kp x Rp), tcgen05 kind::tf32 with the TF32x3
//      terms hi.hi + hi.lo + lo.hi into TMEM accumulator 1;
//   3. T read back (tcgen05.ld), split into TF32 hi / lo and stored as the
//      K-major operand (128 x Rp) over the D buffers, which step 2 has
//      finished reading;
//   4. G = T (F M)^T, (128 x Rp) x (Rp x Np), the same three terms into TMEM
//      accumulator 2;
//   5. the full-form epilogue writes G[P][I] (tc_store_G).
// Tensor work per determinant is 2 (Kp Rp + Rp Np) products instead of
// 2 Kp Np (for the factor's rank r + 2 < 0.45 npair, Rp <= Kp / 2 + 16), and
// the operands take less shared memory: at n = 15 (npair = 120) the full
// TF32 operands exceed it and the factored ones fit.  Precision: T carries
// the FP32 rounding of its accumulation and of its TF32x3 re-split, the same
// order as the rounding of G itself.
#include <cuda_runtime.h>
#include <stdint.h>

#include "sbci_internal.h"
#include "tc_body.cuh"

namespace sbci {

namespace {

// TMEM column of accumulator 2: the power of two at or above Rp (accumulators
// start on 32-column boundaries).
__host__ __device__ constexpr int lr_acc2(int Rp) { return Rp <= 32 ? 32 : Rp <= 64 ? 64 : 128; }

// Shared-memory buffers: the D / T operand (hi, lo), then the pre-split
// factor operands B1 = F^T [Rp][Kp] and B2 = (F M) [Np][Rp] (hi, lo each, in
// one contiguous block, the layout of the context's copy), then the mbarrier
// and the TMEM address slot.
struct LrSmem {
  TcSmem t;  // A, Alo (D, then T) and the mbarrier; t.Bhi / t.Blo unused
  uint32_t *B;  // B1 hi, B1 lo, B2 hi, B2 lo
  uint32_t sB1hi, sB1lo, sB2hi, sB2lo;
  uint32_t *tmem_slot;
};

__device__ __forceinline__ LrSmem lr_carve(unsigned char *smem, int Kp, int Np, int Rp) {
  LrSmem s;
  s.t.A = reinterpret_cast<float *>(smem);
  s.t.Alo = s.t.A + kTcM * Kp;
  s.t.Bhi = s.t.Blo = nullptr;
  s.B = reinterpret_cast<uint32_t *>(s.t.Alo + kTcM * Kp);
  uint64_t *mbar = reinterpret_cast<uint64_t *>(s.B + 2 * Rp * Kp + 2 * Np * Rp);
  s.tmem_slot = reinterpret_cast<uint32_t *>(mbar + 1);
  s.t.sA = smem_u32(s.t.A);
  s.t.sAlo = smem_u32(s.t.Alo);
  s.t.sBhi = s.t.sBlo = 0;
  s.sB1hi = smem_u32(s.B);
  s.sB1lo = s.sB1hi + (uint32_t)(Rp * Kp) * 4;
  s.sB2hi = s.sB1lo + (uint32_t)(Rp * Kp) * 4;
  s.sB2lo = s.sB2hi + (uint32_t)(Np * Rp) * 4;
  s.t.sbar = smem_u32(mbar);
  return s;
}

// Three TF32x3 products per K step of 8, one issuing thread, then a commit
// to the mbarrier.  SBO of both operands: their K extent x 32 bytes.
__device__ __forceinline__ void lr_mma(uint32_t acc, uint32_t sAh, uint32_t sAl, uint32_t sBh, uint32_t sBl, int K,
                                       uint32_t idesc, uint32_t sbar) {
  const uint32_t LBO = 128, SBO = (uint32_t)K * 32;
  for (int kk = 0; kk < K / 8; ++kk) {
    const uint32_t koff = (uint32_t)kk * 256;  // two K-adjacent core matrices
    const uint64_t ah = smem_desc(sAh + koff, LBO, SBO), al = smem_desc(sAl + koff, LBO, SBO);
    const uint64_t bh = smem_desc(sBh + koff, LBO, SBO), bl = smem_desc(sBl + koff, LBO, SBO);
    mma_tf32(acc, ah, bh, idesc, kk > 0 ? 1u : 0u);
    mma_tf32(acc, ah, bl, idesc, 1u);
    mma_tf32(acc, al, bh, idesc, 1u);
  }
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(sbar)
               : "memory");
}

// Bounded wait for the last commit; block-uniform result.
__device__ __forceinline__ bool lr_wait(uint32_t sbar, uint32_t &phase) {
  bool ok = mbar_wait(sbar, phase, kWaitIters);
  ok = __syncthreads_and(ok) != 0;
  if (ok) {
    phase ^= 1u;
    fence_after();
  }
  return ok;
}

__device__ __forceinline__ bool lr_tile(const SigmaArgs &a, const float *cin, long long tile, int Kp, int Np,
                                        int Rp, const LrSmem &sm, uint32_t tmem, uint32_t &phase) {
  const int tid = threadIdx.x, warp = tid >> 5;
  const long long I = tile * kTcM + (tid & (kTcM - 1));
  const bool valid = I < a.ndet;
  const uint32_t acc2 = tmem + (uint32_t)lr_acc2(Rp);
  // 1. D
  tc_gather_split(a, cin, I, valid, Kp, sm.t);
  // 2. T = D F
  if (tid == 0) lr_mma(tmem, sm.t.sA, sm.t.sAlo, sm.sB1hi, sm.sB1lo, Kp, idesc_tf32(kTcM, Rp), sm.t.sbar);
  if (!lr_wait(sm.t.sbar, phase)) return false;
  // 3. T -> TF32 hi / lo operand [128][Rp] over A / Alo; warp w reads lane
  //    quadrant w % 4 and every other 16-column group from w / 4
  {
    const int lrow = (warp & 3) * 32 + (tid & 31);
    const uint32_t lane_addr = tmem + ((uint32_t)((warp & 3) * 32) << 16);
    for (int g = warp >> 2; g < Rp / 16; g += 2) {
      uint32_t v[16];
      tmem_ld16(lane_addr + (uint32_t)(g * 16), v);
#pragma unroll
      for (int j = 0; j < 16; j += 4) {
        float4 h, l;
        const float t0 = __uint_as_float(v[j]), t1 = __uint_as_float(v[j + 1]);
        const float t2 = __uint_as_float(v[j + 2]), t3 = __uint_as_float(v[j + 3]);
        h.x = tf32_round(t0);
        h.y = tf32_round(t1);
        h.z = tf32_round(t2);
        h.w = tf32_round(t3);
        l.x = tf32_round(t0 - h.x);
        l.y = tf32_round(t1 - h.y);
        l.z = tf32_round(t2 - h.z);
        l.w = tf32_round(t3 - h.w);
        const int off = opnd_off(lrow, g * 16 + j, Rp);
        *reinterpret_cast<float4 *>(sm.t.A + off) = h;
        *reinterpret_cast<float4 *>(sm.t.Alo + off) = l;
      }
    }
  }
  fence_async_smem();
  fence_before();
  __syncthreads();
  fence_after();
  // 4. G = T (F M)^T
  if (tid == 0) lr_mma(acc2, sm.t.sA, sm.t.sAlo, sm.sB2hi, sm.sB2lo, Rp, idesc_tf32(kTcM, Np), sm.t.sbar);
  if (!lr_wait(sm.t.sbar, phase)) return false;
  // 5. epilogue
  tc_store_G(a, acc2, I, valid, Np);
  fence_before();
  __syncthreads();
  fence_after();
  return true;
}

__global__ void __launch_bounds__(kTcThreads, 1)
    k_gather_contract_tclr(SigmaArgs a, const uint32_t *Wlr, int Kp, int Np, int Rp, uint32_t tmem_cols,
                           int *status) {
  extern __shared__ __align__(128) unsigned char smem[];
  const LrSmem sm = lr_carve(smem, Kp, Np, Rp);
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
                     smem_u32(sm.tmem_slot)),
                 "r"(tmem_cols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(sm.t.sbar) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  {  // the factor operands (16-byte copies: every block is a multiple of 4 words)
    const int nw = 2 * Rp * Kp + 2 * Np * Rp;
    const uint4 *src = reinterpret_cast<const uint4 *>(Wlr);
    uint4 *dst = reinterpret_cast<uint4 *>(sm.B);
    for (int i = tid; i < nw / 4; i += blockDim.x) dst[i] = __ldg(src + i);
  }
  fence_async_smem();
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = *sm.tmem_slot;
  const long long ntiles = (a.ndet + kTcM - 1) / kTcM;
  uint32_t phase = 0;
  bool ok = true;
  for (long long tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x)
    ok = lr_tile(a, cin, tile, Kp, Np, Rp, sm, tmem, phase);
  if (!ok) {
    if (tid == 0) atomicOr(status, 1);
    mbar_wait(sm.t.sbar, phase, kWaitIters);  // let the outstanding MMAs drain (bounded)
  }
  fence_before();
  __syncthreads();
  fence_after();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(tmem_cols)
                 : "memory");
}

// TF32 hi / lo words of w (the full-form operand's split).
__device__ __forceinline__ void lr_split(double w, uint32_t *hi, uint32_t *lo) {
  const uint32_t h = tf32_bits((float)w);
  *hi = h;
  *lo = tf32_bits((float)(w - (double)__uint_as_float(h)));
}

// B1[n][k] = F^T[n][k] = Ut[n][k] (n < rr, k < npair), B2[n][k] = (F M)[n][k]
// = UL[n][k] (n < npair, k < rr), zero-padded, in the K-major operand layout.
__global__ void k_split_lr_tc(const double *Ut, const double *UL, int rr, int npair, int Kp, int Np, int Rp,
                              uint32_t *out) {
  const int n1 = Rp * Kp, n2 = Np * Rp;
  uint32_t *b1h = out, *b1l = out + n1, *b2h = out + 2 * n1, *b2l = out + 2 * n1 + n2;
  for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < n1 + n2; idx += gridDim.x * blockDim.x) {
    if (idx < n1) {
      const int n = idx / Kp, k = idx - n * Kp;
      const double w = (n < rr && k < npair) ? Ut[(size_t)n * npair + k] : 0.0;
      lr_split(w, &b1h[opnd_off(n, k, Kp)], &b1l[opnd_off(n, k, Kp)]);
    } else {
      const int j = idx - n1, n = j / Rp, k = j - n * Rp;
      const double w = (n < npair && k < rr) ? UL[(size_t)n * rr + k] : 0.0;
      lr_split(w, &b2h[opnd_off(n, k, Rp)], &b2l[opnd_off(n, k, Rp)]);
    }
  }
}

}  // namespace

bool tclr_dims(int npair, int rr, int *Kp, int *Np, int *Rp, uint32_t *cols, size_t *smem) {
  if (npair < 1 || rr < 1) return false;
  const int kp = (npair + 7) / 8 * 8;
  const int np = (npair + 15) / 16 * 16;
  const int rp = (rr + 15) / 16 * 16;
  uint32_t c = 32;
  while (c < (uint32_t)(lr_acc2(rp) + np)) c <<= 1;
  const size_t bytes = (size_t)(2 * kTcM * kp + 2 * rp * kp + 2 * np * rp) * 4 + 16;
  *Kp = kp;
  *Np = np;
  *Rp = rp;
  *cols = c;
  *smem = bytes;
  // T is stored over the D buffers (Rp <= Kp); N of each product <= 256
  return rp <= kp && rp <= 128 && np <= 256 && c <= 512 && bytes <= 227 * 1024;
}

size_t tclr_W_words(int npair, int rr) {
  int Kp, Np, Rp;
  uint32_t cols;
  size_t smem;
  if (!tclr_dims(npair, rr, &Kp, &Np, &Rp, &cols, &smem)) return 0;
  return (size_t)(2 * Rp * Kp + 2 * Np * Rp);
}

cudaError_t launch_split_lr_tc(const double *Ut, const double *UL, int rr, int npair, uint32_t *out,
                               cudaStream_t s) {
  int Kp, Np, Rp;
  uint32_t cols;
  size_t smem;
  if (!tclr_dims(npair, rr, &Kp, &Np, &Rp, &cols, &smem)) return cudaErrorInvalidValue;
  const int n = Rp * Kp + Np * Rp;
  k_split_lr_tc<<<(n + 255) / 256, 256, 0, s>>>(Ut, UL, rr, npair, Kp, Np, Rp, out);
  return cudaGetLastError();
}

int tclr_grid(int npair, int rr, long long ndet, int num_sms) {
  int Kp, Np, Rp;
  uint32_t cols;
  size_t smem;
  if (!tclr_dims(npair, rr, &Kp, &Np, &Rp, &cols, &smem)) return 0;
  int optin = 0;
  const void *f = (const void *)k_gather_contract_tclr;
  if (max_dynamic_smem(f, &optin) != cudaSuccess || (int)smem > optin ||
      cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, optin) != cudaSuccess ||
      cudaFuncSetAttribute(f, cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared) !=
          cudaSuccess)
    return 0;
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, f, kTcThreads, smem) != cudaSuccess) return 0;
  if ((uint32_t)per_sm * cols > 512) per_sm = (int)(512 / cols);
  if (per_sm < 1) return 0;
  const long long ntiles = (ndet + kTcM - 1) / kTcM;
  long long grid = (long long)num_sms * per_sm;
  if (grid > ntiles) grid = ntiles;
  if (grid < 1) grid = 1;
  return (int)grid;
}

cudaError_t launch_gather_contract_tclr(const SigmaArgs &a, const uint32_t *Wlr, int rr, int *status, int grid,
                                        cudaStream_t s) {
  int Kp, Np, Rp;
  uint32_t cols;
  size_t smem;
  if (!Wlr || !tclr_dims(a.npair, rr, &Kp, &Np, &Rp, &cols, &smem) || grid < 1) return cudaErrorInvalidValue;
  k_gather_contract_tclr<<<grid, kTcThreads, smem, s>>>(a, Wlr, Kp, Np, Rp, cols, status);
  return cudaGetLastError();
}

}  // namespace sbci
