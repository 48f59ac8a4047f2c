// Tensor-core (tcgen05) pieces of the TF32x3 gather + contract, shared by the
// one-solve kernel and the persistent batched kernel (kernels_loop.cu, which
// describes the scheme).  The tile arithmetic is additions, conversions and
// MMAs only (nothing a compiler could contract), so inlining cannot change it.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "ctl.h"
#include "sbci_internal.h"

namespace sbci {

constexpr int kTcM = 128;         // determinants per tile = MMA M = TMEM lanes
constexpr int kTcThreads = 256;   // two threads per determinant (alpha / beta links)
constexpr long long kWaitIters = 1LL << 22;

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ uint32_t tf32_bits(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return r;
}

// The same rounding (to nearest, ties away from zero) with two integer
// operations on the bit pattern: add half a TF32 unit to the magnitude bits
// and clear the 13 dropped bits (a carry into the exponent is the correct
// result).  For the finite values of the tile split.
__device__ __forceinline__ float tf32_round(float x) {
  return __uint_as_float((__float_as_uint(x) + 0x1000u) & 0xFFFFE000u);
}

// Shared-memory matrix descriptor: no swizzle, start/LBO/SBO in 16-byte units,
// descriptor version 1 (bit 46).
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
  d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1 << 46;
  return d;
}

// Instruction descriptor of kind::tf32: D = F32 (bits 4-5 = 1), A = B = TF32
// (format 2 at bits 7-9 and 10-12), both K-major, N >> 3 at bits 17-22,
// M >> 4 at bits 24-28.
__host__ __device__ constexpr uint32_t idesc_tf32(int M, int N) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_tf32(uint32_t tmem, uint64_t ad, uint64_t bd, uint32_t idesc,
                                         uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem),
      "l"(ad), "l"(bd), "r"(idesc), "r"(accumulate)
      : "memory");
}

__device__ __forceinline__ bool mbar_wait(uint32_t addr, uint32_t parity, long long iters) {
  for (long long i = 0; i < iters; ++i) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(done)
        : "r"(addr), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&r)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
      "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
}

// tcgen05.ld of 16 columns into r[0..15] without waiting (the caller waits).
__device__ __forceinline__ void tmem_ld16_nowait(uint32_t taddr, uint32_t *r) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
      "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
}

__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory"); }

// Float offset of element (r, q) in a K-major no-swizzle operand with Kp
// columns: core matrix (r/8, q/4) of 8 rows x 4 TF32 (128 bytes), K-adjacent
// core matrices 128 bytes apart (LBO), 8-row groups Kp*32 bytes apart (SBO).
__device__ __forceinline__ int opnd_off(int r, int q, int Kp) {
  return (r >> 3) * (Kp * 8) + (q >> 2) * 32 + (r & 7) * 4 + (q & 3);
}

// Shared-memory operand buffers of one CTA.
struct TcSmem {
  float *A, *Alo;
  uint32_t *Bhi, *Blo;
  uint32_t sA, sAlo, sBhi, sBlo, sbar;
};

// Element (n, k) of operand B: W split into TF32 hi/lo from FP64, zero
// outside npair x npair.
__device__ __forceinline__ void split_W_elem(const double *W, int npair, int n, int k, uint32_t *hi,
                                             uint32_t *lo) {
  const double w = (n < npair && k < npair) ? W[(size_t)n * npair + k] : 0.0;
  const uint32_t h = tf32_bits((float)w);
  *hi = h;
  *lo = tf32_bits((float)(w - (double)__uint_as_float(h)));
}

// Operand B into shared memory, zero-padded to Np x Kp: a copy of the
// pre-split operand when the context has one (a.Wtc), else split here from
// FP64 (same values); ends with the fences that publish it to the tensor core.
__device__ __forceinline__ void tc_load_B(const SigmaArgs &a, int Kp, int Np, const TcSmem &sm) {
  const int nb = Np * Kp;
  if (a.Wtc) {
    const uint4 *src_hi = reinterpret_cast<const uint4 *>(a.Wtc);
    const uint4 *src_lo = reinterpret_cast<const uint4 *>(a.Wtc + nb);
    uint4 *dhi = reinterpret_cast<uint4 *>(sm.Bhi), *dlo = reinterpret_cast<uint4 *>(sm.Blo);
    for (int i = threadIdx.x; i < nb / 4; i += blockDim.x) {
      dhi[i] = __ldg(src_hi + i);
      dlo[i] = __ldg(src_lo + i);
    }
  } else {
    for (int idx = threadIdx.x; idx < nb; idx += blockDim.x) {
      const int n = idx / Kp, k = idx - n * Kp;
      split_W_elem(a.W, a.npair, n, k, &sm.Bhi[opnd_off(n, k, Kp)], &sm.Blo[opnd_off(n, k, Kp)]);
    }
  }
  fence_async_smem();
  fence_before();
  __syncthreads();
  fence_after();
}

// The barrier of the threads that gather a tile: the whole CTA, or (kAll =
// false) the first 256 threads on named barrier 1, in a CTA whose other warps
// have work of their own.
template <bool kAll>
__device__ __forceinline__ void tc_sync() {
  if (kAll) __syncthreads();
  else asm volatile("bar.sync 1, 256;\n" ::: "memory");
}

// Steps 1 and 2 of a tile, row (threadIdx.x % 128) of D for determinant I
// (a zero row when !valid): the gather in FP32, the alpha part into A and the
// beta part into Alo (free until the split), each row owned by one thread;
// then D = alpha part + beta part split in place, A <- tf32(D) and
// Alo <- tf32(D - tf32(D)), each thread half a row.  256 threads, whose
// barrier is tc_sync<kAll>.  Ends with the fences and the barrier that hand
// the operand to the tensor core.
template <bool kAll = true>
__device__ __forceinline__ void tc_gather_split(const SigmaArgs &a, const float *cin, long long I, bool valid,
                                                int Kp, const TcSmem &sm) {
  const int tid = threadIdx.x;
  float *A = sm.A, *Alo = sm.Alo;
  const int row = tid & (kTcM - 1);  // determinant row of this thread
  const int half = tid >> 7;         // 0: alpha links / first half, 1: beta links / second half
  const int q_lo = half ? (Kp / 8) * 4 : 0, q_hi = half ? Kp : (Kp / 8) * 4;
  float *mine = half ? Alo : A;
  for (int q = 0; q < Kp; q += 4)
    *reinterpret_cast<float4 *>(mine + opnd_off(row, q, Kp)) = make_float4(0.f, 0.f, 0.f, 0.f);
  if (valid) {
    int ia, ib;
    split_det(I, a.nb, ia, ib);
    if (half == 0) {
      const uint32_t *la = a.link_a + (size_t)ia * a.nlink_a;
      const float *ccol = cin + ib;
      for_links_pipelined<8, float>(
          la, a.nlink_a, 1, [&](uint32_t v) { return __ldg(ccol + (size_t)link_J(v) * a.nb); },
          [&](uint32_t v, float f) {
            mine[opnd_off(row, link_pair(v), Kp)] += link_neg(v) ? -f : f;
          });
    } else {
      const uint32_t *lb = a.link_bT + ib;
      const float *crow = cin + (size_t)ia * a.nb;
      for_links_pipelined<8, float>(
          lb, a.nlink_b, a.nb, [&](uint32_t v) { return __ldg(crow + link_J(v)); },
          [&](uint32_t v, float f) {
            mine[opnd_off(row, link_pair(v), Kp)] += link_neg(v) ? -f : f;
          });
    }
  }
  tc_sync<kAll>();
  for (int q = q_lo; q < q_hi; q += 4) {
    float4 *p = reinterpret_cast<float4 *>(A + opnd_off(row, q, Kp));
    float4 *pl = reinterpret_cast<float4 *>(Alo + opnd_off(row, q, Kp));
    const float4 va = *p, vb = *pl;
    const float4 v = make_float4(va.x + vb.x, va.y + vb.y, va.z + vb.z, va.w + vb.w);
    float4 h, l;
    h.x = tf32_round(v.x);
    h.y = tf32_round(v.y);
    h.z = tf32_round(v.z);
    h.w = tf32_round(v.w);
    l.x = tf32_round(v.x - h.x);
    l.y = tf32_round(v.y - h.y);
    l.z = tf32_round(v.z - h.z);
    l.w = tf32_round(v.w - h.w);
    *p = h;
    *pl = l;
  }
  fence_async_smem();
  fence_before();
  tc_sync<kAll>();
  fence_after();
}

// Epilogue of a tile: the 128 x Np FP32 accumulator at TMEM column acc into
// G[P][I] (P < npair, valid rows only); warp w reads lane quadrant (w % 4)
// and column half (w / 4).  256 threads.
__device__ __forceinline__ void tc_store_G(const SigmaArgs &a, uint32_t acc, long long I, bool valid, int Np) {
  const int warp = threadIdx.x >> 5;
  float *G = reinterpret_cast<float *>(a.G);
  const uint32_t lane_addr = acc + ((uint32_t)((warp & 3) * 32) << 16);
  const int ncol16 = Np / 16;
  const int c_begin = (warp >> 2) * ((ncol16 + 1) / 2) * 16;
  const int c_end = (warp >> 2) ? Np : ((ncol16 + 1) / 2) * 16;
  for (int c0 = c_begin; c0 < c_end; c0 += 32) {
    // up to two 16-column loads in flight before one wait
    uint32_t r[32];
    tmem_ld16_nowait(lane_addr + (uint32_t)c0, r);
    if (c0 + 16 < c_end) tmem_ld16_nowait(lane_addr + (uint32_t)(c0 + 16), r + 16);
    asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
    if (valid) {
#pragma unroll
      for (int j = 0; j < 32; ++j)
        if (c0 + j < c_end && c0 + j < a.npair) G[(size_t)(c0 + j) * a.ndet + I] = __uint_as_float(r[j]);
    }
  }
}

// One tile of 128 determinants: gather, split, three MMAs per K step, bounded
// wait, epilogue into G.  256 threads.  Returns false (block-uniformly) if
// the MMA-completion wait ran out.
// cin: the FP32 copy of the input vector (written by its producer, or by a
// conversion before a plain sigma call).
__device__ __forceinline__ bool tc_tile(const SigmaArgs &a, const float *cin, long long tile, int Kp, int Np,
                                        const TcSmem &sm, uint32_t tmem, uint32_t &phase) {
  const int tid = threadIdx.x;
  const uint32_t sA = sm.sA, sAlo = sm.sAlo, sBhi = sm.sBhi, sBlo = sm.sBlo, sbar = sm.sbar;
  const uint32_t idesc = idesc_tf32(kTcM, Np);
  const uint32_t LBO = 128, SBO = (uint32_t)Kp * 32;
  const long long I = tile * kTcM + (tid & (kTcM - 1));
  const bool valid = I < a.ndet;
  // 1-2. D gathered and split into A / Alo
  tc_gather_split(a, cin, I, valid, Kp, sm);
  // 3. three products per K step, one issuing thread
  if (tid == 0) {
    for (int kk = 0; kk < Kp / 8; ++kk) {
      const uint32_t koff = (uint32_t)kk * 256;  // two K-adjacent core matrices
      const uint64_t ah = smem_desc(sA + koff, LBO, SBO), al = smem_desc(sAlo + koff, LBO, SBO);
      const uint64_t bh = smem_desc(sBhi + koff, LBO, SBO), bl = smem_desc(sBlo + koff, LBO, SBO);
      mma_tf32(tmem, ah, bh, idesc, kk > 0 ? 1u : 0u);
      mma_tf32(tmem, ah, bl, idesc, 1u);
      mma_tf32(tmem, al, bh, idesc, 1u);
    }
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(sbar)
                 : "memory");
  }
  bool ok = mbar_wait(sbar, phase, kWaitIters);
  ok = __syncthreads_and(ok) != 0;
  if (!ok) return false;
  phase ^= 1u;
  fence_after();
  // 4. epilogue
  tc_store_G(a, tmem, I, valid, Np);
  fence_before();
  __syncthreads();
  fence_after();
  return true;
}

}  // namespace sbci
