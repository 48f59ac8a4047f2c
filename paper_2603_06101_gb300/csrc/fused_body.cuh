// Column-fused sigma of the singlet sector (c = c^T, the same strings for
// both spins), TF32x3 on the tensor cores, shared by the one-solve kernel and
// the persistent batched kernel (kernels_loop.cu).
//
// The sector sigma is sigma = A + A^T with A the alpha part,
//   A[Ia, Ib] = sum over the alpha links (P, Ja, s) of Ia of s * G[P][Ja, Ib],
//   G[P][Ja, Ib] = sum_Q W[P, Q] D[Q][Ja, Ib],
// and D the gathered excitations of z (both spins).  For one column Ib = b,
// A[., b] needs G[., ., b] only, so one CTA builds the whole column without
// writing G to global memory:
//   1. D[Q][Ia, b] for every Ia: the alpha part reads row b of z, staged in
//      shared memory (z[Ja, b] = z[b, Ja]); the beta part reads, for each link
//      (Q, Jb, s) of b, row Jb of z at column Ia (z[Ia, Jb] = z[Jb, Ia]), a
//      coalesced load across the threads of a warp;
//   2. G^T = D_hi W_hi + D_hi W_lo + D_lo W_hi by tcgen05 kind::tf32 into TMEM,
//      one 128-string tile of Ia at a time (two accumulators for Na <= 256);
//   3. the epilogue writes G[P][Ia, b] into shared memory, over the operand
//      buffers the MMAs have finished reading;
//   4. the alpha-only scatter of the column reads G from shared memory and
//      writes A[Ia, b] as row b of A^T (coalesced).  The symmetric finish
//      forms sigma = A^T + A, which is the same matrix.
// D, the split, the MMAs and the scatter's summation order are those of the
// tile kernel (tc_tile) and of the alpha-only scatter (scatter_body), so the
// column kernel gives the same A (up to the sign of zero: the gathers store
// each pair's single term where the tile kernel adds it to zero).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "sbci_internal.h"
#include "tc_body.cuh"

namespace sbci {

constexpr int kFcThreads = 512;  // four threads per string of a 128-string tile
constexpr int kFcMaxStr = 256;   // strings per spin (two tiles of the MMA's M = 128)
constexpr int kFcMaxLink = 64;   // link words of string b staged in shared memory
constexpr int kFcLinkMax = 8192; // 16-bit alpha link words of a space held in shared memory (na * nlink_a)

// Shared-memory buffers of one column CTA.
struct FcSmem {
  float *A, *Alo;       // operand D (alpha part / hi, beta part / lo); G column after the MMAs
  uint32_t *Bhi, *Blo;  // W split into TF32 hi / lo (operand B)
  float *zrow;          // row b of z, kFcMaxStr floats
  uint32_t *lb;         // links of string b, decoded: J * nb | operand column offset << 16 | sign << 31
  uint16_t *la;         // the space's alpha links, J | pair << 8 | sign << 15 (kFcLinkMax)
  uint32_t sA, sAlo, sBhi, sBlo, sbar;
};

// TMEM column offset of the second tile's accumulator: the power of two at or
// above Np (each accumulator starts on a 32-column boundary); a column CTA
// allocates twice that.
__host__ __device__ constexpr int fc_acc_stride(int Np) {
  return Np <= 32 ? 32 : Np <= 64 ? 64 : Np <= 128 ? 128 : 256;
}

// Dynamic shared memory of a column CTA with Kp x Np operands.
__host__ __device__ constexpr size_t fc_smem_bytes(int Kp, int Np) {
  return (size_t)(2 * kTcM * Kp + 2 * Np * Kp + kFcMaxStr + kFcMaxLink) * 4 + (size_t)kFcLinkMax * 2 + 16;
}

__device__ __forceinline__ FcSmem fc_carve(unsigned char *smem, int Kp, int Np) {
  FcSmem sm;
  sm.A = reinterpret_cast<float *>(smem);
  sm.Alo = sm.A + kTcM * Kp;
  sm.Bhi = reinterpret_cast<uint32_t *>(sm.Alo + kTcM * Kp);
  sm.Blo = sm.Bhi + Np * Kp;
  sm.zrow = reinterpret_cast<float *>(sm.Blo + Np * Kp);
  sm.lb = reinterpret_cast<uint32_t *>(sm.zrow + kFcMaxStr);
  sm.sA = smem_u32(sm.A);
  sm.sAlo = smem_u32(sm.Alo);
  sm.sBhi = smem_u32(sm.Bhi);
  sm.sBlo = smem_u32(sm.Blo);
  sm.la = reinterpret_cast<uint16_t *>(sm.lb + kFcMaxLink);
  sm.sbar = smem_u32(sm.la + kFcLinkMax);  // 8-byte aligned: every buffer above is a multiple of 8 bytes
  return sm;
}

// The TMEM address slot, after the mbarrier.
__device__ __forceinline__ uint32_t *fc_tmem_slot(const FcSmem &sm) {
  return reinterpret_cast<uint32_t *>(sm.la + kFcLinkMax) + 2;
}

// The space's alpha links into shared memory (16-byte copies; when a CTA
// starts a solve).  Ends with a barrier.
__device__ __forceinline__ void fc_load_links(const SigmaArgs &a, const FcSmem &sm) {
  const int nw = a.na * a.nlink_a;  // 16-bit words, <= kFcLinkMax
  const uint16_t *src = a.fc_link_a;
  for (int i = threadIdx.x; i < nw; i += blockDim.x) sm.la[i] = __ldg(src + i);
  __syncthreads();
}

// x with the sign flipped where bit 15 of the link word w is set.
__device__ __forceinline__ float fc_sign(float x, uint32_t w) {
  return __uint_as_float(__float_as_uint(x) ^ ((w & 0x8000u) << 16));
}

// Offset of column q within a row of the K-major no-swizzle TF32 operand (the
// row's own part is (r / 8) * Kp * 8 + (r % 8) * 4, see opnd_off).
__device__ __forceinline__ int fc_qoff(int q) { return (q >> 2) * 32 + (q & 3); }

// The tile kernel's operand B loader, on the column CTA's buffers.
__device__ __forceinline__ void fc_load_B(const SigmaArgs &a, int Kp, int Np, const FcSmem &fm) {
  TcSmem t;
  t.A = fm.A;
  t.Alo = fm.Alo;
  t.Bhi = fm.Bhi;
  t.Blo = fm.Blo;
  t.sA = fm.sA;
  t.sAlo = fm.sAlo;
  t.sBhi = fm.sBhi;
  t.sBlo = fm.sBlo;
  t.sbar = fm.sbar;
  tc_load_B(a, Kp, Np, t);
}

// Bounded wait for the MMAs of the last commit; block-uniform result.
__device__ __forceinline__ bool fc_wait(const FcSmem &sm, uint32_t &phase) {
  bool ok = mbar_wait(sm.sbar, phase, kWaitIters);
  ok = __syncthreads_and(ok) != 0;
  if (ok) {
    phase ^= 1u;
    fence_after();
  }
  return ok;
}

// One column b of A (written as row b of A^T into a.symA).  kFcThreads =
// 512 threads, four per string of a 128-string tile: two take halves of its
// alpha links, two halves of the column's beta links (a string's links have
// distinct pairs, so the four write disjoint slots).  TMEM holds two
// accumulators of Np columns, at tmem and tmem + fc_acc_stride(Np).  Returns
// false (block-uniformly) if an MMA-completion wait ran out; *pending is then
// 1 when a commit is still outstanding.
__device__ __forceinline__ bool fc_column(const SigmaArgs &a, const float *zf, int b, int Kp, int Np,
                                          const FcSmem &sm, uint32_t tmem, uint32_t &phase, int *pending) {
  const int tid = threadIdx.x, warp = tid >> 5;
  const int na = a.na, nb = a.nb, npair = a.npair;
  const int ntile = (na + kTcM - 1) / kTcM;
  const uint32_t idesc = idesc_tf32(kTcM, Np);
  const uint32_t LBO = 128, SBO = (uint32_t)Kp * 32;
  // 0. row b of z (z[b][j] = z[j][b]) and the decoded links of b; the previous
  //    column's readers of these buffers finished at its last barrier
  for (int j = tid; j < na; j += blockDim.x) sm.zrow[j] = __ldg(zf + (size_t)b * nb + j);
  for (int e = tid; e < a.nlink_b; e += blockDim.x) {  // J * nb < 2^16 for nb <= 256
    const uint32_t v = __ldg(a.link_b + (size_t)b * a.nlink_b + e);
    sm.lb[e] = (uint32_t)link_J(v) * (uint32_t)nb | (uint32_t)fc_qoff(link_pair(v)) << 16 | (v & kSignBit);
  }
  __syncthreads();
  const int r = tid & (kTcM - 1);
  const int part = tid >> 7;      // 0, 1: alpha link halves; 2, 3: beta link halves
  const bool beta = part >= 2;
  const int sub = part & 1;
  const int rbase = (r >> 3) * (Kp * 8) + (r & 7) * 4;  // row r's part of an operand offset
  const int nla = a.nlink_a, nlb = a.nlink_b;
  const int nl = beta ? nlb : nla, hl = (nl + 1) / 2;
  const int e0 = sub ? hl : 0, e1 = sub ? nl : hl;        // this thread's links
  const int nch = Kp / 4, cq = (nch + 3) / 4;            // float4 chunks of a row, per part
  const int c0 = part * cq, c1 = min(nch, c0 + cq);       // this thread's chunks of the split
  constexpr int kPre = 8;  // beta-link values loaded before the previous tile's MMAs are waited for
  for (int t = 0; t < ntile; ++t) {
    const int ia = t * kTcM + r;
    const bool row_ok = ia < na;
    const float *zc = zf + ia;
    const uint32_t *lw = sm.lb;
    float pre[kPre];
    if (beta && row_ok) {  // their z loads overlap the wait below
#pragma unroll
      for (int j = 0; j < kPre; ++j)
        if (e0 + j < e1) pre[j] = __ldg(zc + (lw[e0 + j] & 0xFFFFu));
    }
    if (t > 0) {  // the previous tile's MMAs read A / Alo: wait before overwriting them
      *pending = 1;
      if (!fc_wait(sm, phase)) return false;
      *pending = 0;
    }
    float *mine = beta ? sm.Alo : sm.A;
    {  // zero this thread's half of its row of its buffer
      const int qh = (Kp / 8) * 4;
      for (int q = sub ? qh : 0; q < (sub ? Kp : qh); q += 4)
        *reinterpret_cast<float4 *>(mine + opnd_off(r, q, Kp)) = make_float4(0.f, 0.f, 0.f, 0.f);
    }
    __syncthreads();  // both halves of a row are zero before either writes its terms
    // each pair receives at most one term per spin (a string's links have
    // distinct pairs), so the gathers store into the zeroed rows
    if (row_ok) {
      if (!beta) {  // all operands in shared memory
        const uint16_t *lr = sm.la + ia * nla;
        const float *zr = sm.zrow;
#pragma unroll 4
        for (int e = e0; e < e1; ++e) {
          const uint32_t w = lr[e];
          mine[rbase + fc_qoff((int)((w >> 8) & 0x7Fu))] = fc_sign(zr[w & 0xFFu], w);
        }
      } else {  // z rows of the column's beta links: coalesced loads
#pragma unroll
        for (int j = 0; j < kPre; ++j)
          if (e0 + j < e1) {
            const uint32_t w = lw[e0 + j];
            mine[rbase + (int)((w >> 16) & 0x7FFFu)] = __uint_as_float(__float_as_uint(pre[j]) ^ (w & kSignBit));
          }
        for (int e = e0 + kPre; e < e1; e += 8) {
          float f[8];
#pragma unroll
          for (int j = 0; j < 8; ++j)
            if (e + j < e1) f[j] = __ldg(zc + (lw[e + j] & 0xFFFFu));
#pragma unroll
          for (int j = 0; j < 8; ++j)
            if (e + j < e1) {
              const uint32_t w = lw[e + j];
              mine[rbase + (int)((w >> 16) & 0x7FFFu)] = __uint_as_float(__float_as_uint(f[j]) ^ (w & kSignBit));
            }
        }
      }
    }
    __syncthreads();
    // D = alpha + beta part, split in place into TF32 hi (A) and lo (Alo);
    // each thread a quarter of its row's float4 chunks
    for (int ch = c0; ch < c1; ++ch) {
      const int q = ch * 4;
      float4 *p = reinterpret_cast<float4 *>(sm.A + opnd_off(r, q, Kp));
      float4 *pl = reinterpret_cast<float4 *>(sm.Alo + opnd_off(r, q, Kp));
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
    __syncthreads();
    fence_after();
    if (tid == 0) {
      const uint32_t acc = tmem + (uint32_t)(t * fc_acc_stride(Np));
      for (int kk = 0; kk < Kp / 8; ++kk) {
        const uint32_t koff = (uint32_t)kk * 256;  // two K-adjacent core matrices
        const uint64_t ah = smem_desc(sm.sA + koff, LBO, SBO), al = smem_desc(sm.sAlo + koff, LBO, SBO);
        const uint64_t bh = smem_desc(sm.sBhi + koff, LBO, SBO), bl = smem_desc(sm.sBlo + koff, LBO, SBO);
        mma_tf32(acc, ah, bh, idesc, kk > 0 ? 1u : 0u);
        mma_tf32(acc, ah, bl, idesc, 1u);
        mma_tf32(acc, al, bh, idesc, 1u);
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
                       sm.sbar)
                   : "memory");
    }
  }
  *pending = 1;
  if (!fc_wait(sm, phase)) return false;
  *pending = 0;
  // 3. epilogue: G[P][Ia] (this column) into shared memory over the operand
  //    buffers, [npair][kFcMaxStr]; warp w reads lane quadrant w % 4 of each
  //    tile and a quarter of the 16-column groups
  float *Gs = sm.A;
  const int ng = Np / 16, gq = (ng + 3) / 4;
  const int g0 = (warp >> 2) * gq, g1 = min(ng, g0 + gq);
  const int lane_row = (warp & 3) * 32 + (tid & 31);
  for (int t = 0; t < ntile; ++t) {
    const uint32_t lane_addr = tmem + (uint32_t)(t * fc_acc_stride(Np)) + ((uint32_t)((warp & 3) * 32) << 16);
    const int row = t * kTcM + lane_row;
    for (int g = g0; g < g1; ++g) {
      uint32_t v[16];
      tmem_ld16_nowait(lane_addr + (uint32_t)(g * 16), v);
      asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
#pragma unroll
      for (int j = 0; j < 16; ++j)
        if (g * 16 + j < npair) Gs[(g * 16 + j) * kFcMaxStr + row] = __uint_as_float(v[j]);
    }
  }
  fence_before();
  __syncthreads();
  fence_after();
  // 4. alpha-only scatter of the column: A[Ia, b] -> A^T[b][Ia], one thread
  //    per string, in link order (the order of the scatter kernel's sums)
  float *At = reinterpret_cast<float *>(a.symA) + (size_t)b * nb;
  for (int ia = tid; ia < na; ia += blockDim.x) {
    const uint16_t *lr = sm.la + ia * nla;
    float acc = 0.f;
#pragma unroll 4
    for (int e = 0; e < nla; ++e) {
      const uint32_t w = lr[e];
      acc += fc_sign(Gs[((w >> 8) & 0x7Fu) * kFcMaxStr + (w & 0xFFu)], w);
    }
    At[ia] = acc;
  }
  __syncthreads();  // G readers are done before the next column's writers
  return true;
}

}  // namespace sbci
