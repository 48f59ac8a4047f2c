// FP64 gather + contract on the tensor cores by exact integer slices (the
// error-free splitting of Ozaki, Ogita & Oishi, "Error-free transformations
// of matrix multiplication by using fast routines of matrix multiplication and
// its applications", Numer. Algorithms 59, 2012).  GB300 runs FP64 FMAs at a
// small fraction of its tensor rate; this kernel computes the same
// G[P, I] = sum_q W[P, q] D[q, I] as the FP64 SIMT kernel with the products on
// the BF16 tensor pipe and no rounding in them:
//
//  * D is gathered in FP64 (about 2 nlink additions per determinant).  Each
//    determinant row is scaled by a power of two 2^-e_I with max_q |D[I, q]|
//    < 2^e_I and rounded to a 56-bit integer (more than the 53 bits of the
//    FP64 values), F = sum_{s=1..7} m_s 2^(56-8s) with balanced base-2^8
//    digits |m_1| <= 256, |m_s| <= 128: every digit is an integer that BF16
//    holds exactly.  W is split the same way per output pair P (exponent f_P),
//    once per context.
//  * For each slice pair (s, t) the tensor cores form sum_q m_s[I, q] n_t[q, P]
//    over the npair <= 55 nonzero columns: exact integers in the FP32
//    accumulator.  Pairs with the same level L = s + t share the scale
//    2^(e_I + f_P - 8L) and one accumulator; the largest level sum (L = 8:
//    two pairs with a first digit, five without) stays below
//    55 (2 * 2^15 + 5 * 2^14) < 2^23, still exact.  Levels 2..9 are kept (34
//    of the 49 pairs); the dropped levels weigh about 2^-56 of
//    max|W| max|D|, the rounding of the inputs at most 2^-55 per term.
//  * The epilogue adds the eight levels as 64-bit integers (shifted to a
//    common scale 2^(e_I + f_P - 56)), converts once to FP64 and sets the
//    exponent: besides the 56-bit inputs, that conversion is the only
//    rounding of the whole contraction.
//
// Every step but the FP64 gather is integer or tensor-core arithmetic, so the
// kernel does not wait on the FP64 pipe.  Shared memory: D slices 7 x 128 x Kp
// BF16, W slices 7 x Np x Kp BF16, the FP64 gather rows 128 x npair: it fits
// for npair <= 55 (n <= 10 orbitals, Kp = Np = 64); the eight accumulators take
// all 512 TMEM columns (one CTA per SM).
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "sbci_internal.h"
#include "tc_body.cuh"

namespace sbci {

namespace {

constexpr int kOsSlices = 7;
constexpr int kOsBeta = 8;
constexpr int kOsLevels = 8;  // L = 2..9
constexpr int kOsKp = 64, kOsNp = 64;
constexpr int kOsMaxPair = 55;
constexpr int kOsThreads = 512;  // four per row of a 128-determinant tile

// Instruction descriptor of kind::f16 with BF16 A and B (format 1 at bits
// 7-9 and 10-12), F32 D (bits 4-5 = 1), both K-major, N >> 3 at bits 17-22,
// M >> 4 at bits 24-28.
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t tmem, uint64_t ad, uint64_t bd, uint32_t idesc,
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
__device__ __forceinline__ int opnd16(int r, int q, int Kp) {
  return (r >> 3) * (Kp * 8) + (q >> 3) * 64 + (r & 7) * 8 + (q & 7);
}

// Biased exponent of |x| (0 for zeros and subnormals, which are dropped).
__device__ __forceinline__ int bexp(double x) {
  return (int)((__double_as_longlong(x) >> 52) & 0x7FF);
}

// The 56-bit integer of x scaled by 2^(56 - e), e = emax_biased - 1022
// (so that every |x| of the row or column is below 2^e): the 53-bit
// significand M times 2^(E - emax + 3), exact for the three largest binades
// and rounded to nearest below them.
__device__ __forceinline__ long long fixed56(double x, int emax) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const int E = (int)((b >> 52) & 0x7FF);
  if (E == 0) return 0;
  const long long M = (long long)((b & 0xFFFFFFFFFFFFFull) | 0x10000000000000ull);
  const int sh = emax - E - 3;  // >= -3
  long long F;
  if (sh <= 0) F = M * (1LL << (-sh));
  else if (sh >= 60) F = 0;
  else F = (M + (1LL << (sh - 1))) >> sh;
  return (b >> 63) ? -F : F;
}

// Digits of F (|F| < 2^56) in base 2^8, most significant first: m_2..m_7 in
// [-128, 127] are the six low bytes of F + 0x808080808080 less 128 each, m_1
// (|m_1| <= 256) the rest, so that F = sum_s m_s 2^(56 - 8s).
__device__ __forceinline__ void digits(long long F, int (&m)[kOsSlices]) {
  const long long G = F + 0x808080808080LL;
  m[0] = (int)(G >> 48);
  const uint32_t lo = (uint32_t)G, hi = (uint32_t)(G >> 32);
  m[1] = (int)((hi >> 8) & 0xFF) - 128;
  m[2] = (int)(hi & 0xFF) - 128;
  m[3] = (int)(lo >> 24) - 128;
  m[4] = (int)((lo >> 16) & 0xFF) - 128;
  m[5] = (int)((lo >> 8) & 0xFF) - 128;
  m[6] = (int)(lo & 0xFF) - 128;
}

// BF16 bits of a small integer (|d| <= 256, exact in FP32 and in BF16): the
// FP32 value through the 1.5 * 2^23 bias, then its upper half.
__device__ __forceinline__ uint32_t bf16_of_int(int d) {
  const float f = __int_as_float(0x4B400000 + d) - 12582912.0f;
  return __float_as_uint(f) >> 16;
}

// v * 2^k as FP64, rounded to nearest even, by integer operations (v != 0,
// |v| < 2^63; the result in the normal range, else through ldexp).
__device__ __forceinline__ double scaled_ll_to_double(long long v, int k) {
  const unsigned long long sign = v < 0 ? (1ull << 63) : 0ull;
  unsigned long long a = v < 0 ? (unsigned long long)(-v) : (unsigned long long)v;
  const int lz = __clzll((long long)a);
  a <<= lz;  // leading bit at 63
  unsigned long long m = a >> 11;
  const unsigned long long rem = a & 0x7FFull;
  if (rem > 0x400ull || (rem == 0x400ull && (m & 1ull))) ++m;
  int E = 1023 + (63 - lz) + k;
  if (m == (1ull << 53)) {
    m >>= 1;
    ++E;
  }
  if (E <= 0 || E >= 2047) return ldexp((double)v, k);
  return __longlong_as_double((long long)(sign | ((unsigned long long)E << 52) | (m & 0xFFFFFFFFFFFFFull)));
}

// Operand B: the slices of W (K-major, output pair P = row n, input pair q = k)
// and the exponent f_P of each output pair (biased, 0 for an all-zero row).
__global__ void k_split_W_os(const double *W, int npair, __nv_bfloat16 *out, int *fexp) {
  const int P = blockIdx.x * blockDim.x + threadIdx.x;
  if (P >= kOsNp) return;
  int emax = 0;
  if (P < npair)
    for (int q = 0; q < npair; ++q) emax = max(emax, bexp(W[(size_t)P * npair + q]));
  fexp[P] = emax;
  const int nb = kOsNp * kOsKp;
  for (int q = 0; q < kOsKp; ++q) {
    int m[kOsSlices] = {0, 0, 0, 0, 0, 0, 0};
    if (P < npair && q < npair && emax > 0) digits(fixed56(W[(size_t)P * npair + q], emax), m);
    for (int s = 0; s < kOsSlices; ++s) out[(size_t)s * nb + opnd16(P, q, kOsKp)] = __float2bfloat16_rn((float)m[s]);
  }
}

struct OsSmem {
  __nv_bfloat16 *A;  // [7][128 x Kp]
  __nv_bfloat16 *B;  // [7][Np x Kp]
  double *D;         // [128][npair]
  int *eI;           // [128] biased row exponents
  int *eQ;           // [4][128] exponents of the row quarters
  int *fP;           // [Np]
  uint64_t *bar;
  uint32_t *tmem_slot;
};

__global__ void __launch_bounds__(kOsThreads, 1)
    k_gather_contract_os(SigmaArgs a, const __nv_bfloat16 *Wos, const int *fexp, int *status) {
  extern __shared__ __align__(128) unsigned char smem[];
  OsSmem sm;
  const int npair = a.npair;
  sm.A = reinterpret_cast<__nv_bfloat16 *>(smem);
  sm.B = sm.A + kOsSlices * kTcM * kOsKp;
  sm.D = reinterpret_cast<double *>(sm.B + kOsSlices * kOsNp * kOsKp);
  sm.eI = reinterpret_cast<int *>(sm.D + kTcM * npair);
  sm.eQ = sm.eI + kTcM;
  sm.fP = sm.eQ + 4 * kTcM;
  sm.bar = reinterpret_cast<uint64_t *>(sm.fP + kOsNp);
  sm.tmem_slot = reinterpret_cast<uint32_t *>(sm.bar + 1);
  const int tid = threadIdx.x, warp = tid >> 5;
  const uint32_t sA = smem_u32(sm.A), sB = smem_u32(sm.B), sbar = smem_u32(sm.bar);
  const uint32_t kCols = 512;
  const double *cin = a.c;
  if (a.ctl) {  // inside the SB step loop: the controller's next z
    if (a.ctl->halt) return;  // uniform: before any TMEM allocation or barrier
    cin = a.ctl->zn;
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(
                     smem_u32(sm.tmem_slot)),
                 "r"(kCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(sbar) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  // operand B and the column exponents; the padding columns of A stay zero
  {
    const uint4 *src = reinterpret_cast<const uint4 *>(Wos);
    uint4 *dst = reinterpret_cast<uint4 *>(sm.B);
    for (int i = tid; i < kOsSlices * kOsNp * kOsKp / 8; i += kOsThreads) dst[i] = __ldg(src + i);
    uint4 *az = reinterpret_cast<uint4 *>(sm.A);
    for (int i = tid; i < kOsSlices * kTcM * kOsKp / 8; i += kOsThreads) az[i] = make_uint4(0, 0, 0, 0);
    for (int i = tid; i < kOsNp; i += kOsThreads) sm.fP[i] = fexp[i];
  }
  fence_async_smem();
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = *sm.tmem_slot;
  const uint32_t idesc = idesc_bf16(kTcM, kOsNp);
  const uint32_t LBO = 128, SBO = (uint32_t)kOsKp * 16;
  const uint32_t sliceA = (uint32_t)(kTcM * kOsKp * 2), sliceB = (uint32_t)(kOsNp * kOsKp * 2);
  double *G = reinterpret_cast<double *>(a.G);
  const long long ntiles = (a.ndet + kTcM - 1) / kTcM;
  uint32_t phase = 0;
  bool ok = true;
  for (long long tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x) {
    // 1. gather: threads r and 128 + r build the alpha part of row r of D in
    //    FP64 (halves of its alpha links), threads 256 + r and 384 + r the
    //    beta part in the A-slice area (free until the slices are written; the
    //    previous tile's MMAs have completed); a string's links have distinct
    //    pairs, so the two halves write disjoint entries of the zeroed row
    const int r = tid & (kTcM - 1), part = tid >> 7, sub = part & 1;
    {
      const bool beta = part >= 2;
      double *row = beta ? reinterpret_cast<double *>(sm.A) + (size_t)r * npair : sm.D + (size_t)r * npair;
      const int hz = npair / 2;
      for (int q = sub ? hz : 0; q < (sub ? npair : hz); ++q) row[q] = 0.0;
      __syncthreads();
      const long long I = tile * kTcM + r;
      if (I < a.ndet) {
        int ia, ib;
        split_det(I, a.nb, ia, ib);
        const int nl = beta ? a.nlink_b : a.nlink_a, hl = (nl + 1) / 2;
        const int e0 = sub ? hl : 0, ne = sub ? nl - hl : hl;
        if (!beta) {
          const uint32_t *la = a.link_a + (size_t)ia * a.nlink_a + e0;
          const double *ccol = cin + ib;
          for_links<8, double>(
              la, ne, 1, [&](uint32_t v) { return __ldg(ccol + (size_t)link_J(v) * a.nb); },
              [&](uint32_t v, double cv) { row[link_pair(v)] += link_neg(v) ? -cv : cv; });
        } else {
          const uint32_t *lb = a.link_bT + (size_t)e0 * a.nb + ib;
          const double *crow = cin + (size_t)ia * a.nb;
          for_links<8, double>(
              lb, ne, a.nb, [&](uint32_t v) { return __ldg(crow + link_J(v)); },
              [&](uint32_t v, double cv) { row[link_pair(v)] += link_neg(v) ? -cv : cv; });
        }
      }
    }
    __syncthreads();
    // D = alpha part + beta part (alpha first, as the FP64 SIMT kernel adds
    // them); four threads per row, each a quarter of the columns
    const int quarter = ((npair + 31) / 32) * 8;  // quarters at multiples of 8 columns
    {
      const int q0 = min(part * quarter, npair), q1 = min(q0 + quarter, npair);
      double *row = sm.D + (size_t)r * npair;
      const double *rb = reinterpret_cast<const double *>(sm.A) + (size_t)r * npair;
      int emax = 0;
      for (int q = q0; q < q1; ++q) {
        const double d = row[q] + rb[q];
        row[q] = d;
        emax = max(emax, bexp(d));
      }
      sm.eQ[part * kTcM + r] = emax;
    }
    __syncthreads();
    // 2. the seven digit slices: each thread 8 consecutive columns of a row at
    //    a time (one core-matrix row: a 16-byte store per slice), its quarter
    //    of the padded width (the beta staging overwrote the padding columns)
    {
      const int q0 = part * quarter, q_end = (part == 3) ? kOsKp : min((part + 1) * quarter, kOsKp);
      const int q1 = npair;
      const int emax = max(max(sm.eQ[r], sm.eQ[kTcM + r]), max(sm.eQ[2 * kTcM + r], sm.eQ[3 * kTcM + r]));
      if (part == 0) sm.eI[r] = emax;
      const double *row = sm.D + (size_t)r * npair;
      for (int qc = q0; qc < q_end; qc += 8) {
        uint32_t w[kOsSlices][4];
#pragma unroll
        for (int sl = 0; sl < kOsSlices; ++sl) w[sl][0] = w[sl][1] = w[sl][2] = w[sl][3] = 0u;
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          int m[kOsSlices] = {0, 0, 0, 0, 0, 0, 0};
          if (qc + j < q1 && emax > 0) digits(fixed56(row[qc + j], emax), m);
#pragma unroll
          for (int sl = 0; sl < kOsSlices; ++sl) w[sl][j >> 1] |= bf16_of_int(m[sl]) << ((j & 1) * 16);
        }
        const int off = opnd16(r, qc, kOsKp);  // 8-element aligned: a 16-byte core-matrix row
#pragma unroll
        for (int sl = 0; sl < kOsSlices; ++sl)
          *reinterpret_cast<uint4 *>(sm.A + (size_t)sl * kTcM * kOsKp + off) =
              make_uint4(w[sl][0], w[sl][1], w[sl][2], w[sl][3]);
      }
    }
    fence_async_smem();
    fence_before();
    __syncthreads();
    fence_after();
    // 3. levels L = 2..9: accumulator L-2 gets every (s, t) with s + t = L
    if (tid == 0) {
      for (int L = 2; L <= kOsLevels + 1; ++L) {
        const uint32_t acc = tmem + (uint32_t)((L - 2) * kOsNp);
        bool first = true;
        for (int s = 1; s <= kOsSlices; ++s) {
          const int t = L - s;
          if (t < 1 || t > kOsSlices) continue;
          for (int kk = 0; kk < kOsKp / 16; ++kk) {
            const uint32_t koff = (uint32_t)kk * 256;  // two K-adjacent core matrices
            const uint64_t ad = smem_desc(sA + (uint32_t)(s - 1) * sliceA + koff, LBO, SBO);
            const uint64_t bd = smem_desc(sB + (uint32_t)(t - 1) * sliceB + koff, LBO, SBO);
            mma_bf16(acc, ad, bd, idesc, first ? 0u : 1u);
            first = false;
          }
        }
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(sbar)
                   : "memory");
    }
    ok = mbar_wait(sbar, phase, kWaitIters);
    ok = __syncthreads_and(ok) != 0;
    if (!ok) break;
    phase ^= 1u;
    fence_after();
    // 4. epilogue: warp w reads lane quadrant (w % 4) and column quarter
    //    (w / 4); the eight levels of 4 columns at a time, added as integers
    {
      const int rr = (warp & 3) * 32 + (tid & 31);
      const long long I = tile * kTcM + rr;
      const int eI = sm.eI[rr];
      const uint32_t lane_addr = tmem + ((uint32_t)((warp & 3) * 32) << 16);
      const int c_begin = (warp >> 2) * (kOsNp / 4);
      for (int c0 = c_begin; c0 < c_begin + kOsNp / 4; c0 += 4) {
        uint32_t v[kOsLevels][4];
#pragma unroll
        for (int g = 0; g < kOsLevels; ++g)
          asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0,%1,%2,%3}, [%4];\n"
                       : "=r"(v[g][0]), "=r"(v[g][1]), "=r"(v[g][2]), "=r"(v[g][3])
                       : "r"(lane_addr + (uint32_t)(g * kOsNp + c0)));
        asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
        if (I < a.ndet) {
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            const int P = c0 + j;
            if (P >= npair) continue;
            // sum_L v_L 2^(56 - 8L) as a 64-bit integer (L = 2..9: shifts 40 .. -16;
            // |v_2| <= 55 * 2^16 < 2^22, so every term stays below 2^62)
            long long acc = 0;
#pragma unroll
            for (int g = 0; g < kOsLevels; ++g) {
              const long long vi = (long long)__float2int_rn(__uint_as_float(v[g][j]));
              const int sh = 56 - kOsBeta * (g + 2);
              acc += sh >= 0 ? vi * (1LL << sh) : (vi >> (-sh));
            }
            double out = 0.0;
            const int fP = sm.fP[P];
            if (eI == 2047)  // a NaN or infinity in the row: propagate it as the FMA kernel would
              out = __longlong_as_double(0x7FF8000000000000LL);
            else if (acc != 0 && eI > 0 && fP > 0)  // acc 2^(e_I + f_P - 56), e = biased - 1022
              out = scaled_ll_to_double(acc, (eI - 1022) + (fP - 1022) - 56);
            G[(size_t)P * a.ndet + I] = out;
          }
        }
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
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(kCols) : "memory");
}

size_t os_smem_bytes(int npair) {
  return (size_t)kOsSlices * kTcM * kOsKp * 2 + (size_t)kOsSlices * kOsNp * kOsKp * 2 +
         (size_t)kTcM * npair * 8 + (size_t)(5 * kTcM + kOsNp) * 4 + 16;
}

}  // namespace

size_t os_W_bytes() { return (size_t)kOsSlices * kOsNp * kOsKp * 2; }

bool os_supported(int npair) { return npair >= 1 && npair <= kOsMaxPair; }

cudaError_t launch_split_W_os(const double *W, int npair, void *out, int *fexp, cudaStream_t s) {
  if (!os_supported(npair)) return cudaErrorInvalidValue;
  k_split_W_os<<<1, kOsNp, 0, s>>>(W, npair, reinterpret_cast<__nv_bfloat16 *>(out), fexp);
  return cudaGetLastError();
}

// Resident CTAs: one per SM (all of TMEM, nearly all of shared memory).
int os_grid(long long ndet, int nsm) {
  const long long ntiles = (ndet + kTcM - 1) / kTcM;
  long long g = nsm;
  if (g > ntiles) g = ntiles;
  return (int)(g < 1 ? 1 : g);
}

cudaError_t prepare_os_kernel(int npair) {
  if (!os_supported(npair)) return cudaErrorInvalidValue;
  int optin = 0;
  cudaError_t e = max_dynamic_smem((const void *)k_gather_contract_os, &optin);
  if (e != cudaSuccess) return e;
  if ((int)os_smem_bytes(npair) > optin) return cudaErrorInvalidValue;
  return cudaFuncSetAttribute(k_gather_contract_os, cudaFuncAttributeMaxDynamicSharedMemorySize, optin);
}

cudaError_t launch_gather_contract_os(const SigmaArgs &a, const void *Wos, const int *fexp, int *status, int grid,
                                      cudaStream_t s) {
  if (!os_supported(a.npair)) return cudaErrorInvalidValue;
  k_gather_contract_os<<<grid, kOsThreads, os_smem_bytes(a.npair), s>>>(
      a, reinterpret_cast<const __nv_bfloat16 *>(Wos), fexp, status);
  return cudaGetLastError();
}

}  // namespace sbci
