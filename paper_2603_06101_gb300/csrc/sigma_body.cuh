// Body of the gather-form scatter of the sigma build, shared by the
// one-solve kernel and the persistent batched kernel (kernels_loop.cu, the
// only translation unit that includes this header, compiled without implicit
// multiply-add contraction, so both kernels round identically):
//   sigma[I] = sum over the links of I of sign * G[pair, J]
// with the dots of sigma against up to three vectors; in device-controlled
// mode the solve's last virtual block finishes the dots and runs the subspace
// solve (ctl.h).  Processes virtual block vb of nvb; returns true when this
// call ran the last block and the controller halted.
#pragma once

#include <cuda_runtime.h>

#include "ctl.h"
#include "devreduce.cuh"
#include "sbci_internal.h"
#include "tc_body.cuh"

namespace sbci {

constexpr int kScTile = 256;                 // threads per scatter block (and determinants per unit)
constexpr int kScStageBytes = 100 * 1024;    // shared-memory budget of the staged scatter

// Bytes of one staged segment of nf floats: the 16-byte aligned cover of the
// segment (bulk copies move 16-byte aligned blocks) plus one block of slack.
__host__ __device__ inline int sc_slot_bytes(int nf) { return ((nf * 4 + 15) / 16 + 1) * 16; }

// Shared memory of a staged unit of `rows` alpha rows: the unit's own G rows
// (all pairs, for the beta links), the G rows its alpha links point to, the
// per-segment offsets, and the mbarrier.
__host__ __device__ inline size_t scatter_stage_bytes(int npair, int nlink_a, int rows, int nb) {
  const int nd = rows * nb;
  return (size_t)npair * sc_slot_bytes(nd) + (size_t)rows * nlink_a * sc_slot_bytes(nb) +
         (size_t)(npair + rows * nlink_a) * 4 + 16;
}

__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void *src, uint32_t bytes, uint32_t bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(dst),
               "l"(src), "r"(bytes), "r"(bar)
               : "memory");
}

// Accumulates sign * G over the links of determinant I: the alpha links, then
// the beta links, in list order.  Alpha links from global memory (coalesced:
// threads of a warp hold consecutive beta strings) or, when staged, from the
// unit's shared copies of the linked G rows (slotA: per link, the float index
// of the row in shared memory, sign in bit 31); beta links from global memory
// or from the unit's own staged G rows (offB: per pair, float index).
template <typename AccT>
__device__ __forceinline__ AccT scatter_det(const SigmaArgs &a, const AccT *G, long long I, const float *sm,
                                            const int *slotA, const int *offB, int r, int nd) {
  const int ia = (int)(I / a.nb), ib = (int)(I - (long long)ia * a.nb);
  AccT acc = (AccT)0;
  if (sm) {
    const int *sa = slotA + r * a.nlink_a;
    for (int e = 0; e < a.nlink_a; ++e) {
      const int s = sa[e];
      const AccT g = (AccT)sm[(s & 0x7FFFFFFF) + ib];
      acc += (s < 0) ? -g : g;
    }
    const uint32_t *lb = a.link_bT + ib;
    const int rb = r * a.nb;
    for_links<8, AccT>(
        lb, a.nlink_b, a.nb, [&](uint32_t v) { return (AccT)sm[offB[link_pair(v)] + rb + link_J(v)]; },
        [&](uint32_t v, AccT g) { acc += link_neg(v) ? -g : g; });
    return acc;
  }
  const uint32_t *la = a.link_a + (size_t)ia * a.nlink_a;
  const AccT *gcol = G + ib;
  for_links<8, AccT>(
      la, a.nlink_a, 1,
      [&](uint32_t v) { return __ldg(gcol + (size_t)link_pair(v) * a.ndet + (size_t)link_J(v) * a.nb); },
      [&](uint32_t v, AccT g) { acc += link_neg(v) ? -g : g; });
  const uint32_t *lb = a.link_bT + ib;
  const AccT *grow = G + (size_t)ia * a.nb;
  for_links<8, AccT>(
      lb, a.nlink_b, a.nb, [&](uint32_t v) { return __ldg(grow + (size_t)link_pair(v) * a.ndet + link_J(v)); },
      [&](uint32_t v, AccT g) { acc += link_neg(v) ? -g : g; });
  return acc;
}

// Stages unit u (rows ia0 .. ia0 + nr - 1) with bulk copies issued by warp 0:
// segment c < npair is G[c][ia0*nb .. +nd) (the unit's own rows), segment
// npair + r*nlink + e is the G row of alpha link e of row ia0 + r.  Each copy
// moves the 16-byte aligned cover of its segment; the float offset of the
// segment inside its slot is recorded.  Lane 0 arms the mbarrier with the
// total byte count before any copy is issued.
__device__ __forceinline__ void scatter_stage(const SigmaArgs &a, const float *G, int ia0, int nr, float *sm,
                                              int *slotA, int *offB, uint32_t bar) {
  const int lane = threadIdx.x & 31;
  const int nd = nr * a.nb;
  const int sbf = sc_slot_bytes(nd) / 4, saf = sc_slot_bytes(a.nb) / 4;
  const int nB = a.npair, ncopy = nB + nr * a.nlink_a;
  const float *baseA = sm + (size_t)nB * sbf;
  uint32_t bytes = 0;
  for (int c = lane; c < ncopy; c += 32) {
    const float *src;
    int nf;
    if (c < nB) {
      src = G + (size_t)c * a.ndet + (size_t)ia0 * a.nb;
      nf = nd;
    } else {
      const int k = c - nB, r = k / a.nlink_a, e = k - r * a.nlink_a;
      const uint32_t v = __ldg(a.link_a + (size_t)(ia0 + r) * a.nlink_a + e);
      src = G + (size_t)link_pair(v) * a.ndet + (size_t)link_J(v) * a.nb;
      nf = a.nb;
    }
    const uintptr_t s0 = (uintptr_t)src & ~(uintptr_t)15, s1 = ((uintptr_t)(src + nf) + 15) & ~(uintptr_t)15;
    bytes += (uint32_t)(s1 - s0);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) bytes += __shfl_xor_sync(0xffffffffu, bytes, o);
  if (lane == 0)
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(bar), "r"(bytes) : "memory");
  __syncwarp();
  for (int c = lane; c < ncopy; c += 32) {
    const float *src;
    int nf;
    float *dst;
    uint32_t neg = 0;
    if (c < nB) {
      src = G + (size_t)c * a.ndet + (size_t)ia0 * a.nb;
      nf = nd;
      dst = sm + (size_t)c * sbf;
    } else {
      const int k = c - nB, r = k / a.nlink_a, e = k - r * a.nlink_a;
      const uint32_t v = __ldg(a.link_a + (size_t)(ia0 + r) * a.nlink_a + e);
      src = G + (size_t)link_pair(v) * a.ndet + (size_t)link_J(v) * a.nb;
      nf = a.nb;
      dst = const_cast<float *>(baseA) + (size_t)k * saf;
      neg = link_neg(v) ? 0x80000000u : 0u;
    }
    const uintptr_t s0 = (uintptr_t)src & ~(uintptr_t)15, s1 = ((uintptr_t)(src + nf) + 15) & ~(uintptr_t)15;
    const int off = (int)(((uintptr_t)src - s0) / 4);
    if (c < nB) offB[c] = (int)((size_t)c * sbf) + off;
    else slotA[c - nB] = (int)(((uint32_t)((size_t)(dst - sm) + off)) | neg);
    bulk_g2s(smem_u32(dst), (const void *)s0, (uint32_t)(s1 - s0), bar);
  }
}

// sigma[I] = sum over the links of I of sign * G[pair, J], with its dots.
// Work units: a.sc_rows > 0 (FP32 G only): sc_rows whole alpha rows per unit,
// staged in shared memory by bulk copies (the unit's own G rows for the beta
// links, the linked G rows for the alpha links), then summed from shared
// memory; else 256 consecutive determinants per unit, gathered from global
// memory.  Both give the same sums (same terms, same order).  A bulk-copy wait
// that runs out raises bit 1 of *a.status and ends the work of the call.
template <typename AccT>
__device__ __forceinline__ bool scatter_body(const SigmaArgs &a, int vb, int nvb) {
  double *sig = a.sigma;
  const double *du[3] = {a.dot_u[0], a.dot_u[1], a.dot_u[2]};
  if (a.ctl) {
    if (a.ctl->halt) return false;
    sig = a.ctl->Zn;
    du[2] = a.ctl->zn;
  }
  const int tid = threadIdx.x;
  const AccT *G = reinterpret_cast<const AccT *>(a.G);
  double dots[3] = {0.0, 0.0, 0.0};
  auto finish_det = [&](long long I, AccT acc) {
    const double sv = (double)acc;
    sig[I] = sv;
#pragma unroll
    for (int j = 0; j < 3; ++j)
      if (du[j]) dots[j] = fma(du[j][I], sv, dots[j]);
  };
  if (sizeof(AccT) == 4 && a.sc_rows > 0) {
    extern __shared__ __align__(16) unsigned char sc_smem[];
    const int rows = a.sc_rows;
    const int nd_full = rows * a.nb;
    float *sm = reinterpret_cast<float *>(sc_smem);
    int *offB = reinterpret_cast<int *>(sc_smem + (size_t)a.npair * sc_slot_bytes(nd_full) +
                                        (size_t)rows * a.nlink_a * sc_slot_bytes(a.nb));
    int *slotA = offB + a.npair;
    uint64_t *mb = reinterpret_cast<uint64_t *>(
        sc_smem + ((scatter_stage_bytes(a.npair, a.nlink_a, rows, a.nb) - 16 + 7) & ~(size_t)7));
    const uint32_t bar = smem_u32(mb);
    __syncthreads();  // earlier users of this shared memory are done
    if (tid == 0) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(bar) : "memory");
      asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    __syncthreads();
    uint32_t phase = 0;
    const int units = (a.na + rows - 1) / rows;
    for (int u = vb; u < units; u += nvb) {
      const int ia0 = u * rows;
      const int nr = (a.na - ia0 < rows) ? a.na - ia0 : rows;
      const int nd = nr * a.nb;
      if (tid < 32)
        scatter_stage(a, reinterpret_cast<const float *>(G), ia0, nr, sm, slotA, offB, bar);
      bool ok = mbar_wait(bar, phase, kWaitIters);
      ok = __syncthreads_and(ok) != 0;
      if (!ok) {
        if (tid == 0 && a.status) atomicOr(a.status, 2);
        mbar_wait(bar, phase, kWaitIters);  // let the copies land (bounded) before leaving
        break;
      }
      phase ^= 1u;
      if (tid < nd) {
        const long long I = (long long)ia0 * a.nb + tid;
        finish_det(I, scatter_det<AccT>(a, G, I, sm, slotA, offB, tid / a.nb, nd));
      }
      fence_async_smem();  // this thread's reads of the slots precede the next unit's copies
      __syncthreads();
    }
    __syncthreads();
    if (tid == 0) asm volatile("mbarrier.inval.shared::cta.b64 [%0];\n" ::"r"(bar) : "memory");
  } else {
    const long long ntiles = (a.ndet + kScTile - 1) / kScTile;
    for (long long tile = vb; tile < ntiles; tile += nvb) {
      const long long I = tile * kScTile + tid;
      if (I >= a.ndet) continue;
      finish_det(I, scatter_det<AccT>(a, G, I, (const float *)nullptr, nullptr, nullptr, 0, 0));
    }
  }
  if (!du[0] && !du[1] && !du[2]) return false;
  int slots[3];
#pragma unroll
  for (int j = 0; j < 3; ++j) slots[j] = du[j] ? a.dot_slot[j] : -1;
  block_partials<3, kScTile>(dots, slots, a.partials, nvb, vb);
  if (!a.ctl) return false;  // host mode: the host reduces the partials
  if (!last_block(a.counter, nvb)) return false;
  finish_slots(a.partials, nvb, a.dot_slot, 3, a.ctl->dots, a.counter);
  __shared__ int s_halt;
  if (threadIdx.x == 0) {
    ctl_solve(*a.ctl);
    s_halt = a.ctl->halt;
  }
  __syncthreads();
  return s_halt != 0;
}

}  // namespace sbci
