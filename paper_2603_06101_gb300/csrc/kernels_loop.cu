// The kernels of the SB step loop, in one translation unit: the one-solve
// kernels (update, projection, tensor-core gather + contract, scatter) and the
// batched persistent kernels that serve many solves per launch.  Both run the
// same bodies (step_body.cuh, sigma_body.cuh, tc_body.cuh, ctl.h), and this
// file is compiled without implicit multiply-add contraction (every fused
// operation is an explicit fma()), so a solve run alone and the same solve run
// in a batch round identically and give bitwise the same results.
//
// One-solve kernels: scalars come from the device controller state (ctl.h);
// the last block of the update sweep finishes its dot products and runs the
// convergence / restart test, the last block of the scatter solves the
// subspace problem, so consecutive steps need no host round trip.  Every
// kernel returns at once when the controller has halted, and then clears the
// loop condition of the enclosing graph (if any), so a graph while-loop over
// these kernels always ends.
//
// Tensor-core (tcgen05) gather + contract in 3-term TF32 split precision, per
// tile of 128 determinants (one per TMEM lane, two threads each):
//   1. gather   D[I, Q] = sum_{links of I} sign * c[J]   into shared memory,
//               FP32, laid out as the K-major no-swizzle canonical operand A
//               (8-row x 16-byte core matrices); thread r gathers the alpha
//               links of row r into A, thread r + 128 the beta links into the
//               A_lo buffer, so every element has one writer;
//   2. split    D = alpha + beta part = D_hi + D_lo, both TF32, in place;
//   3. MMA      G^T = D_hi W_hi + D_hi W_lo + D_lo W_hi  (M=128, N=Np, K=8 per
//               instruction), issued by one thread, accumulated in TMEM (FP32);
//   4. epilogue tcgen05.ld: warps w and w + 4 read the lanes of quadrant w,
//               half of the columns each -> G[P][I] (FP32) in global.
// W (symmetric, packed pairs) is split once per CTA into TF32 hi/lo operand B
// that stays in shared memory.  The dropped D_lo W_lo term and the TF32
// rounding of the lo parts leave a relative error of about 2^-21 per product.
// Every wait on the MMA-completion mbarrier is bounded; on timeout the kernel
// raises bit 0 of *status, waits once more (bounded) for its MMAs, frees its
// TMEM and returns.
//
// Batched kernels: one launch of each serves every solve of a batch through
// the device job table (batch.h), a work queue of (solve, virtual block)
// items; the tensor-core kernel takes (solve, tile) items from an atomic
// queue and reloads a solve's W operand when the solve changes.  A final
// one-thread kernel ends the graph while-loop when any solve's controller has
// halted, so the host can act on it.
#include <cuda_runtime.h>
#include <stdint.h>

#include "batch.h"
#include "ctl.h"
#include "fused_body.cuh"
#include "sbci_internal.h"
#include "sigma_body.cuh"
#include "step_body.cuh"
#include "tc_body.cuh"

namespace sbci {

// Largest dynamic shared memory a launch of kernel f may opt into on the
// current device: the per-block opt-in limit minus f's static shared memory.
cudaError_t max_dynamic_smem(const void *f, int *bytes) {
  int dev = 0, optin = 0;
  cudaFuncAttributes fa{};
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, f);
  if (e != cudaSuccess) return e;
  *bytes = optin - (int)fa.sharedSizeBytes;
  return cudaSuccess;
}

// CTAs of kernel f (threads per CTA, dynamic shared memory dyn) that fit one
// SM, from the device's shared-memory and register budgets and the kernel's
// register count and static shared memory (the larger of this and the
// runtime's occupancy answer is used: launching more CTAs than fit is legal,
// they wait for a slot).
static int resident_ctas(const void *f, int threads, size_t dyn) {
  int dev = 0, smem_sm = 0, reserved = 0, regs_sm = 0, api = 0;
  cudaFuncAttributes fa{};
  if (cudaGetDevice(&dev) != cudaSuccess || cudaFuncGetAttributes(&fa, f) != cudaSuccess ||
      cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&regs_sm, cudaDevAttrMaxRegistersPerMultiprocessor, dev) != cudaSuccess)
    return 1;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&api, f, threads, dyn) != cudaSuccess) api = 0;
  const size_t per_cta_smem = dyn + fa.sharedSizeBytes + (size_t)reserved;
  const int by_smem = (int)((size_t)smem_sm / per_cta_smem);
  const int warp_regs = (fa.numRegs * 32 + 255) / 256 * 256;  // allocation unit: 256 registers per warp
  const int by_regs = regs_sm / (warp_regs * ((threads + 31) / 32));
  int n = by_smem < by_regs ? by_smem : by_regs;
  if (api > n) n = api;
  return n < 1 ? 1 : n;
}

// ---------------------------------------------------------------- one solve

__device__ __forceinline__ void halt_loop(unsigned long long cond) {
  if (cond && blockIdx.x == 0 && threadIdx.x == 0)
    cudaGraphSetConditional((cudaGraphConditionalHandle)cond, 0u);
}

__global__ void __launch_bounds__(kStepThreads) k_update_ctl(StepArgs a) {
  if (a.ctl->halt) {
    halt_loop(a.cond);
    return;
  }
  __shared__ __align__(16) unsigned char s_upd[kUpdSmemBytes];
  const bool halted = a.sector ? update_body_sym(a, blockIdx.x, gridDim.x, s_upd)
                               : update_body(a, blockIdx.x, gridDim.x, s_upd);
  if (halted && a.cond && threadIdx.x == 0)
    cudaGraphSetConditional((cudaGraphConditionalHandle)a.cond, 0u);
}

__global__ void __launch_bounds__(kStepThreads) k_project_ctl(StepArgs a) {
  if (a.ctl->halt) {
    halt_loop(a.cond);
    return;
  }
  project_body(a, blockIdx.x, gridDim.x);
}

int step_grid(long long n, int nsm) {
  long long g = (n + 4 * kStepThreads - 1) / (4 * kStepThreads);  // ~4 elements per thread
  if (g > 2LL * nsm) g = 2LL * nsm;
  if (g < 1) g = 1;
  return (int)g;
}

cudaError_t launch_update_ctl(const StepArgs &a, int grid, cudaStream_t s) {
  k_update_ctl<<<grid, kStepThreads, 0, s>>>(a);
  return cudaGetLastError();
}

__global__ void k_pinv(const double *diag, double E, double guard, long long n, double *out) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    out[i] = recip(guarded(diag[i] - E, guard));
}

cudaError_t launch_pinv(const double *diag, double E, double guard, long long n, double *out, cudaStream_t s) {
  long long g = (n + 255) / 256;
  if (g > 4096) g = 4096;
  k_pinv<<<(int)(g < 1 ? 1 : g), 256, 0, s>>>(diag, E, guard, n, out);
  return cudaGetLastError();
}

__global__ void k_restart_resync(CtlState *ctl, const double *dots, RestartArgs r) {
  CtlHead &h = *ctl;
  const double xx = dots[0], xX = dots[1];
  if (!(xx > 0.0) || !isfinite(xx) || !isfinite(xX)) {  // the host finds the failure at its next read
    h.halt = H_NUMERIC;
    return;
  }
  const double sx = 1.0 / sqrt(xx), E = xX / xx;
  h.halt = H_RUN;
  h.pending_check = 0;
  h.first = 1;
  h.sx_pending = 1.0;
  h.t = 0;
  h.E = E;
  h.stage = 1;
  h.n_sync = 0;
  h.prec = r.prec;
  h.zf = r.zf;
  h.up.sx = sx;
  h.up.sy = 0.0;
  h.up.b = 0.0;
  h.up.c = 0.0;
  h.up.E = E;
  h.up.kinv = 1.0;
  h.up.Epre = r.ground ? E : r.Epre_fixed;
  h.iters = 0;
  h.iter_cap = r.iter_cap;
  h.zc = r.z0;
  h.Zc = r.Z0;
  h.zn = r.z1;
  h.Zn = r.Z1;
  h.n_sigma += 1;  // the FP64 re-sync
  h.n_sigma_fp64 += 1;
  h.ntrace = 0;
}

cudaError_t launch_restart_resync(CtlState *ctl, const double *dots, const RestartArgs &r, cudaStream_t s) {
  k_restart_resync<<<1, 1, 0, s>>>(ctl, dots, r);
  return cudaGetLastError();
}

cudaError_t launch_project_ctl(const StepArgs &a, int grid, cudaStream_t s) {
  k_project_ctl<<<grid, kStepThreads, 0, s>>>(a);
  return cudaGetLastError();
}

template <typename AccT>
__global__ void __launch_bounds__(kScTile, 3) k_scatter(SigmaArgs a) {
  if (a.ctl && a.ctl->halt) {
    if (a.cond && blockIdx.x == 0 && threadIdx.x == 0)
      cudaGraphSetConditional((cudaGraphConditionalHandle)a.cond, 0u);
    return;
  }
  const bool halted = scatter_body<AccT>(a, blockIdx.x, gridDim.x);
  if (halted && a.cond && threadIdx.x == 0)
    cudaGraphSetConditional((cudaGraphConditionalHandle)a.cond, 0u);
}

int scatter_grid(long long ndet, int nsm) {
  long long g = (ndet + kScTile - 1) / kScTile;
  if (g > 8LL * nsm) g = 8LL * nsm;
  if (g < 1) g = 1;
  return (int)g;
}

template <typename AccT>
static cudaError_t launch_sc_t(const SigmaArgs &a, cudaStream_t s) {
  k_scatter<AccT><<<a.grid, kScTile, 0, s>>>(a);
  return cudaGetLastError();
}

template <typename AccT>
__global__ void __launch_bounds__(kScTile) k_symfin(SigmaArgs a) {
  if (a.ctl->halt) {
    if (a.cond && blockIdx.x == 0 && threadIdx.x == 0)
      cudaGraphSetConditional((cudaGraphConditionalHandle)a.cond, 0u);
    return;
  }
  const bool halted = symfin_body<AccT>(a, blockIdx.x, gridDim.x);
  if (halted && a.cond && threadIdx.x == 0)
    cudaGraphSetConditional((cudaGraphConditionalHandle)a.cond, 0u);
}

int symfin_grid(int na, int nsm) {
  const long long T = (na + kSfT - 1) / kSfT;
  long long g = T * (T + 1) / 2;
  if (g > 8LL * nsm) g = 8LL * nsm;
  if (g < 1) g = 1;
  return (int)g;
}

cudaError_t launch_symfin(const SigmaArgs &a, int prec, cudaStream_t s) {
  if (prec == 0) k_symfin<double><<<a.sf_grid, kScTile, 0, s>>>(a);
  else k_symfin<float><<<a.sf_grid, kScTile, 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_scatter(const SigmaArgs &a, int prec, cudaStream_t s) {
  return prec == 0 ? launch_sc_t<double>(a, s) : launch_sc_t<float>(a, s);
}


__global__ void __launch_bounds__(kTcThreads, 2)
    k_gather_contract_tc(SigmaArgs a, int Kp, int Np, uint32_t tmem_cols, int *status) {
  extern __shared__ __align__(128) unsigned char smem[];
  TcSmem sm;
  sm.A = reinterpret_cast<float *>(smem);
  sm.Alo = sm.A + kTcM * Kp;
  sm.Bhi = reinterpret_cast<uint32_t *>(sm.Alo + kTcM * Kp);
  sm.Blo = sm.Bhi + Np * Kp;
  uint64_t *mbar = reinterpret_cast<uint64_t *>(sm.Blo + Np * Kp);
  uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(mbar + 1);
  sm.sA = smem_u32(sm.A);
  sm.sAlo = smem_u32(sm.Alo);
  sm.sBhi = smem_u32(sm.Bhi);
  sm.sBlo = smem_u32(sm.Blo);
  sm.sbar = smem_u32(mbar);
  const int tid = threadIdx.x, warp = tid >> 5;
  const float *cin = a.cf;
  if (a.ctl) {
    if (a.ctl->halt) return;  // uniform: before any TMEM allocation or barrier
    cin = a.ctl->zf;
  }
  if (!cin) {  // no FP32 input: refuse (uniform, before any allocation)
    if (threadIdx.x == 0) atomicOr(status, 4);
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
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(sm.sbar) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  tc_load_B(a, Kp, Np, sm);
  const uint32_t tmem = *tmem_slot;
  const long long ntiles = (a.ndet + kTcM - 1) / kTcM;
  uint32_t phase = 0;
  bool ok = true;
  for (long long tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x)
    ok = tc_tile(a, cin, tile, Kp, Np, sm, tmem, phase);
  if (!ok) {
    if (tid == 0) atomicOr(status, 1);
    mbar_wait(sm.sbar, phase, kWaitIters);  // let the outstanding MMAs drain (bounded)
  }
  fence_before();
  __syncthreads();
  fence_after();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(tmem_cols)
                 : "memory");
}

// Operand sizes of the TF32 split kernel for npair packed pairs.
bool tc_dims(int npair, int *Kp, int *Np, uint32_t *cols, size_t *smem) {
  const int kp = (npair + 7) / 8 * 8;
  const int np = (npair + 15) / 16 * 16;
  uint32_t c = 32;
  while (c < (uint32_t)np) c <<= 1;
  const size_t bytes = (size_t)(2 * kTcM * kp + 2 * np * kp) * 4 + 16;
  *Kp = kp;
  *Np = np;
  *cols = c;
  *smem = bytes;
  return np <= 256 && bytes <= 227 * 1024;
}

// Grid of the persistent tensor-core kernel (resident CTAs, capped by TMEM
// columns), computed outside any stream capture.  0 if the shape is unsupported.
int tc_grid(int npair, long long ndet, int num_sms) {
  int Kp, Np;
  uint32_t cols;
  size_t smem;
  if (!tc_dims(npair, &Kp, &Np, &cols, &smem)) return 0;
  // the opt-in limit is a property of the function shared by all contexts:
  // always the largest, so that a context of another shape cannot lower it
  int optin = 0;
  if (max_dynamic_smem((const void *)k_gather_contract_tc, &optin) != cudaSuccess || (int)smem > optin ||
      cudaFuncSetAttribute(k_gather_contract_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, optin) !=
          cudaSuccess)
    return 0;
  // all of the unified L1/shared storage as shared memory: two CTAs per SM
  // whenever the operands fit twice
  if (cudaFuncSetAttribute(k_gather_contract_tc, cudaFuncAttributePreferredSharedMemoryCarveout,
                           cudaSharedmemCarveoutMaxShared) != cudaSuccess)
    return 0;
  int per_sm = resident_ctas((const void *)k_gather_contract_tc, kTcThreads, smem);
  if ((uint32_t)per_sm * cols > 512) per_sm = (int)(512 / cols);
  const long long ntiles = (ndet + kTcM - 1) / kTcM;
  long long grid = (long long)num_sms * per_sm;
  if (grid > ntiles) grid = ntiles;
  if (grid < 1) grid = 1;
  return (int)grid;
}

__global__ void k_split_W(const double *W, int npair, int Kp, int Np, uint32_t *out) {
  const int nb = Np * Kp;
  for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < nb; idx += gridDim.x * blockDim.x) {
    const int n = idx / Kp, k = idx - n * Kp;
    split_W_elem(W, npair, n, k, &out[opnd_off(n, k, Kp)], &out[nb + opnd_off(n, k, Kp)]);
  }
}

cudaError_t launch_split_W(const double *W, int npair, int Kp, int Np, uint32_t *out, cudaStream_t s) {
  const int nb = Np * Kp;
  k_split_W<<<(nb + 255) / 256, 256, 0, s>>>(W, npair, Kp, Np, out);
  return cudaGetLastError();
}

cudaError_t launch_gather_contract_tc(const SigmaArgs &a, int *status, int grid, cudaStream_t s) {
  int Kp, Np;
  uint32_t cols;
  size_t smem;
  if (!tc_dims(a.npair, &Kp, &Np, &cols, &smem) || grid < 1) return cudaErrorInvalidValue;
  k_gather_contract_tc<<<grid, kTcThreads, smem, s>>>(a, Kp, Np, cols, status);
  return cudaGetLastError();
}

// ------------------------------------------------- column-fused sector sigma

// TMEM allocation, mbarrier set-up and operand B of a column CTA (uniform:
// every thread calls it).
__device__ __forceinline__ void fc_begin(const FcSmem &sm, uint32_t tmem_cols) {
  if ((threadIdx.x >> 5) == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(
                     smem_u32(fc_tmem_slot(sm))),
                 "r"(tmem_cols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
  }
  if (threadIdx.x == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(sm.sbar) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
}

// Error path and TMEM release at the end of a column CTA.
__device__ __forceinline__ void fc_end(const FcSmem &sm, bool ok, int pending, uint32_t phase, uint32_t tmem,
                                       uint32_t tmem_cols, int *status) {
  if (!ok) {
    if (threadIdx.x == 0) atomicOr(status, 1);
    if (pending) mbar_wait(sm.sbar, phase, kWaitIters);  // let the outstanding MMAs drain (bounded)
  }
  fence_before();
  __syncthreads();
  fence_after();
  if ((threadIdx.x >> 5) == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(tmem_cols)
                 : "memory");
}

__global__ void __launch_bounds__(kFcThreads, 2)
    k_fused_column(SigmaArgs a, int Kp, int Np, uint32_t tmem_cols, int *status) {
  extern __shared__ __align__(128) unsigned char smem[];
  const FcSmem sm = fc_carve(smem, Kp, Np);
  if (!a.ctl || a.ctl->halt) return;  // uniform: before any TMEM allocation or barrier
  const float *zf = a.ctl->zf;
  if (!zf || !a.symA || !a.fc_link_a) {  // the column kernel needs these: refuse
    if (threadIdx.x == 0) atomicOr(status, 4);
    return;
  }
  if ((int)blockIdx.x >= a.nb) return;
  fc_begin(sm, tmem_cols);
  fc_load_links(a, sm);
  fc_load_B(a, Kp, Np, sm);  // (ends with a barrier)
  const uint32_t tmem = *fc_tmem_slot(sm);
  uint32_t phase = 0;
  int pending = 0;
  bool ok = true;
  for (int b = blockIdx.x; b < a.nb && ok; b += gridDim.x) ok = fc_column(a, zf, b, Kp, Np, sm, tmem, phase, &pending);
  fc_end(sm, ok, pending, phase, tmem, tmem_cols, status);
}

bool fc_dims(int npair, int na, int nb, int nlink_b, int *Kp, int *Np, uint32_t *cols, size_t *smem) {
  uint32_t tc_cols;
  size_t tc_smem;
  if (na != nb || na < 1 || na > kFcMaxStr || nlink_b > kFcMaxLink || npair > 128 ||
      (long long)na * nlink_b > kFcLinkMax || !tc_dims(npair, Kp, Np, &tc_cols, &tc_smem))
    return false;
  const uint32_t c = 2u * (uint32_t)fc_acc_stride(*Np);
  *cols = c;
  *smem = fc_smem_bytes(*Kp, *Np);
  return c <= 512 && *smem <= 227 * 1024;
}

// Sets the opt-in shared-memory limit of a column kernel and returns its
// resident CTAs per SM for a launch with smem bytes and cols TMEM columns.
static int fc_prepare(const void *f, size_t smem, uint32_t cols) {
  int optin = 0;
  if (max_dynamic_smem(f, &optin) != cudaSuccess || (int)smem > optin ||
      cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, optin) != cudaSuccess ||
      cudaFuncSetAttribute(f, cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared) !=
          cudaSuccess)
    return 0;
  int per_sm = resident_ctas(f, kFcThreads, smem);
  if ((uint32_t)per_sm * cols > 512) per_sm = (int)(512 / cols);
  return per_sm;
}

int fc_grid(int npair, int na, int nb, int nlink_b, int num_sms) {
  int Kp, Np;
  uint32_t cols;
  size_t smem;
  if (!fc_dims(npair, na, nb, nlink_b, &Kp, &Np, &cols, &smem)) return 0;
  const int per_sm = fc_prepare((const void *)k_fused_column, smem, cols);
  if (per_sm < 1) return 0;
  long long grid = (long long)num_sms * per_sm;
  if (grid > nb) grid = nb;
  return (int)grid;
}

cudaError_t launch_fused_column(const SigmaArgs &a, int *status, int grid, cudaStream_t s) {
  int Kp, Np;
  uint32_t cols;
  size_t smem;
  if (!fc_dims(a.npair, a.na, a.nb, a.nlink_b, &Kp, &Np, &cols, &smem) || grid < 1) return cudaErrorInvalidValue;
  k_fused_column<<<grid, kFcThreads, smem, s>>>(a, Kp, Np, cols, status);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- batched

__device__ __forceinline__ int find_job(const int *off, int njobs, int item) {
  int lo = 0, hi = njobs;  // off[lo] <= item < off[hi]
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (off[mid] <= item) lo = mid;
    else hi = mid;
  }
  return lo;
}

__global__ void __launch_bounds__(kStepThreads) k_update_batch(BatchTable *bt) {
  __shared__ __align__(16) unsigned char s_upd[kUpdSmemBytes];
  const int nj = bt->njobs;
  const int total = bt->off_step[nj];
  for (int item = blockIdx.x; item < total; item += gridDim.x) {
    const int j = find_job(bt->off_step, nj, item);
    const int vb = item - bt->off_step[j], nvb = bt->off_step[j + 1] - bt->off_step[j];
    const StepArgs &sa = bt->job[j].step;
    const bool halted = sa.sector ? update_body_sym(sa, vb, nvb, s_upd) : update_body(sa, vb, nvb, s_upd);
    if (halted && threadIdx.x == 0) bt->halted[j] = 1;
  }
}

__global__ void __launch_bounds__(kStepThreads) k_project_batch(BatchTable *bt) {
  const int nj = bt->njobs;
  const int total = bt->off_step[nj];
  for (int item = blockIdx.x; item < total; item += gridDim.x) {
    const int j = find_job(bt->off_step, nj, item);
    const int vb = item - bt->off_step[j], nvb = bt->off_step[j + 1] - bt->off_step[j];
    project_body(bt->job[j].step, vb, nvb);
  }
}

// Items in reverse job order: the tensor-core kernel just wrote the G of the
// last jobs, which are the ones still in L2.
__global__ void __launch_bounds__(kScTile, 2) k_scatter_batch(BatchTable *bt) {
  const int nj = bt->njobs;
  const int total = bt->off_sc[nj];
  for (int it = blockIdx.x; it < total; it += gridDim.x) {
    const int item = total - 1 - it;
    const int j = find_job(bt->off_sc, nj, item);
    const int vb = item - bt->off_sc[j], nvb = bt->off_sc[j + 1] - bt->off_sc[j];
    if (scatter_body<float>(bt->job[j].sig, vb, nvb) && threadIdx.x == 0) bt->halted[j] = 1;
  }
}

__global__ void __launch_bounds__(kScTile) k_symfin_batch(BatchTable *bt) {
  const int nj = bt->njobs;
  const int total = bt->off_sf[nj];
  for (int item = blockIdx.x; item < total; item += gridDim.x) {
    const int j = find_job(bt->off_sf, nj, item);
    const int vb = item - bt->off_sf[j], nvb = bt->off_sf[j + 1] - bt->off_sf[j];
    if (symfin_body<float>(bt->job[j].sig, vb, nvb) && threadIdx.x == 0) bt->halted[j] = 1;
  }
}

__global__ void __launch_bounds__(kTcThreads, 2)
    k_tc_batch(BatchTable *bt, int Kpmax, int Npmax, uint32_t tmem_cols, int *status) {
  extern __shared__ __align__(128) unsigned char smem[];
  TcSmem sm;
  sm.A = reinterpret_cast<float *>(smem);
  sm.Alo = sm.A + kTcM * Kpmax;
  sm.Bhi = reinterpret_cast<uint32_t *>(sm.Alo + kTcM * Kpmax);
  sm.Blo = sm.Bhi + Npmax * Kpmax;
  uint64_t *mbar = reinterpret_cast<uint64_t *>(sm.Blo + Npmax * Kpmax);
  uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(mbar + 1);
  // per-job data of the table, read once: tile offsets, halted flags, inputs
  __shared__ int s_off[kMaxBatch + 1];
  __shared__ int s_halt[kMaxBatch];
  __shared__ const float *s_zf[kMaxBatch];
  __shared__ __align__(16) SigmaArgs s_args;  // the current job's arguments
  sm.sA = smem_u32(sm.A);
  sm.sAlo = smem_u32(sm.Alo);
  sm.sBhi = smem_u32(sm.Bhi);
  sm.sBlo = smem_u32(sm.Blo);
  sm.sbar = smem_u32(mbar);
  const int tid = threadIdx.x, warp = tid >> 5;
  const int nj = bt->njobs;
  const int total = bt->off_tc[nj];
  // contiguous chunks of tiles: a CTA meets one or two jobs, so it loads
  // operand B once or twice
  const int chunk = (total + gridDim.x - 1) / gridDim.x;
  const int first = blockIdx.x * chunk, last = min(total, first + chunk);
  if (first >= last) return;  // uniform: before any TMEM allocation or barrier
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(
                     smem_u32(tmem_slot)),
                 "r"(tmem_cols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(sm.sbar) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  for (int i = tid; i <= nj; i += blockDim.x) s_off[i] = bt->off_tc[i];
  for (int i = tid; i < nj; i += blockDim.x) {
    const CtlState *c = bt->job[i].step.ctl;
    s_halt[i] = c->halt;
    s_zf[i] = c->zf;
  }
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = *tmem_slot;
  uint32_t phase = 0;
  bool ok = true;
  int cur = -1, Kp = 0, Np = 0;
  for (int item = first; item < last && ok; ++item) {
    const int j = find_job(s_off, nj, item);
    if (s_halt[j]) continue;  // block-uniform
    if (j != cur) {
      const uint32_t *src = reinterpret_cast<const uint32_t *>(&bt->job[j].sig);
      uint32_t *dst = reinterpret_cast<uint32_t *>(&s_args);
      for (int i = tid; i < (int)(sizeof(SigmaArgs) / 4); i += blockDim.x) dst[i] = src[i];
      Kp = bt->job[j].Kp;
      Np = bt->job[j].Np;
      __syncthreads();
      tc_load_B(s_args, Kp, Np, sm);  // (ends with a barrier)
      cur = j;
    }
    const long long tile = item - s_off[j];
    if (!s_zf[j]) {  // a batched solve always has its FP32 copy of z; refuse otherwise
      if (tid == 0) atomicOr(status, 4);
      continue;
    }
    ok = tc_tile(s_args, s_zf[j], tile, Kp, Np, sm, tmem, phase);
  }
  if (!ok) {
    if (tid == 0) atomicOr(status, 1);
    mbar_wait(sm.sbar, phase, kWaitIters);  // let the outstanding MMAs drain (bounded)
  }
  fence_before();
  __syncthreads();
  fence_after();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(tmem_cols)
                 : "memory");
}

// Column-fused sector sigma over the table's fused jobs: (job, column) items
// in contiguous chunks per CTA (a CTA meets one or two jobs and loads
// operand B once or twice).
__global__ void __launch_bounds__(kFcThreads, 2)
    k_fused_batch(BatchTable *bt, int Kpmax, int Npmax, uint32_t tmem_cols, int *status) {
  extern __shared__ __align__(128) unsigned char smem[];
  const FcSmem sm = fc_carve(smem, Kpmax, Npmax);
  __shared__ int s_off[kMaxBatch + 1];
  __shared__ int s_halt[kMaxBatch];
  __shared__ const float *s_zf[kMaxBatch];
  __shared__ __align__(16) SigmaArgs s_args;  // the current job's arguments
  const int tid = threadIdx.x;
  const int nj = bt->njobs;
  const int total = bt->off_fc[nj];
  const int chunk = (total + gridDim.x - 1) / gridDim.x;
  const int first = blockIdx.x * chunk, last = min(total, first + chunk);
  if (first >= last) return;  // uniform: before any TMEM allocation or barrier
  fc_begin(sm, tmem_cols);
  for (int i = tid; i <= nj; i += blockDim.x) s_off[i] = bt->off_fc[i];
  for (int i = tid; i < nj; i += blockDim.x) {
    const CtlState *c = bt->job[i].step.ctl;
    s_halt[i] = c->halt;
    s_zf[i] = c->zf;
  }
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = *fc_tmem_slot(sm);
  uint32_t phase = 0;
  int pending = 0;
  bool ok = true;
  int cur = -1, Kp = 0, Np = 0;
  for (int item = first; item < last && ok; ++item) {
    const int j = find_job(s_off, nj, item);
    if (s_halt[j]) continue;  // block-uniform
    if (!s_zf[j] || !bt->job[j].sig.symA || !bt->job[j].sig.fc_link_a) {  // a fused job has all three
      if (tid == 0) atomicOr(status, 4);
      continue;
    }
    if (j != cur) {
      const uint32_t *src = reinterpret_cast<const uint32_t *>(&bt->job[j].sig);
      uint32_t *dst = reinterpret_cast<uint32_t *>(&s_args);
      for (int i = tid; i < (int)(sizeof(SigmaArgs) / 4); i += blockDim.x) dst[i] = src[i];
      Kp = bt->job[j].Kp;
      Np = bt->job[j].Np;
      __syncthreads();
      fc_load_links(s_args, sm);
      fc_load_B(s_args, Kp, Np, sm);  // (ends with a barrier)
      cur = j;
    }
    ok = fc_column(s_args, s_zf[j], item - s_off[j], Kp, Np, sm, tmem, phase, &pending);
  }
  fc_end(sm, ok, pending, phase, tmem, tmem_cols, status);
}

// Ends a batched loop body (kMaxBatch threads, one per job): resets the tile
// queue, counts the body, and ends the while-loop when a solve halted (or the
// table is empty), so the host can act on it.
__global__ void __launch_bounds__(kMaxBatch) k_batch_end(BatchTable *bt, unsigned long long cond) {
  const int j = threadIdx.x, nj = bt->njobs;
  int h = 0;
  if (j < nj) {
    if (bt->job[j].step.ctl->halt) bt->halted[j] = 1;
    h = bt->halted[j];
  }
  const int stop = __syncthreads_or(h) || nj == 0;
  if (j == 0) {
    bt->tc_next = 0u;
    bt->bodies += 1ull;
    bt->stop = stop;
    if (stop && cond) cudaGraphSetConditional((cudaGraphConditionalHandle)cond, 0u);
  }
}

cudaError_t batch_config(int num_sms, const BatchClass &k, BatchConfig *cfg) {
  const int Kp = k.Kp, Np = k.Np;
  if (Kp < 8 || Np < 16 || Kp % 8 || Np % 16 || Np > 256) return cudaErrorInvalidValue;
  cfg->Kp = Kp;
  cfg->Np = Np;
  cfg->mask = k.mask | (1u << BK_UPDATE) | (1u << BK_PROJECT) | (1u << BK_END);
  cfg->cols = 32;
  while (cfg->cols < (uint32_t)Np) cfg->cols <<= 1;
  cfg->smem = (size_t)(2 * kTcM * Kp + 2 * Np * Kp) * 4 + 16;
  if (cfg->smem > 227 * 1024) return cudaErrorInvalidValue;

  // the opt-in limit is a property of the function, shared by every class and
  // context: always the largest the device allows (minus the kernel's static
  // shared memory), so no later setting can fail a launch
  int optin = 0;
  cudaError_t e = max_dynamic_smem((const void *)k_tc_batch, &optin);
  if (e != cudaSuccess) return e;
  if ((int)cfg->smem > optin) return cudaErrorInvalidValue;
  e = cudaFuncSetAttribute(k_tc_batch, cudaFuncAttributeMaxDynamicSharedMemorySize, optin);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(k_tc_batch, cudaFuncAttributePreferredSharedMemoryCarveout,
                           cudaSharedmemCarveoutMaxShared);
  if (e != cudaSuccess) return e;
  int per_sm = resident_ctas((const void *)k_tc_batch, kTcThreads, cfg->smem);
  if ((uint32_t)per_sm * cfg->cols > 512) per_sm = (int)(512 / cfg->cols);
  cfg->tc_per_sm_max = per_sm;
  // the column kernel (sized for the largest fused job)
  cfg->fKp = k.fKp;
  cfg->fNp = k.fNp;
  cfg->fcols = 2u * (uint32_t)fc_acc_stride(k.fNp);
  cfg->fsmem = fc_smem_bytes(k.fKp, k.fNp);
  cfg->fc_per_sm_max = 1;
  if (cfg->mask & (1u << BK_FUSED)) {
    if (k.fKp < 8 || k.fNp < 16 || cfg->fcols > 512 || cfg->fsmem > 227 * 1024) return cudaErrorInvalidValue;
    cfg->fc_per_sm_max = fc_prepare((const void *)k_fused_batch, cfg->fsmem, cfg->fcols);
    if (cfg->fc_per_sm_max < 1) return cudaErrorInvalidValue;
  }
  // defaults until the autotuner has measured this class
  cfg->ctas[BK_UPDATE] = 2 * num_sms;
  cfg->ctas[BK_PROJECT] = 4 * num_sms;
  cfg->ctas[BK_TC] = num_sms * per_sm;
  cfg->ctas[BK_FUSED] = num_sms * cfg->fc_per_sm_max;
  cfg->ctas[BK_SCATTER] = 3 * num_sms;
  cfg->ctas[BK_SYMFIN] = 2 * num_sms;
  cfg->ctas[BK_END] = 1;
  return cudaSuccess;
}

cudaError_t launch_batch_kernel(int which, const BatchConfig &cfg, BatchTable *d_table, int *status,
                                unsigned long long cond, cudaStream_t s) {
  switch (which) {
    case BK_UPDATE: k_update_batch<<<cfg.ctas[BK_UPDATE], kStepThreads, 0, s>>>(d_table); break;
    case BK_PROJECT: k_project_batch<<<cfg.ctas[BK_PROJECT], kStepThreads, 0, s>>>(d_table); break;
    case BK_TC:
      k_tc_batch<<<cfg.ctas[BK_TC], kTcThreads, cfg.smem, s>>>(d_table, cfg.Kp, cfg.Np, cfg.cols, status);
      break;
    case BK_FUSED:
      k_fused_batch<<<cfg.ctas[BK_FUSED], kFcThreads, cfg.fsmem, s>>>(d_table, cfg.fKp, cfg.fNp, cfg.fcols, status);
      break;
    case BK_SCATTER: k_scatter_batch<<<cfg.ctas[BK_SCATTER], kScTile, 0, s>>>(d_table); break;
    case BK_SYMFIN: k_symfin_batch<<<cfg.ctas[BK_SYMFIN], kScTile, 0, s>>>(d_table); break;
    case BK_END: k_batch_end<<<1, kMaxBatch, 0, s>>>(d_table, cond); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t build_batch_graph(const BatchConfig &cfg, BatchTable *d_table, int *status, cudaStream_t s,
                              cudaGraph_t *graph, cudaGraphExec_t *exec) {
  cudaError_t e;
  cudaGraph_t g = nullptr;
  if ((e = cudaGraphCreate(&g, 0)) != cudaSuccess) return e;
  cudaGraphConditionalHandle h;
  if ((e = cudaGraphConditionalHandleCreate(&h, g, 1u, cudaGraphCondAssignDefault)) != cudaSuccess) return e;
  cudaGraphNodeParams np{};
  np.type = cudaGraphNodeTypeConditional;
  np.conditional.handle = h;
  np.conditional.type = cudaGraphCondTypeWhile;
  np.conditional.size = 1;
  cudaGraphNode_t node;
  if ((e = cudaGraphAddNode(&node, g, nullptr, nullptr, 0, &np)) != cudaSuccess) return e;
  cudaGraph_t body = np.conditional.phGraph_out[0];
  if ((e = cudaStreamBeginCaptureToGraph(s, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal)) !=
      cudaSuccess)
    return e;
  for (int k = 0; k < BK_COUNT; ++k)
    if (cfg.mask & (1u << k)) launch_batch_kernel(k, cfg, d_table, status, (unsigned long long)h, s);
  cudaGraph_t captured = nullptr;
  e = cudaStreamEndCapture(s, &captured);
  if (e != cudaSuccess) return e;
  if ((e = cudaGraphInstantiate(exec, g, 0)) != cudaSuccess) return e;
  *graph = g;
  return cudaSuccess;
}


}  // namespace sbci
