// Device job table of the batched step kernels (kernels_loop.cu): every
// active solve of a serving batch is one job; the kernels walk the table as a
// work queue of (job, virtual block) items, so one launch of each step kernel
// serves all solves whatever their determinant counts.
#pragma once

#include <cuda_runtime.h>

#include "ctl.h"
#include "sbci_internal.h"
#include "step.h"

namespace sbci {

constexpr int kMaxBatch = 64;

struct BatchJob {
  StepArgs step;  // update / projection arguments (cond = 0)
  SigmaArgs sig;  // sigma arguments (ctl set, cond = 0)
  int Kp, Np;     // tensor-core operand sizes of this solve
  int fused;      // 1: its sigma is the column-fused sector kernel (no tile kernel, no scatter)
};

struct BatchTable {
  int njobs;
  int off_step[kMaxBatch + 1];  // prefix sums of the update / projection virtual blocks
  int off_sc[kMaxBatch + 1];    // prefix sums of the scatter virtual blocks
  int off_tc[kMaxBatch + 1];    // prefix sums of the 128-determinant tensor-core tiles
  int off_sf[kMaxBatch + 1];    // prefix sums of the symmetric-finish virtual blocks (0 if none)
  int off_fc[kMaxBatch + 1];    // prefix sums of the column-fused sigma's columns (0 unless fused)
  unsigned int tc_next;         // work-queue head of the tensor-core kernel
  unsigned long long bodies;    // loop bodies run (BK_COUNT kernels each)
  int stop;                     // the last body ended with a halted solve
  int halted[kMaxBatch];        // set by a job's last block when its controller halts
  BatchJob job[kMaxBatch];
};

// Largest orbital-pair count a batched solve may have (n <= 14: Kp = Np =
// 112, 215 KB of shared memory per tensor-core CTA).
constexpr int kBatchMaxPair = 105;


// The kernels of one batched loop body, in launch order: the tile kernel and
// the scatter serve the solves whose sigma is not column-fused, the column
// kernel the singlet-sector solves with at most 256 strings per spin, the
// symmetric finish every singlet-sector solve (the others finish in the
// scatter).  A class's graph launches only the kernels its tables use.
enum BatchKernel { BK_UPDATE = 0, BK_PROJECT, BK_TC, BK_FUSED, BK_SCATTER, BK_SYMFIN, BK_END, BK_COUNT };

// Launch shapes of the batched kernels on a device with num_sms SMs for one
// operand class: the tensor-core buffers are sized for the largest Kp x Np of
// the jobs in the table (so a table of small solves fits more CTAs per SM).
struct BatchConfig {
  int Kp, Np;          // tensor-core operand buffers (multiples of 8 and 16)
  uint32_t cols;       // TMEM columns per tensor-core CTA
  size_t smem;         // dynamic shared memory of the tensor-core kernel
  int tc_per_sm_max;   // tensor-core CTAs that fit one SM (shared memory, TMEM)
  int fKp, fNp;        // operand buffers of the column kernel (largest of the fused jobs)
  uint32_t fcols;      // TMEM columns per column CTA (two accumulators)
  size_t fsmem;        // dynamic shared memory of the column kernel
  int fc_per_sm_max;   // column CTAs that fit one SM
  unsigned mask;       // bit k set: kernel k is launched (it has work in this class)
  int ctas[BK_COUNT];  // CTAs of each kernel of the body (the autotuner's choice)
};

// Kernels a table needs (bits of BatchConfig::mask) and its operand class:
// the largest Kp / Np of the tile-kernel jobs and of the column-kernel jobs.
struct BatchClass {
  int Kp, Np, fKp, fNp;
  unsigned mask;
};
BatchClass table_class(const BatchTable &t);

cudaError_t batch_config(int num_sms, const BatchClass &k, BatchConfig *cfg);

// One kernel of the body; cond = 0 outside a graph (the end kernel then only
// records the stop flag).
cudaError_t launch_batch_kernel(int which, const BatchConfig &cfg, BatchTable *d_table, int *status,
                                unsigned long long cond, cudaStream_t s);

// Captures the batched step body into a CUDA graph while-loop over the table.
cudaError_t build_batch_graph(const BatchConfig &cfg, BatchTable *d_table, int *status, cudaStream_t s,
                              cudaGraph_t *graph, cudaGraphExec_t *exec);

}  // namespace sbci
