// Internal declarations shared by the host C++ and the CUDA translation units
// of libsbci.  Nothing here is part of the C ABI (see include/sbci.h).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/sbci.h"

namespace sbci {

struct CtlState;

// ---------------------------------------------------------------------------
// Packed excitation-table entry.  For string I, entry e encodes
//   a+_k a_l |I> = sign |J>  as  J | pair(k,l) << 20 | (sign < 0) << 31.
// J < 2^20 strings, pair < 2^11.
constexpr uint32_t kJMask = (1u << 20) - 1u;
constexpr int kPairShift = 20;
constexpr uint32_t kPairMask = (1u << 11) - 1u;
constexpr uint32_t kSignBit = 1u << 31;

__host__ __device__ inline int link_J(uint32_t v) { return (int)(v & kJMask); }
__host__ __device__ inline int link_pair(uint32_t v) { return (int)((v >> kPairShift) & kPairMask); }
__host__ __device__ inline bool link_neg(uint32_t v) { return (v & kSignBit) != 0u; }

#ifdef __CUDACC__
// (Ia, Ib) of flat determinant index I = Ia * nb + Ib.  Determinant counts
// stay below 2^31 (the largest space, n = 16, has 165.6 M), so 32-bit
// unsigned division suffices; 64-bit division is a long instruction sequence.
__device__ __forceinline__ void split_det(long long I, int nb, int &ia, int &ib) {
  const unsigned u = (unsigned)I, q = u / (unsigned)nb;
  ia = (int)q;
  ib = (int)(u - q * (unsigned)nb);
}

// Unit u of the T (T + 1) / 2 pairs of 32 x 32 tiles (ti, tj), ti >= tj, of
// a square matrix (row-major over ti): the work units of the kernels that
// read a tile and its transpose together.
__device__ __forceinline__ void tri_unit(int u, int *ti, int *tj) {
  int t = (int)((sqrtf(8.0f * (float)u + 1.0f) - 1.0f) * 0.5f);
  while (t * (t + 1) / 2 > u) --t;
  while ((t + 1) * (t + 2) / 2 <= u) ++t;
  *ti = t;
  *tj = u - t * (t + 1) / 2;
}

// Visits the links of one string U at a time: the U list entries, then the U
// gathered values (independent loads, all in flight), then the U updates.
// Entry e of the list is lst[e * stride] (stride 1: a row of a [N][nlink]
// table; stride N: a column of the transposed [nlink][N] table, whose loads
// coalesce across threads that hold consecutive strings).
// load(v) returns the gathered value of link word v; use(v, x) consumes it.
template <int U, typename T, typename Load, typename Use>
__device__ __forceinline__ void for_links(const uint32_t *lst, int n, long long stride, Load load, Use use) {
  int e = 0;
  for (; e + U <= n; e += U) {
    uint32_t v[U];
    T x[U];
#pragma unroll
    for (int j = 0; j < U; ++j) v[j] = __ldg(lst + (e + j) * stride);
#pragma unroll
    for (int j = 0; j < U; ++j) x[j] = load(v[j]);
#pragma unroll
    for (int j = 0; j < U; ++j) use(v[j], x[j]);
  }
  if (e < n) {  // the partial last batch: predicated, its loads still issued together
    const int m = n - e;
    uint32_t v[U];
    T x[U];
#pragma unroll
    for (int j = 0; j < U; ++j)
      if (j < m) v[j] = __ldg(lst + (e + j) * stride);
#pragma unroll
    for (int j = 0; j < U; ++j)
      if (j < m) x[j] = load(v[j]);
#pragma unroll
    for (int j = 0; j < U; ++j)
      if (j < m) use(v[j], x[j]);
  }
}


// The same visit with the list loads of batch k + 1 issued before the
// gathered values of batch k are used, so each batch waits for one memory
// round trip (its values) instead of two (entries, then values).  Same order
// of use as for_links.
template <int U, typename T, typename Load, typename Use>
__device__ __forceinline__ void for_links_pipelined(const uint32_t *lst, int n, long long stride, Load load,
                                                    Use use) {
  uint32_t v[U];
#pragma unroll
  for (int j = 0; j < U; ++j)
    if (j < n) v[j] = __ldg(lst + j * stride);
  for (int e = 0; e < n; e += U) {
    const int m = n - e;
    T x[U];
#pragma unroll
    for (int j = 0; j < U; ++j)
      if (j < m) x[j] = load(v[j]);
    uint32_t vn[U];
#pragma unroll
    for (int j = 0; j < U; ++j)
      if (e + U + j < n) vn[j] = __ldg(lst + (e + U + j) * stride);
#pragma unroll
    for (int j = 0; j < U; ++j)
      if (j < m) use(v[j], x[j]);
#pragma unroll
    for (int j = 0; j < U; ++j) v[j] = vn[j];
  }
}
#endif

constexpr int kMaxOrb = 16;
constexpr int kMaxPair = kMaxOrb * (kMaxOrb + 1) / 2;  // 136
constexpr int kMaxStates = 8;

// Host-side string data of one spin.
struct StringSet {
  int norb = 0, nelec = 0, nstr = 0, nlink = 0;
  std::vector<uint32_t> masks;  // increasing
  std::vector<uint32_t> links;  // [nstr][nlink]
};
void build_strings(int norb, int nelec, StringSet &out);

// ---------------------------------------------------------------------------
// Dot-product slots of the per-step reduction buffer.
enum Slot : int {
  S_NXX = 0, S_NXY, S_NYY, S_HXX, S_HXY, S_HYY, S_ZPZP,   // written by the update sweep
  S_NXZ, S_NYZ, S_NZZ,                                   // update (no projection) or project
  S_HXZ, S_HYZ, S_HZZ,                                   // sigma epilogue
  S_XCW0,                                                // x_c^i . w, i < kMaxStates
  S_GEN0 = S_XCW0 + kMaxStates,                          // general-purpose dots
  S_YDY = S_GEN0 + 16,                                   // y . (D y) of the update (Eq. S136 diagnostic)
  S_COUNT
};

// Arguments of the sigma kernels for one vector.
struct SigmaArgs {
  const double *c;       // [Na*Nb]
  const float *cf;       // FP32 copy of c for the tensor-core gather (plain calls)
  double *sigma;         // [Na*Nb]
  void *G;               // [npair][ndet] FP64 or FP32 scratch
  const uint32_t *link_a, *link_b;
  const uint32_t *link_bT;  // beta lists transposed, [nlink_b][nb]
  const double *W;       // [npair_pad][npair] FP64 (rows padded with zeros)
  const float *Wf;       // FP32 copy (same layout), SBCI_FP32 mode
  const uint32_t *Wtc;   // TF32 hi then lo of W in the tensor-core operand layout
                         // ([2][Np*Kp], see tc_body.cuh), or nullptr
  const uint16_t *fc_link_a;  // alpha links for the column-fused kernel, [na][nlink_a] of
                              // J | pair << 8 | (sign < 0) << 15, or nullptr
  int na, nb, nlink_a, nlink_b, npair, npair_pad;
  long long ndet;
  // epilogue dots of sigma against up to three vectors (nullptr = unused)
  const double *dot_u[3];
  int dot_slot[3];
  double *partials;      // [S_COUNT][grid]
  int grid;
  // singlet-sector split (c = c^T exactly, n_alpha = n_beta): the scatter
  // writes only the alpha part A (AccT, [Na][Nb]) here, and sigma = A + A^T is
  // formed by the symmetric finish, which also takes the dots (nullptr: off)
  void *symA;
  int sf_grid;           // virtual blocks of the symmetric finish
  // device-controlled mode (ctl != nullptr): input z and output Z come from the
  // controller, the scatter's dots are against (dot_u[0], dot_u[1], ctl->zn),
  // and its last block runs the subspace solve
  struct CtlState *ctl;
  unsigned int *counter;       // last-block counter of the scatter
  unsigned long long cond;     // graph while-loop handle (0: none)
};

// Launchers (kernels_sigma.cu)
// prec: 0 = FP64 scratch and contraction, 1 = FP32 (SIMT) contraction
cudaError_t launch_gather_contract(const SigmaArgs &a, int prec, cudaStream_t s);
cudaError_t launch_scatter(const SigmaArgs &a, int prec, cudaStream_t s);
// Virtual blocks of the scatter: min(256-determinant tiles, 8 x SMs).
int scatter_grid(long long ndet, int nsm);
// Virtual blocks of the symmetric finish: min(32 x 32 tile pairs, 8 x SMs).
int symfin_grid(int na, int nsm);
cudaError_t launch_symfin(const SigmaArgs &a, int prec, cudaStream_t s);
cudaError_t prepare_sigma_kernels();
// tcgen05 TF32x3 gather + contract (kernels_loop.cu); writes FP32 G like prec 1.
bool tc_dims(int npair, int *Kp, int *Np, uint32_t *cols, size_t *smem);
int tc_grid(int npair, long long ndet, int num_sms);
// Writes W (FP64 [npair_pad][npair]) as TF32 hi/lo operand B, [2][Np*Kp].
cudaError_t launch_split_W(const double *W, int npair, int Kp, int Np, uint32_t *out, cudaStream_t s);
cudaError_t launch_gather_contract_tc(const SigmaArgs &a, int *status, int grid, cudaStream_t s);
// The same contraction with the epilogue of one tile overlapped with the
// gather and MMAs of the next (kernels_tcp.cu: 8 gather warps, 4 epilogue
// warps, two TMEM accumulators); writes the same G.
int tcp_grid(int npair, long long ndet, int num_sms);  // 0: unsupported shape
cudaError_t launch_gather_contract_tcp(const SigmaArgs &a, int *status, int grid, cudaStream_t s);
// Column-fused TF32x3 sigma of the singlet sector (kernels_loop.cu,
// fused_body.cuh): gather, contraction and alpha-only scatter of one column
// of A per CTA step, G kept in shared memory; device-controlled mode only
// (input z from the controller's FP32 copy, A^T written to a.symA).
// Supported for n_alpha = n_beta strings per spin <= 256.
bool fc_dims(int npair, int na, int nb, int nlink_b, int *Kp, int *Np, uint32_t *cols, size_t *smem);
int fc_grid(int npair, int na, int nb, int nlink_b, int num_sms);  // 0: unsupported shape
cudaError_t launch_fused_column(const SigmaArgs &a, int *status, int grid, cudaStream_t s);
// tcgen05 BF16x3 gather + contract (kernels_bf.cu) for npair <= 136; writes
// FP32 G like prec 1.  W as BF16 hi / lo operand B: bf_W_elems(npair) uint16,
// made once per context by launch_split_W_bf.
bool bf_dims(int npair, int *Kp, int *Np, uint32_t *cols, size_t *smem);
int bf_grid(int npair, long long ndet, int num_sms);  // 0: unsupported shape
size_t bf_W_elems(int npair);
cudaError_t launch_split_W_bf(const double *W, int npair, uint16_t *out, cudaStream_t s);
cudaError_t launch_gather_contract_bf(const SigmaArgs &a, const uint16_t *Wbf, int *status, int grid,
                                      cudaStream_t s);
// Factored (density-fitted) TF32x3 gather + contract (kernels_tclr.cu):
// W = F M F^T of rank rr (lowrank.h), G = (D F)(F M)^T as two chained tcgen05
// products per tile; writes FP32 G like prec 1.  The factor as pre-split
// operands, tclr_W_words(npair, rr) words from launch_split_lr_tc (Ut = F^T
// [rr][npair], UL = F M [npair][rr], FP64).
bool tclr_dims(int npair, int rr, int *Kp, int *Np, int *Rp, uint32_t *cols, size_t *smem);
size_t tclr_W_words(int npair, int rr);  // 0: unsupported shape
cudaError_t launch_split_lr_tc(const double *Ut, const double *UL, int rr, int npair, uint32_t *out,
                               cudaStream_t s);
int tclr_grid(int npair, int rr, long long ndet, int num_sms);  // 0: unsupported shape
cudaError_t launch_gather_contract_tclr(const SigmaArgs &a, const uint32_t *Wlr, int rr, int *status, int grid,
                                        cudaStream_t s);
size_t sigma_scratch_bytes(int npair, long long ndet, int prec);

// Helper kernels (kernels_vec.cu)
// out = (float) in, elementwise.
cudaError_t launch_to_float(const double *in, float *out, long long n, cudaStream_t s);
// out = sum_i coef_i in_i (out may alias in[0]); up to 8 inputs.
cudaError_t launch_lincomb(double *out, const double *const *in, const double *coef, int nin,
                           long long n, cudaStream_t s);
// partial dots of up to 16 (u, v) pairs into slots S_GEN0 + i.
cudaError_t launch_dots(const double *const *u, const double *const *v, int npairs, long long n,
                        double *partials, int grid, cudaStream_t s);
// result[slot] = sum of partials[slot][0..grid) in fixed order, slots [s0, s1).
cudaError_t launch_reduce(const double *partials, int grid, int s0, int s1, double *result,
                          cudaStream_t s);
// D_I from per-string energies and ja[Ia][q] = sum_{p in a} (pp|qq).
cudaError_t launch_diagonal(double *diag, const double *ea, const double *eb, const double *ja,
                            const uint32_t *mask_b, int na, int nb, int norb, cudaStream_t s);
cudaError_t launch_symmetrize(double *v, int n, cudaStream_t s);
// dst[pairs[2 q]] = pairs[2 q + 1], q < n (indices stored as exact doubles).
cudaError_t launch_sparse_set(double *dst, const double *pairs, int n, cudaStream_t s);
// out[q] = src[offs[q]], q < n (offsets stored as exact doubles).
cudaError_t launch_gather_at(const double *src, const double *offs, int n, double *out, cudaStream_t s);
// r[I] = SplitMix64 vector of (seed, alpha) in [-1, 1)
cudaError_t launch_splitmix(double *r, long long n, unsigned long long seed, int alpha, cudaStream_t s);

// Largest dynamic shared memory a launch of kernel f may opt into on the
// current device (the opt-in limit minus f's static shared memory).
cudaError_t max_dynamic_smem(const void *f, int *bytes);

// FP64 gather + contract on the tensor cores by exact BF16 integer slices
// (kernels_os.cu), for npair <= 55.  W slices: os_W_bytes() bytes plus 64
// column exponents, made once per context by launch_split_W_os.
bool os_supported(int npair);
size_t os_W_bytes();
cudaError_t launch_split_W_os(const double *W, int npair, void *out, int *fexp, cudaStream_t s);
cudaError_t prepare_os_kernel(int npair);
int os_grid(long long ndet, int nsm);
cudaError_t launch_gather_contract_os(const SigmaArgs &a, const void *Wos, const int *fexp, int *status, int grid,
                                      cudaStream_t s);

// Kernels of the block Davidson-Liu solver and of the SBCI2 pair steps
// (kernels_dav.cu).
constexpr int kDavMaxSpace = 64;                  // subspace vectors
constexpr int kDavMaxPairs = 2 * kDavMaxSpace;    // dot pairs per launch
constexpr int kDavMaxIn = kDavMaxSpace + 8;       // inputs of one combination
constexpr int kDavMaxOut = 12;                    // outputs of one combination
int dav_dots_grid(long long n, int nsm);
// partials[p * grid + b] = block b's part of u_p . v_p (finish with launch_reduce).
cudaError_t launch_dav_dots(const double *const *u, const double *const *v, int npairs, long long n,
                            double *partials, int grid, cudaStream_t s);
// out_j = sum_q coef[q * nout + j] in_q; an output may be one of the inputs.
cudaError_t launch_dav_combine(double *const *out, int nout, const double *const *in, int nin,
                               const double *coef, long long n, int nsm, cudaStream_t s);
// out <- in / guarded(D - shift) (out may be in)
cudaError_t launch_dav_precond(double *out, const double *in, const double *diag, double shift, double guard,
                               long long n, int nsm, cudaStream_t s);
// The same two with device-resident coefficients / shift (written by the
// SBCI2 pair controller): coef[q * kDavMaxOut + j]; the combination does
// nothing while *active == 0 (active may be null).
cudaError_t launch_dav_combine_dev(double *const *out, int nout, const double *const *in, int nin,
                                   const double *coef, const int *active, long long n, int nsm, cudaStream_t s);
cudaError_t launch_dav_precond_dev(double *out, const double *in, const double *diag, const double *shift,
                                   double guard, long long n, int nsm, cudaStream_t s);

// SBCI2 pair controller kernels (kernels_sbci2.cu, pair_ctl.h), one thread
// each, on the device state of one pair: res holds the reduced dots of the
// step (launch_reduce), cond the graph's while-loop handle (0: none).
struct PairCtl;
cudaError_t launch_pair_proj_coef(PairCtl *ctl, const double *res, cudaStream_t s);
cudaError_t launch_pair_after_dots(PairCtl *ctl, const double *res, cudaStream_t s);
cudaError_t launch_pair_decide(PairCtl *ctl, const double *res, unsigned long long cond, cudaStream_t s);

// ---------------------------------------------------------------------------
// Small dense symmetric eigen-solver (cyclic Jacobi), ascending eigenvalues,
// eigenvectors in columns of V (row-major n x n), n <= kDavMaxSpace.
void jacobi_eigh(int n, const double *A, double *w, double *V);

void set_error(const std::string &msg);
std::string last_error();  // this thread's message (to carry it to another thread)

}  // namespace sbci

struct sbci_ctx;
namespace sbci {
// Fills the sigma arguments of a context without allocating anything (G and
// the dot outputs are left null).  Returns false on a null context.
bool ctx_sigma_args(const sbci_ctx *c, SigmaArgs *a, cudaStream_t *stream);
// Serving support (api.cpp): asynchronous rounds of an active solve.
sbci_status solve_round_launch(sbci_ctx *c);
sbci_status solve_round_finish(sbci_ctx *c, int *done, bool own_graph = true);
// solve_round_finish in two halves, so that the FP64 re-syncs of several
// halted solves (on their own streams) overlap: solve_round_read reads the
// controller and, for a halt whose host work starts with a re-sync, queues it
// and sets *deferred = 1; solve_round_complete then waits for it and finishes
// the halt.  Otherwise the halt is handled at once and *deferred = 0.
sbci_status solve_round_read(sbci_ctx *c, int *done, bool own_graph, int *deferred);
sbci_status solve_round_complete(sbci_ctx *c, int *done);
cudaStream_t ctx_stream(const sbci_ctx *c);
// Makes waiter wait for the work issued so far on the context's stream (the
// host's asynchronous state changes of a halted solve, before a batch round
// that includes it reads its vectors and controller).
cudaError_t ctx_fence(sbci_ctx *c, cudaStream_t waiter);
struct BatchJob;
// Fills the batched-kernel view of an active TF32x3 solve with npair within the
// batched kernels' limit; false if the solve cannot join a batch.
bool ctx_batch_job(sbci_ctx *c, BatchJob *j);
int ctx_step_blocks(const sbci_ctx *c);
int ctx_scatter_blocks(const sbci_ctx *c);
int ctx_symfin_blocks(const sbci_ctx *c);  // 0 unless the solve uses the singlet-sector split
long long ctx_ndet(const sbci_ctx *c);
int ctx_device(const sbci_ctx *c);  // CUDA device the context was created on
long long ctx_launch_count(const sbci_ctx *c);
size_t ctx_device_bytes(int norb, int nalpha, int nbeta, int k);

}  // namespace sbci
