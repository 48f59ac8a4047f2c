// Low-rank (density-fitting) form of the sigma contraction (kernels_sigma.cu).
//
// The packed operator W[P, Q] = (ij|kl)/2 + (k_ij d_kl + d_ij k_kl)/(2N) is
// symmetric; with density-fitted integrals, (ij|kl) = sum_A B^A_ij B^A_kl, its
// rank is at most naux + 2.  A context factors it once: a pivoted Cholesky of
// the pair matrix, (ij|kl) = L L^T up to 1e-13 of its largest diagonal, and
// W = F M F^T with F = [L | kappa | delta] (kappa_P = k_ij, delta_P = [i == j])
// and M = diag(I/2, [[0, 1/(2N)], [1/(2N), 0]]), rank r + 2.  When
// 2 (r + 2) < 0.9 npair the FP64 SIMT contraction (npair > 55, beyond the
// exact-slice kernel) forms G = (F M) (F^T D): 2 (r + 2) npair multiply-adds
// per determinant instead of npair^2 (the density-fitted contraction, T = B D
// then G = B^T T, with the Cholesky vectors in place of B).  That contraction
// is bound by GB300's FP64 pipe, so the flops count; the FP32 SIMT one is
// bound by its gathers and keeps the full form (the two-pass form measured
// 2.4x slower there).  The TF32x3 tensor-core contraction has a factored
// kernel of its own (kernels_tclr.cu), two chained products per tile on the
// pre-split factor.
#pragma once

#include <cuda_runtime.h>

#include <vector>

#include "sbci_internal.h"

namespace sbci {

// Ut: [r][npair] (F^T), UL: [npair][r] (F M), r = rank + 2, in the
// precision of the contraction (prec 0: double, else float).
cudaError_t launch_gather_contract_lr(const SigmaArgs &a, int prec, const void *Ut, const void *UL, int r,
                                      cudaStream_t s);

// The factor on the host (strings.cpp): pivoted Cholesky of the pair matrix
// V [np][np] plus the one-electron part (kappa, delta [np], N electrons).
// Returns r + 2 with Ut = F^T [r+2][np] and UL = F M [np][r+2], or 0 when the
// full form is kept.
int df_factor(int np, const double *V, const double *kappa, const double *delta, int N,
              std::vector<double> &Ut, std::vector<double> &UL);

}  // namespace sbci
