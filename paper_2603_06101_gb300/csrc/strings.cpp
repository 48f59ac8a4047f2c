// Host construction of occupation strings and single-excitation tables, a
// small Jacobi eigen-solver for the subspace problems of the initial guess,
// Davidson-Liu and SBCI2, and the density-fitted factor of the packed
// two-electron operator.
//
// The paper represents H over Slater determinants (Results, SBCI1) and leaves
// the determinant machinery to its host program; the conventions here are
// stated in include/sbci.h: strings in increasing bitmask order, addressed by
// the combinatorial number system, excitation entries a+_k a_l |I> = sign |J>
// for l occupied (ascending) and k unoccupied or k == l (ascending).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "lowrank.h"
#include "sbci_internal.h"

namespace sbci {

static long long binom(int n, int k) {
  if (k < 0 || k > n) return 0;
  long long r = 1;
  for (int i = 1; i <= k; ++i) r = r * (n - k + i) / i;
  return r;
}

// C(p, k) for p < 32, k <= 32 (the ranks of the masks of up to 32 orbitals).
struct BinomTable {
  long long c[32][33];
  BinomTable() {
    for (int p = 0; p < 32; ++p)
      for (int k = 0; k <= 32; ++k) c[p][k] = binom(p, k);
  }
};

// Rank of a bitmask among masks of equal popcount: sum_k C(o_k, k) over its
// set bits o_1 < o_2 < ...
static int string_address(uint32_t mask) {
  static const BinomTable T;
  long long a = 0;
  int k = 1;
  for (uint32_t m = mask; m; m &= m - 1u) a += T.c[__builtin_ctz(m)][k++];
  return (int)a;
}

static int popcount32(uint32_t v) {
  int c = 0;
  while (v) {
    v &= v - 1u;
    ++c;
  }
  return c;
}

void build_strings(int norb, int nelec, StringSet &out) {
  out.norb = norb;
  out.nelec = nelec;
  out.nstr = (int)binom(norb, nelec);
  out.nlink = nelec * (norb - nelec + 1);
  out.masks.assign(out.nstr, 0u);
  // enumerate masks of popcount nelec in increasing order (next-permutation of bits)
  if (nelec == 0) {
    out.masks[0] = 0u;
  } else {
    uint32_t v = (nelec == 32) ? 0xffffffffu : ((1u << nelec) - 1u);
    for (int i = 0; i < out.nstr; ++i) {
      out.masks[i] = v;
      uint32_t t = v | (v - 1u);
      v = (t + 1u) | (((~t & (t + 1u)) - 1u) >> (__builtin_ctz(v) + 1));
    }
  }
  out.links.assign((size_t)out.nstr * out.nlink, 0u);
  for (int I = 0; I < out.nstr; ++I) {
    const uint32_t m = out.masks[I];
    int e = 0;
    for (int l = 0; l < norb; ++l) {
      if (!(m >> l & 1u)) continue;
      for (int k = 0; k < norb; ++k) {
        if (k != l && (m >> k & 1u)) continue;
        uint32_t target = m;
        bool neg = false;
        if (k != l) {
          target = (m & ~(1u << l)) | (1u << k);
          const int lo = k < l ? k : l, hi = k < l ? l : k;
          const uint32_t between = m & ((1u << hi) - 1u) & ~((2u << lo) - 1u);
          neg = popcount32(between) & 1;
        }
        const int J = string_address(target);
        const int a = k > l ? k : l, b = k > l ? l : k;
        const uint32_t pair = (uint32_t)(a * (a + 1) / 2 + b);
        out.links[(size_t)I * out.nlink + e] =
            (uint32_t)J | (pair << kPairShift) | (neg ? kSignBit : 0u);
        ++e;
      }
    }
  }
}

void jacobi_eigh(int n, const double *Ain, double *w, double *V) {
  std::vector<double> A(Ain, Ain + (size_t)n * n);
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) V[i * n + j] = (i == j) ? 1.0 : 0.0;
  for (int sweep = 0; sweep < 100; ++sweep) {
    double off = 0.0, diag = 0.0;
    for (int i = 0; i < n; ++i) {
      diag += A[i * n + i] * A[i * n + i];
      for (int j = i + 1; j < n; ++j) off += A[i * n + j] * A[i * n + j];
    }
    if (off <= 1e-36 * (diag + 1e-300)) break;
    for (int p = 0; p < n; ++p) {
      for (int q = p + 1; q < n; ++q) {
        const double apq = A[p * n + q];
        if (apq == 0.0) continue;
        const double app = A[p * n + p], aqq = A[q * n + q];
        const double theta = (aqq - app) / (2.0 * apq);
        const double t = (theta >= 0 ? 1.0 : -1.0) / (std::fabs(theta) + std::sqrt(theta * theta + 1.0));
        const double c = 1.0 / std::sqrt(t * t + 1.0), s = t * c;
        for (int k = 0; k < n; ++k) {  // A <- A J (columns p, q)
          const double akp = A[k * n + p], akq = A[k * n + q];
          A[k * n + p] = c * akp - s * akq;
          A[k * n + q] = s * akp + c * akq;
        }
        for (int k = 0; k < n; ++k) {  // A <- J^T A (rows p, q)
          const double apk = A[p * n + k], aqk = A[q * n + k];
          A[p * n + k] = c * apk - s * aqk;
          A[q * n + k] = s * apk + c * aqk;
        }
        for (int k = 0; k < n; ++k) {  // V <- V J
          const double vkp = V[k * n + p], vkq = V[k * n + q];
          V[k * n + p] = c * vkp - s * vkq;
          V[k * n + q] = s * vkp + c * vkq;
        }
      }
    }
  }
  // sort ascending (selection sort on columns)
  for (int i = 0; i < n; ++i) w[i] = A[i * n + i];
  for (int i = 0; i < n; ++i) {
    int m = i;
    for (int j = i + 1; j < n; ++j)
      if (w[j] < w[m]) m = j;
    if (m != i) {
      std::swap(w[i], w[m]);
      for (int k = 0; k < n; ++k) std::swap(V[k * n + i], V[k * n + m]);
    }
  }
}

// Density-fitted factor of the packed operator (lowrank.h).  A pivoted
// Cholesky of the PSD pair matrix V = (ij|kl) gives V = L L^T up to 1e-13 of
// its largest diagonal; with kappa_P = k_ij and delta_P = [i == j],
//   W = 1/2 L L^T + (kappa delta^T + delta kappa^T) / (2N) = F M F^T,
//   F = [L | kappa | delta],  M = diag(1/2 I_r, [[0, 1/(2N)], [1/(2N), 0]]),
// a factor of rank r + 2 (density-fitted integrals: r <= naux).  Worth it
// when 2 (r + 2) < 0.9 npair; the factorisation stops as soon as r passes
// that bound, so full-rank spaces pay O(npair r^2).  A V that is not positive
// semi-definite leaves more than the small diagonal behind, so the whole
// remainder is checked (1e-12 of the largest diagonal) before the factor is
// trusted.  Returns r + 2 with Ut = F^T [r+2][np] and UL = F M [np][r+2], or
// 0 (keep the full form).
int df_factor(int np, const double *V, const double *kappa, const double *delta, int N,
              std::vector<double> &Ut, std::vector<double> &UL) {
  std::vector<double> d(np);
  double dmax = 0.0;
  for (int P = 0; P < np; ++P) dmax = std::max(dmax, d[P] = V[(size_t)P * np + P]);
  std::vector<double> L;  // columns of the factor, np each
  std::vector<char> used(np, 0);
  int r = 0;
  bool low = dmax > 0.0 && N > 0;
  while (low) {
    int piv = -1;
    double best = 1e-13 * dmax;
    for (int P = 0; P < np; ++P)
      if (!used[P] && d[P] > best) best = d[P], piv = P;
    if (piv < 0) break;
    if (!(2.0 * (r + 1 + 2) < 0.9 * np)) low = false;  // no gain over the full form
    used[piv] = 1;
    const double s = std::sqrt(d[piv]);
    std::vector<double> col(np);
    for (int P = 0; P < np; ++P) {
      double v = V[(size_t)P * np + piv];
      for (int q = 0; q < r; ++q) v -= L[(size_t)q * np + P] * L[(size_t)q * np + piv];
      col[P] = v / s;
    }
    for (int P = 0; P < np; ++P) d[P] -= col[P] * col[P];
    L.insert(L.end(), col.begin(), col.end());
    ++r;
  }
  for (int P = 0; low && P < np; ++P)
    for (int Q = 0; Q <= P; ++Q) {
      double v = V[(size_t)P * np + Q];
      for (int q = 0; q < r; ++q) v -= L[(size_t)q * np + P] * L[(size_t)q * np + Q];
      if (!(std::fabs(v) <= 1e-12 * dmax)) {
        low = false;
        break;
      }
    }
  if (!low) return 0;
  const int rr = r + 2;
  Ut.assign((size_t)rr * np, 0.0);
  UL.assign((size_t)np * rr, 0.0);
  for (int P = 0; P < np; ++P) {
    for (int q = 0; q < r; ++q) {
      Ut[(size_t)q * np + P] = L[(size_t)q * np + P];
      UL[(size_t)P * rr + q] = 0.5 * L[(size_t)q * np + P];
    }
    Ut[(size_t)r * np + P] = kappa[P];
    Ut[(size_t)(r + 1) * np + P] = delta[P];
    UL[(size_t)P * rr + r] = delta[P] / (2.0 * N);
    UL[(size_t)P * rr + r + 1] = kappa[P] / (2.0 * N);
  }
  return rr;
}

}  // namespace sbci
