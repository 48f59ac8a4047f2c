// Host build of the library's string-table builder, small eigen-solver and
// density-fitted factor (csrc/strings.cpp) for the CPU tests, with plain-array
// entry points for ctypes.  Test infrastructure only.
#include <cstring>
#include <string>

#include "lowrank.h"
#include "sbci_internal.h"

namespace sbci {
void set_error(const std::string &) {}  // the library's error slot lives in api.cpp
}  // namespace sbci

extern "C" {

// Sizes of the tables for (norb, nelec): out = nstr, nlink.
int host_string_sizes(int norb, int nelec, int *out) {
  sbci::StringSet s;
  sbci::build_strings(norb, nelec, s);
  out[0] = s.nstr;
  out[1] = s.nlink;
  return 0;
}

// masks [nstr], links [nstr * nlink] (packed entries, see sbci_internal.h).
int host_build_strings(int norb, int nelec, uint32_t *masks, uint32_t *links) {
  sbci::StringSet s;
  sbci::build_strings(norb, nelec, s);
  std::memcpy(masks, s.masks.data(), sizeof(uint32_t) * s.masks.size());
  std::memcpy(links, s.links.data(), sizeof(uint32_t) * s.links.size());
  return 0;
}

void host_jacobi_eigh(int n, const double *A, double *w, double *V) { sbci::jacobi_eigh(n, A, w, V); }

// The density-fitted factor: returns r + 2 (0: full form kept) and copies
// Ut [(r+2) np] and UL [np (r+2)] when they fit cap doubles each.
int host_df_factor(int np, const double *V, const double *kappa, const double *delta, int N, double *Ut,
                   double *UL, long long cap) {
  std::vector<double> a, b;
  const int rr = sbci::df_factor(np, V, kappa, delta, N, a, b);
  if (rr > 0 && (long long)a.size() <= cap && (long long)b.size() <= cap) {
    std::memcpy(Ut, a.data(), sizeof(double) * a.size());
    std::memcpy(UL, b.data(), sizeof(double) * b.size());
  }
  return rr;
}

}  // extern "C"
