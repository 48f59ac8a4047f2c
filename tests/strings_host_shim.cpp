// Host build of the library's string-table builder and small eigen-solver
// (csrc/strings.cpp) for the CPU tests, with plain-array entry points for
// ctypes.  Test infrastructure only.
#include <cstring>
#include <string>

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

}  // extern "C"
