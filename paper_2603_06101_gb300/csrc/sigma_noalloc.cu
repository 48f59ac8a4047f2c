// sbci_sigma_noalloc: the FP64 sigma build with its scratch in a fixed,
// statically allocated device array, for callers that must not allocate.
//
// Who cannot allocate: code that runs while a CUDA stream is being captured
// into a graph (cudaMalloc is not allowed inside a capture), code embedded in
// a host framework that owns all device memory through its own pool and
// forbids raw allocations, and latency-critical loops where cudaMalloc /
// cudaFree would synchronise the device.  The ordinary sbci_sigma may
// allocate its [npair][Ndet] scratch on first use; this entry point never
// does.
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "../../include/sbci.h"
#include "sbci_internal.h"

namespace sbci {

// The scratch: one array per GPU that loads the library, held until exit.
static __device__ __align__(256) unsigned char g_noalloc_scratch[SBCI_NOALLOC_SCRATCH_BYTES];

namespace {
constexpr int kMaxDevices = 64;
std::mutex g_mu;
void *g_scratch_ptr[kMaxDevices] = {};  // device address of the array, per device

// Host code may not pass the symbol itself to a kernel: in host code it names
// a host-side stand-in.  Look up its device address once per device, with
// that device current.
cudaError_t scratch_address(void **out) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_scratch_ptr[dev]) {
    void *p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_ptr[dev] = p;
  }
  *out = g_scratch_ptr[dev];
  return cudaSuccess;
}
}  // namespace

}  // namespace sbci

using namespace sbci;

extern "C" sbci_status sbci_sigma_noalloc(const sbci_ctx *ctx, const double *c, double *sigma,
                                          void *cuda_stream) {
  SigmaArgs a;
  cudaStream_t s = nullptr;
  if (!ctx_sigma_args(ctx, &a, &s) || !c || !sigma) {
    set_error("sbci_sigma_noalloc: NULL argument");
    return SBCI_ERR_INVALID;
  }
  const size_t need = sigma_scratch_bytes(a.npair, a.ndet, 0);
  if (need > (size_t)SBCI_NOALLOC_SCRATCH_BYTES) {
    set_error("sbci_sigma_noalloc: this space needs " + std::to_string(need) +
              " bytes of sigma scratch, more than the fixed " +
              std::to_string((size_t)SBCI_NOALLOC_SCRATCH_BYTES) + "; use sbci_sigma");
    return SBCI_ERR_INVALID;
  }
  // the kernels run on the context's device, and the scratch address below is
  // the array on the current device: the two must be the same GPU
  int cur = -1;
  if (cudaGetDevice(&cur) != cudaSuccess || cur != ctx_device(ctx)) {
    set_error("sbci_sigma_noalloc: the current CUDA device (" + std::to_string(cur) +
              ") is not the context's device (" + std::to_string(ctx_device(ctx)) +
              "); make the context's device current first");
    return SBCI_ERR_INVALID;
  }
  if (cuda_stream) s = (cudaStream_t)cuda_stream;
  void *G = nullptr;
  cudaError_t e = scratch_address(&G);
  if (e == cudaSuccess) {
    a.c = c;
    a.sigma = sigma;
    a.G = G;  // fully overwritten by the gather+contract kernel before it is read
    e = launch_gather_contract(a, 0, s);
  }
  if (e == cudaSuccess) e = launch_scatter(a, 0, s);
  if (e != cudaSuccess) {
    set_error(std::string("sbci_sigma_noalloc: ") + cudaGetErrorString(e));
    return SBCI_ERR_CUDA;
  }
  return SBCI_OK;
}
