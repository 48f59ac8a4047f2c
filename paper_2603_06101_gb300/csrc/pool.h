// Caching allocator of the library's device and pinned host buffers.
//
// A context allocates a few dozen buffers (link tables, packed operator,
// vectors, reduction scratch, pinned result words) and frees them when it is
// destroyed; cudaMalloc / cudaMallocHost are slow and cudaFree synchronises
// the whole device.  Freed blocks up to kPoolMaxBlock bytes go to per-size
// free lists (per device for device memory) and serve the next request of the
// same rounded size, up to kPoolMaxCached cached bytes in all; larger blocks
// and the overflow go straight back to CUDA.  The caller must have finished
// using a block (its stream synchronised) before it frees it: a cached block
// may be handed to another context at once.  Thread-safe.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>

namespace sbci {

constexpr size_t kPoolMaxBlock = (size_t)256 << 20;   // larger blocks are not cached
constexpr size_t kPoolMaxCached = (size_t)2 << 30;    // cached bytes, device and host together

cudaError_t pool_malloc(void **p, size_t bytes);       // device memory of the current device
cudaError_t pool_free(void *p);                        // nullptr: no-op
cudaError_t pool_malloc_host(void **p, size_t bytes);  // pinned host memory
cudaError_t pool_free_host(void *p);                   // nullptr: no-op

// Frees every cached block; returns the first CUDA error.
cudaError_t pool_trim();
// Bytes currently cached (free, held by the pool) and the allocations served
// from the cache / from CUDA since the process started.
void pool_stats(size_t *cached, long long *hits, long long *misses);

}  // namespace sbci
