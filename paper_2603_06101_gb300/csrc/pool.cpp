// Caching allocator of the library's buffers (pool.h).
#include "pool.h"

#include <mutex>
#include <unordered_map>
#include <vector>

namespace sbci {

namespace {

struct Block {
  size_t bytes;  // rounded size
  int device;    // -1: pinned host memory
};

struct Pool {
  std::mutex mu;
  // free lists keyed by (device + 1) << 48 | rounded size
  std::unordered_map<unsigned long long, std::vector<void *>> free_list;
  std::unordered_map<void *, Block> live;  // every block the pool handed out and still tracks
  size_t cached = 0;
  long long hits = 0, misses = 0;
};

Pool &pool() {
  static Pool *p = new Pool();  // never destroyed: blocks may be freed during process exit
  return *p;
}

size_t round_size(size_t bytes) { return ((bytes ? bytes : 1) + 255) / 256 * 256; }

unsigned long long key_of(int device, size_t bytes) {
  return ((unsigned long long)(device + 1) << 48) | (unsigned long long)bytes;
}

cudaError_t acquire(void **p, size_t bytes, bool host) {
  *p = nullptr;
  const size_t rb = round_size(bytes);
  int dev = -1;
  if (!host) {
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
  }
  Pool &P = pool();
  if (rb <= kPoolMaxBlock) {
    std::lock_guard<std::mutex> lock(P.mu);
    auto it = P.free_list.find(key_of(dev, rb));
    if (it != P.free_list.end() && !it->second.empty()) {
      *p = it->second.back();
      it->second.pop_back();
      P.cached -= rb;
      ++P.hits;
      return cudaSuccess;
    }
  }
  cudaError_t e = host ? cudaMallocHost(p, rb) : cudaMalloc(p, rb);
  if (e != cudaSuccess) {
    *p = nullptr;
    return e;
  }
  std::lock_guard<std::mutex> lock(P.mu);
  ++P.misses;
  P.live[*p] = Block{rb, dev};
  return cudaSuccess;
}

cudaError_t release(void *p, bool host) {
  if (!p) return cudaSuccess;
  Pool &P = pool();
  Block b{};
  {
    std::lock_guard<std::mutex> lock(P.mu);
    auto it = P.live.find(p);
    if (it == P.live.end()) return host ? cudaFreeHost(p) : cudaFree(p);  // (not the pool's)
    b = it->second;
    if (b.bytes <= kPoolMaxBlock && P.cached + b.bytes <= kPoolMaxCached) {
      P.free_list[key_of(b.device, b.bytes)].push_back(p);
      P.cached += b.bytes;
      return cudaSuccess;
    }
    P.live.erase(it);
  }
  return host ? cudaFreeHost(p) : cudaFree(p);
}

}  // namespace

cudaError_t pool_malloc(void **p, size_t bytes) { return acquire(p, bytes, false); }
cudaError_t pool_free(void *p) { return release(p, false); }
cudaError_t pool_malloc_host(void **p, size_t bytes) { return acquire(p, bytes, true); }
cudaError_t pool_free_host(void *p) { return release(p, true); }

cudaError_t pool_trim() {
  Pool &P = pool();
  std::vector<std::pair<void *, bool>> drop;
  {
    std::lock_guard<std::mutex> lock(P.mu);
    for (auto &kv : P.free_list) {
      const bool host = (kv.first >> 48) == 0;
      for (void *p : kv.second) {
        drop.emplace_back(p, host);
        P.live.erase(p);
      }
    }
    P.free_list.clear();
    P.cached = 0;
  }
  cudaError_t first = cudaSuccess;
  for (auto &d : drop) {
    const cudaError_t e = d.second ? cudaFreeHost(d.first) : cudaFree(d.first);
    if (first == cudaSuccess) first = e;
  }
  return first;
}

void pool_stats(size_t *cached, long long *hits, long long *misses) {
  Pool &P = pool();
  std::lock_guard<std::mutex> lock(P.mu);
  if (cached) *cached = P.cached;
  if (hits) *hits = P.hits;
  if (misses) *misses = P.misses;
}

}  // namespace sbci
