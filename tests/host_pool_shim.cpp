// Host build of the library's worker pool (csrc/host_pool.cpp) for the CPU
// tests: plain entry points for ctypes.  Test infrastructure only.
#include <atomic>
#include <thread>
#include <vector>

#include "host_pool.h"

using namespace sbci;

extern "C" {

// Runs `jobs` jobs of n tasks each; counts[j * n + i] = times task i of job j
// ran; threads[j * n + i] = a small id of the thread that ran it.  Returns the
// number of distinct threads seen.
int host_pool_run(int jobs, int n, int *counts, int *threads) {
  std::vector<std::thread::id> ids;
  std::atomic<int> lock{0};
  for (int j = 0; j < jobs; ++j)
    host_parallel_for(n, [&](int i) {
      // a little work, so that several threads take part
      volatile double x = 0.0;
      for (int k = 0; k < 20000; ++k) x = x + 1e-9 * k;
      __atomic_fetch_add(&counts[j * n + i], 1, __ATOMIC_RELAXED);
      const std::thread::id me = std::this_thread::get_id();
      while (lock.exchange(1)) {
      }
      int id = -1;
      for (size_t q = 0; q < ids.size(); ++q)
        if (ids[q] == me) id = (int)q;
      if (id < 0) {
        ids.push_back(me);
        id = (int)ids.size() - 1;
      }
      lock.store(0);
      threads[j * n + i] = id;
    });
  return (int)ids.size();
}

}  // extern "C"
