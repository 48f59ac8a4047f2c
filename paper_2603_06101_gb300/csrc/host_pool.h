// A fixed pool of host worker threads for the per-solve host work of a
// batched solve: the initial guesses and the handling of halted solves.
// Each task works on its own context and CUDA stream, so the tasks' launches,
// copies and waits overlap instead of queueing behind one another.  The
// workers are created on first use and live until the process exits;
// SBCI_HOST_THREADS=0 (read on first use) runs every task on the calling
// thread.
#pragma once

#include <functional>

namespace sbci {

// Runs f(0), ..., f(n - 1) on the workers and the calling thread and returns
// when all have returned.  One job at a time (concurrent callers queue).  f
// must not throw.
void host_parallel_for(int n, const std::function<void(int)> &f);

}  // namespace sbci
