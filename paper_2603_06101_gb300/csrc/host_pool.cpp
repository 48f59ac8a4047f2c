// Host worker pool of the batched solves (host_pool.h).
#include "host_pool.h"

#include <algorithm>
#include <atomic>
#include <condition_variable>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <thread>
#include <vector>

namespace sbci {

namespace {

class HostPool {
 public:
  explicit HostPool(int workers) {
    for (int w = 0; w < workers; ++w) th_.emplace_back([this] { worker(); });
  }

  void run(int n, const std::function<void(int)> &f) {
    if (n <= 0) return;
    if (n == 1 || th_.empty()) {
      for (int i = 0; i < n; ++i) f(i);
      return;
    }
    std::lock_guard<std::mutex> one(run_mu_);
    {
      std::lock_guard<std::mutex> lk(mu_);
      f_ = &f;
      n_ = n;
      next_.store(0);
      active_ = (int)th_.size();
      ++gen_;
    }
    cv_job_.notify_all();
    for (int i; (i = next_.fetch_add(1)) < n;) f(i);
    std::unique_lock<std::mutex> lk(mu_);
    cv_done_.wait(lk, [&] { return active_ == 0; });  // every worker has left this job
    f_ = nullptr;
  }

 private:
  void worker() {
    unsigned long long seen = 0;
    for (;;) {
      const std::function<void(int)> *f;
      int n;
      {
        std::unique_lock<std::mutex> lk(mu_);
        cv_job_.wait(lk, [&] { return gen_ != seen; });
        seen = gen_;
        f = f_;
        n = n_;
      }
      for (int i; (i = next_.fetch_add(1)) < n;) (*f)(i);
      std::lock_guard<std::mutex> lk(mu_);
      if (--active_ == 0) cv_done_.notify_one();
    }
  }

  std::mutex run_mu_;  // one job at a time
  std::mutex mu_;
  std::condition_variable cv_job_, cv_done_;
  const std::function<void(int)> *f_ = nullptr;
  int n_ = 0;
  std::atomic<int> next_{0};
  int active_ = 0;
  unsigned long long gen_ = 0;
  std::vector<std::thread> th_;
};

HostPool &pool_instance() {
  // never destroyed: the workers block on a condition variable until exit
  static HostPool *p = [] {
    const char *e = std::getenv("SBCI_HOST_THREADS");
    int w = 0;
    if (!(e && std::strcmp(e, "0") == 0)) {
      const int hw = (int)std::thread::hardware_concurrency();
      w = std::max(0, std::min(15, hw - 1));
    }
    return new HostPool(w);
  }();
  return *p;
}

}  // namespace

void host_parallel_for(int n, const std::function<void(int)> &f) { pool_instance().run(n, f); }

}  // namespace sbci
