// Worker pool for the CPU hop of host-thread staging (see host_pool.h).
#include "host_pool.h"

#include <algorithm>
#include <cstring>

namespace mpt {

HostCopyPool::HostCopyPool(unsigned workers) {
  threads_.reserve(workers);
  for (unsigned i = 0; i < workers; ++i) threads_.emplace_back([this] { worker(); });
}

HostCopyPool::~HostCopyPool() {
  {
    std::lock_guard<std::mutex> g(mu_);
    stop_ = true;
  }
  work_cv_.notify_all();
  for (std::thread& t : threads_) t.join();
}

void HostCopyPool::run(const Part& p) {
  std::memcpy(p.dst, p.src, p.n);
  if (p.call->left.fetch_sub(1, std::memory_order_acq_rel) == 1) {
    std::lock_guard<std::mutex> g(mu_);  // pairs with the waiter's predicate check
    done_cv_.notify_all();
  }
}

bool HostCopyPool::try_run_one() {
  Part p;
  {
    std::lock_guard<std::mutex> g(mu_);
    if (queue_.empty()) return false;
    p = queue_.front();
    queue_.pop_front();
  }
  run(p);
  return true;
}

void HostCopyPool::worker() {
  while (true) {
    Part p;
    {
      std::unique_lock<std::mutex> lk(mu_);
      work_cv_.wait(lk, [this] { return stop_ || !queue_.empty(); });
      if (queue_.empty()) return;  // stopping, and nothing left to copy
      p = queue_.front();
      queue_.pop_front();
    }
    run(p);
  }
}

void HostCopyPool::copy(void* dst, const void* src, size_t n) {
  if (n == 0) return;
  uint8_t* d = static_cast<uint8_t*>(dst);
  const uint8_t* s = static_cast<const uint8_t*>(src);
  const size_t most = (size_t)workers() + 1;
  const size_t parts = std::max<size_t>(1, std::min<size_t>(most, n / kMinPart));
  if (parts == 1) {
    std::memcpy(d, s, n);
    return;
  }
  // Part boundaries on 64-byte multiples (whole cache lines per thread where possible).
  const size_t step = ((n / parts) + 63) & ~(size_t)63;
  Call call;
  std::vector<Part> mine;
  for (size_t off = 0; off < n; off += step) mine.push_back(Part{d + off, s + off, std::min(step, n - off), &call});
  call.left.store(mine.size(), std::memory_order_relaxed);
  {
    std::lock_guard<std::mutex> g(mu_);
    for (size_t i = 1; i < mine.size(); ++i) queue_.push_back(mine[i]);
  }
  work_cv_.notify_all();
  run(mine[0]);
  // Help with queued parts (ours or another caller's) instead of idling, then wait.
  while (call.left.load(std::memory_order_acquire) != 0 && try_run_one()) {
  }
  std::unique_lock<std::mutex> lk(mu_);
  done_cv_.wait(lk, [&] { return call.left.load(std::memory_order_acquire) == 0; });
}

void host_copy_fn(void* arg) {
  HostCopyJob* job = static_cast<HostCopyJob*>(arg);
  job->pool->copy(job->dst, job->src, job->bytes);
  if (job->self_delete) delete job;
}

}  // namespace mpt
