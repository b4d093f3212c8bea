// Host-thread copies for the host-staged path's CPU hop (MPT_HS_HOST_THREADS).
//
// Sec. 4.3 stages a chunk through host memory in two hops, the second ordered after the
// first (Algorithm 2 StageHostCopy).  With host-thread staging the host side of the route is
// a CPU copy between the caller's host buffer -- page-locked or ordinary pageable memory --
// and a page-locked slot, and the device side is a copy-engine hop between the slot and
// device memory.  The CPU hop runs as a CUDA host function (a graph host node, or
// cudaLaunchHostFunc on the eager engine's lane stream), which hands the bytes to this pool
// of worker threads and returns when they are all copied.
#pragma once
#include <atomic>
#include <condition_variable>
#include <cstddef>
#include <cstdint>
#include <deque>
#include <mutex>
#include <thread>
#include <vector>

namespace mpt {

class HostCopyPool {
 public:
  explicit HostCopyPool(unsigned workers);
  ~HostCopyPool();
  HostCopyPool(const HostCopyPool&) = delete;
  HostCopyPool& operator=(const HostCopyPool&) = delete;

  // Copy n bytes (non-overlapping ranges) with up to workers() + 1 threads: the range is cut
  // into contiguous parts of at least kMinPart bytes; the caller copies one part itself and
  // helps drain the queue until every part of its own call is done.  Safe to call from
  // several threads at once.
  void copy(void* dst, const void* src, size_t n);
  unsigned workers() const { return (unsigned)threads_.size(); }

  static constexpr size_t kMinPart = 128u << 10;

 private:
  struct Call {
    std::atomic<size_t> left{0};
  };
  struct Part {
    uint8_t* dst;
    const uint8_t* src;
    size_t n;
    Call* call;
  };
  void run(const Part& p);
  void worker();
  bool try_run_one();

  std::vector<std::thread> threads_;
  std::mutex mu_;
  std::condition_variable work_cv_, done_cv_;
  std::deque<Part> queue_;
  bool stop_ = false;
};

// One CPU hop of a chunk: the userData of a host node or host function.
struct HostCopyJob {
  HostCopyPool* pool;
  void* dst;
  const void* src;
  size_t bytes;
  bool self_delete;  // eager launches: the job frees itself after it ran
};

// The host function that runs a HostCopyJob (signature of cudaHostFn_t).
void host_copy_fn(void* job);

}  // namespace mpt
