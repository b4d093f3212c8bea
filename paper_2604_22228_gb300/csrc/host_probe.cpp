// Host-memory bandwidth probe: the bound that every host-link route shares with the CPU.
//
// Copy engines, the zero-copy kernel and the staged paths all read or write page-locked host
// memory through the host link (Sec. 4.3 host-staged path; Sec. 5.2 host-path results).  The
// rate they reach can be capped by the link or by the host memory behind it.  This probe
// streams over a host buffer with CPU threads alone, so that the host memory's own rate can be
// set beside what the GPU paths reach, and measured while they run.
#include <algorithm>
#include <chrono>
#include <cstring>
#include <thread>
#include <vector>

#include "internal.h"

namespace {

double now_s() {
  return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

// Sum of the 8-byte words of [p, p+n): every byte is loaded once.
uint64_t read_words(const uint8_t* p, size_t n) {
  const uint64_t* w = reinterpret_cast<const uint64_t*>(p);
  const size_t nw = n / 8;
  uint64_t a0 = 0, a1 = 0, a2 = 0, a3 = 0;
  size_t i = 0;
  for (; i + 4 <= nw; i += 4) {
    a0 += w[i];
    a1 += w[i + 1];
    a2 += w[i + 2];
    a3 += w[i + 3];
  }
  for (; i < nw; ++i) a0 += w[i];
  return a0 + a1 + a2 + a3;
}

void write_words(uint8_t* p, size_t n, uint64_t v) {
  uint64_t* w = reinterpret_cast<uint64_t*>(p);
  const size_t nw = n / 8;
  for (size_t i = 0; i < nw; ++i) w[i] = v + i;
}

}  // namespace

extern "C" {

mpt_status mpt_host_bandwidth(void* ptr, uint64_t nbytes, uint32_t threads, uint32_t op, uint32_t reps,
                              double* out_gbs) {
  if (!ptr || !out_gbs) return mpt::fail(MPT_EINVAL, "mpt_host_bandwidth: NULL argument");
  if (op > 2) return mpt::fail(MPT_EINVAL, "mpt_host_bandwidth: op %u is not 0 (read), 1 (write) or 2 (copy)", op);
  if (threads == 0 || threads > 1024) return mpt::fail(MPT_EINVAL, "mpt_host_bandwidth: threads must be 1..1024");
  if (nbytes < (uint64_t)threads * 4096 * (op == 2 ? 2 : 1))
    return mpt::fail(MPT_EINVAL, "mpt_host_bandwidth: %llu bytes is too small for %u threads",
                     (unsigned long long)nbytes, threads);
  reps = std::max(1u, reps);
  uint8_t* base = static_cast<uint8_t*>(ptr);
  // op 2 copies the first half into the second; each thread owns a contiguous part
  const uint64_t span = op == 2 ? nbytes / 2 : nbytes;
  const uint64_t part = (span / threads) / 64 * 64;
  std::vector<uint64_t> sink(threads, 0);
  double best = 0;
  for (uint32_t r = 0; r < reps; ++r) {
    std::vector<std::thread> ts;
    ts.reserve(threads);
    const double t0 = now_s();
    for (uint32_t k = 0; k < threads; ++k) {
      ts.emplace_back([&, k]() {
        uint8_t* p = base + k * part;
        if (op == 0) {
          sink[k] += read_words(p, part);
        } else if (op == 1) {
          write_words(p, part, k + r);
        } else {
          std::memcpy(p + span, p, part);
        }
      });
    }
    for (auto& t : ts) t.join();
    const double dt = now_s() - t0;
    // bytes of host memory traffic: read or written once (read), written once (write),
    // read once and written once (copy)
    const double traffic = (double)part * threads * (op == 2 ? 2 : 1);
    best = std::max(best, traffic / dt / 1e9);
  }
  volatile uint64_t keep = 0;
  for (uint64_t s : sink) keep = keep + s;
  (void)keep;
  *out_gbs = best;
  return MPT_OK;
}

}  // extern "C"
