// Host-side check of the host-thread staging pool (no GPU): several caller threads copy
// ragged ranges through one pool at once; every destination must equal the source byte for
// byte, bytes around it must be untouched, and the pool must shut down with idle workers.
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <random>
#include <thread>
#include <vector>

#include "host_pool.h"

static int check(mpt::HostCopyPool& pool, unsigned caller, unsigned rounds) {
  std::mt19937_64 rng(0x5EED0000u + caller);
  for (unsigned r = 0; r < rounds; ++r) {
    const size_t sizes[] = {0, 1, 63, 4096, mpt::HostCopyPool::kMinPart - 1, mpt::HostCopyPool::kMinPart + 7,
                            3 * mpt::HostCopyPool::kMinPart + 5, (size_t)(rng() % (9u << 20))};
    for (size_t n : sizes) {
      const size_t so = rng() % 64, dof = rng() % 64, pad = 64;
      std::vector<uint8_t> src(n + so + pad), dst(n + dof + 2 * pad, 0xA5);
      for (auto& b : src) b = (uint8_t)rng();
      pool.copy(dst.data() + pad + dof, src.data() + so, n);
      if (std::memcmp(dst.data() + pad + dof, src.data() + so, n) != 0) {
        std::fprintf(stderr, "caller %u: copy of %zu bytes differs\n", caller, n);
        return 1;
      }
      for (size_t i = 0; i < pad + dof; ++i)
        if (dst[i] != 0xA5) return std::fprintf(stderr, "caller %u: wrote before the range\n", caller), 1;
      for (size_t i = pad + dof + n; i < dst.size(); ++i)
        if (dst[i] != 0xA5) return std::fprintf(stderr, "caller %u: wrote past the range\n", caller), 1;
    }
  }
  return 0;
}

int main() {
  for (unsigned workers : {0u, 1u, 3u, 7u}) {
    mpt::HostCopyPool pool(workers);
    std::vector<int> rc(4, 0);
    std::vector<std::thread> callers;
    for (unsigned c = 0; c < rc.size(); ++c) callers.emplace_back([&, c] { rc[c] = check(pool, c, 6); });
    for (auto& t : callers) t.join();
    for (int v : rc)
      if (v) return 1;
    std::printf("workers=%u ok\n", workers);
  }
  { mpt::HostCopyPool idle(5); }  // destroyed without any work
  std::printf("all ok\n");
  return 0;
}
