// Digests of several device byte ranges without allocating any memory.
//
// Some callers cannot call cudaMalloc at the moment they need a digest: code running
// under a caller-owned memory budget or a custom allocator that must not be bypassed, or
// code that must not synchronise the device the way cudaMalloc/cudaFree may.  This entry
// point serves them: it runs the same digest kernel as mpt_hash_device, but the kernel's
// scratch -- one 64-bit accumulator per range -- lives in the file-scope device array
// below instead of memory a context allocated.  Every GPU that loads this library holds
// that array (8 KiB) until the process exits.
//
// Host code must not hand the array's name to a kernel: in host code it is a host-side
// stand-in, not a device address.  The device address is looked up once per device with
// cudaGetSymbolAddress (with that device current) and cached.
#include <mutex>

#include "internal.h"
#include "kernels.cuh"

namespace {

constexpr uint32_t kMaxRanges = MPT_NOALLOC_MAX_RANGES;  // accumulators in the scratch array
constexpr int kMaxDevices = 64;

__device__ __align__(256) unsigned long long g_digest_scratch[kMaxRanges];

std::mutex g_setup_mu;
unsigned long long* g_scratch_addr[kMaxDevices] = {};
int g_sms[kMaxDevices] = {};

// First call on a device: find the scratch array's device address and the SM count.
mpt_status setup_device(int dev, unsigned long long** scratch, int* sms) {
  if (dev < 0 || dev >= kMaxDevices) return mpt::fail(MPT_ENOTSUP, "mpt_hash_ranges_noalloc: device %d", dev);
  std::lock_guard<std::mutex> lock(g_setup_mu);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_digest_scratch);
    if (e != cudaSuccess)
      return mpt::fail(MPT_ECUDA, "mpt_hash_ranges_noalloc: cudaGetSymbolAddress: %s", cudaGetErrorString(e));
    int n = 0;
    e = cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess)
      return mpt::fail(MPT_ECUDA, "mpt_hash_ranges_noalloc: SM count: %s", cudaGetErrorString(e));
    g_sms[dev] = n;
    g_scratch_addr[dev] = static_cast<unsigned long long*>(p);
  }
  *scratch = g_scratch_addr[dev];
  *sms = g_sms[dev];
  return MPT_OK;
}

}  // namespace

extern "C" MPT_API mpt_status mpt_hash_ranges_noalloc(const void* const* ptrs, const uint64_t* nbytes, uint32_t n,
                                                      void* stream, uint64_t* out) {
  if (n > kMaxRanges)
    return mpt::fail(MPT_EINVAL, "mpt_hash_ranges_noalloc: %u ranges exceed the maximum of %u", n, kMaxRanges);
  if (n == 0) return MPT_OK;
  if (!ptrs || !nbytes || !out) return mpt::fail(MPT_EINVAL, "mpt_hash_ranges_noalloc: NULL argument");
  for (uint32_t i = 0; i < n; ++i)
    if (nbytes[i] > 0 && !ptrs[i]) return mpt::fail(MPT_EINVAL, "mpt_hash_ranges_noalloc: range %u is NULL", i);
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return mpt::fail(MPT_ECUDA, "mpt_hash_ranges_noalloc: %s", cudaGetErrorString(e));
  unsigned long long* scratch = nullptr;
  int sms = 0;
  mpt_status st = setup_device(dev, &scratch, &sms);
  if (st != MPT_OK) return st;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  // The array keeps the previous call's sums: clear the accumulators this call uses.
  e = cudaMemsetAsync(scratch, 0, n * sizeof(unsigned long long), s);
  if (e != cudaSuccess) return mpt::fail(MPT_ECUDA, "mpt_hash_ranges_noalloc: %s", cudaGetErrorString(e));
  for (uint32_t i = 0; i < n; ++i) {
    const uint64_t words = (nbytes[i] + 7) / 8;
    const uint64_t want = (words + 255) / 256;
    const uint32_t blocks = (uint32_t)(want < 1 ? 1 : (want > 4ull * (uint64_t)sms ? 4ull * (uint64_t)sms : want));
    mpt::k_hash<<<blocks, 256, 0, s>>>(static_cast<const uint8_t*>(ptrs[i]), nbytes[i], scratch + i);
  }
  e = cudaGetLastError();
  if (e != cudaSuccess) return mpt::fail(MPT_ECUDA, "mpt_hash_ranges_noalloc: launch: %s", cudaGetErrorString(e));
  e = cudaMemcpyAsync(out, scratch, n * sizeof(unsigned long long), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return mpt::fail(MPT_ECUDA, "mpt_hash_ranges_noalloc: %s", cudaGetErrorString(e));
  return MPT_OK;
}
