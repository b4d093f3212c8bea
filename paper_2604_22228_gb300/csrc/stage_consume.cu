// Hop two of the host-to-device staged path (Algorithm 2 StageHostCopy: a chunk's second
// hop runs after its first).  Copy-engine nodes fill the chunks of a device stage from the
// host buffer, and a memset node after each raises that chunk's ready flag.  This one
// consumer kernel, launched beside them in the same graph, walks the chunks' 64 KiB tiles,
// waits (bounded) for each chunk's flag, and moves the tile from the stage to its
// destination.
//
// Flags and tile counters are put back to 0 by a memset node at the head of every replay,
// ordered before the copy-engine nodes and before this kernel.  A replay therefore never
// sees a flag raised by an earlier one, even when an earlier replay's wait gave up part way
// (its CTAs return at once, leaving raised flags and partial counts behind).
//
// The stage is written by copy engines while this kernel runs, so its bytes are read with
// coherent loads after an acquire of the flag, never through the read-only (.nc) path.
#include "copy_device.cuh"
#include "kernels.cuh"

namespace mpt {

__global__ void __launch_bounds__(kVecThreads) k_stage_consume(StageArgs a) {
  __shared__ int ok;
  constexpr uint64_t kTile = kVecTileVecs * 16;
  const uint32_t total = a.nchunks * a.tiles_per_chunk;
  const uint32_t tid = threadIdx.x;
  for (uint32_t t = blockIdx.x; t < total; t += gridDim.x) {
    const uint32_t k = t / a.tiles_per_chunk;
    const uint32_t lt = t - k * a.tiles_per_chunk;
    if (tid == 0) {
      const uint64_t limit = a.wait_ns ? *(volatile const uint64_t*)a.wait_ns : a.timeout_ns;
      const uint64_t deadline = global_ns() + limit;
      int seen = 0;
      while (true) {
        uint32_t v;
        asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(a.ready + k) : "memory");
        if (v != 0) {
          seen = 1;
          break;
        }
        if (global_ns() > deadline) break;
        __nanosleep(128);
      }
      ok = seen;
      if (!seen) record_timeout(a.status, kSiteStageFlag);
    }
    // thread 0's acquire, then the barrier, orders every thread's stage loads after the flag
    __syncthreads();
    if (!ok) return;
    const StageChunk c = a.chunks[k];
    const uint64_t off = (uint64_t)lt * kTile;
    if (off < c.bytes) {
      const uint64_t n = c.bytes - off < kTile ? c.bytes - off : kTile;
      cta_copy<true, true>(a.stage + c.stage_off + off, a.dst + c.dst_off + off, n);
    }
    __syncthreads();
    if (tid == 0) {
      __threadfence();
      atomicAdd(a.done + k, 1u);  // tiles of chunk k moved (read back by tests and tools)
    }
  }
}

}  // namespace mpt
