// Data-moving kernels of the transfer paths, written for sm_103a.
//
//  k_sm_copy_vec   SM copy kernel, 128-bit loads/stores: each CTA walks 64 KiB tiles of
//                  the ranges it is given, every thread keeping eight 16-byte vectors in
//                  flight.  The device-to-device path the SMs add next to the copy
//                  engines (Sec. 4.3's horizontal split over paths).
//  k_sm_copy_vec8k the same loop with one vector per thread (8 KiB tiles), so that a
//                  message of a few MiB spreads over every SM instead of a few dozen.
//  k_zc_copy       zero-copy kernel: the vec128 loop with plain (coherent) loads, used on
//                  mapped page-locked host memory for host<->device transfers.
//  k_hash          digest of a byte range (test utility).
//
// The bulk-copy variant of the SM copy kernel (cp.async.bulk through shared memory) is in
// copy_bulk.cu.
#include "kernels.cuh"
#include "bulk_config.h"
#include "copy_device.cuh"

#include <algorithm>

namespace mpt {

namespace {

// Before waiting on the kernel ahead (programmatic dependent launch), one thread asks L2 for
// the source bytes of the CTA's first tile.  This is only a hint to L2, the GPU's point of
// coherence: if the kernel ahead writes those bytes before the wait returns, its stores
// update the lines in L2, and the loads after the wait, which miss L1, read the new bytes.
// No data reaches registers before the wait.  The short messages of a stream of copies then
// find their source in L2 instead of HBM once the kernel ahead completes.
template <int kU>
__device__ __forceinline__ void prefetch_first_tile(const CopyArgs& a) {
  if (threadIdx.x != 0 || blockIdx.x >= a.ntiles) return;
  constexpr uint64_t kTileBytes = (uint64_t)kVecThreads * kU * 16;
  const int r = find_range(a, blockIdx.x);
  const RangeDesc& d = a.r[r];
  const uint64_t lt = blockIdx.x - a.tile_start[r];
  // bytes of the range this tile reads: from the range start (tile 0 also copies the head)
  // or one word before the tile (the shifted path reads a word pair), to one word past it
  const uint64_t lo = lt == 0 ? 0 : d.head + lt * kTileBytes - 16;
  const uint64_t end = d.head + (lt + 1) * kTileBytes + 16;
  const uint64_t hi = end < d.bytes ? end : d.bytes;
  if (hi <= lo) return;
  // whole 16-byte blocks around [lo, hi): each holds a source byte, so it is mapped memory
  const uintptr_t base = reinterpret_cast<uintptr_t>(a.src + d.src_off);
  const uintptr_t p0 = (base + lo) & ~(uintptr_t)15, p1 = (base + hi + 15) & ~(uintptr_t)15;
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p0), "r"((uint32_t)(p1 - p0)) : "memory");
}

// kU 16-byte vectors per thread per tile: tiles of kVecThreads * kU * 16 bytes (64 KiB for
// kU = 8, 8 KiB for kU = 1).
template <bool kCoherent, bool kAny, int kU>
__device__ __forceinline__ void copy_tiles_vec(const CopyArgs& a) {
  constexpr uint64_t kTileVecs = (uint64_t)kVecThreads * kU;
  constexpr int kHalf = kU >= 2 ? kU / 2 : 1;  // shifted path: vector pairs per round
  const uint32_t tid = threadIdx.x;
  for (uint32_t t = blockIdx.x; t < a.ntiles; t += gridDim.x) {
    const int r = find_range(a, t);
    const uint32_t lt = t - a.tile_start[r];
    const RangeDesc d = a.r[r];
    const uint8_t* s = a.src + d.src_off;
    uint8_t* o = a.dst + d.dst_off;
    const uint64_t nvec = (d.bytes - d.head) >> 4;
    if (lt == 0) copy_edges(s, o, d, nvec << 4);
    uint4* ov = reinterpret_cast<uint4*>(o + d.head);
    const uint64_t v0 = (uint64_t)lt * kTileVecs + tid;
    if (!kAny || d.shift == 0) {
      const uint4* sv = reinterpret_cast<const uint4*>(s + d.head);
      uint4 buf[kU];
#pragma unroll
      for (int u = 0; u < kU; ++u) {
        const uint64_t i = v0 + (uint64_t)u * kVecThreads;
        if (i < nvec) buf[u] = kCoherent ? ld_plain(sv + i) : ld_stream(sv + i);
      }
#pragma unroll
      for (int u = 0; u < kU; ++u) {
        const uint64_t i = v0 + (uint64_t)u * kVecThreads;
        if (i < nvec) st_plain(ov + i, buf[u]);
      }
    } else {
      // source and destination differ modulo 16: two aligned source words per output word
      const uint4* sw = reinterpret_cast<const uint4*>(s + d.head - d.shift);
      const uint32_t k = d.shift >> 2, r = (d.shift & 3u) * 8u;
#pragma unroll
      for (int half = 0; half < kU; half += kHalf) {
        uint4 w0[kHalf], w1[kHalf];
#pragma unroll
        for (int u = 0; u < kHalf; ++u) {
          const uint64_t i = v0 + (uint64_t)(half + u) * kVecThreads;
          if (i < nvec) {
            w0[u] = kCoherent ? ld_plain(sw + i) : ld_stream(sw + i);
            w1[u] = kCoherent ? ld_plain(sw + i + 1) : ld_stream(sw + i + 1);
          }
        }
#pragma unroll
        for (int u = 0; u < kHalf; ++u) {
          const uint64_t i = v0 + (uint64_t)(half + u) * kVecThreads;
          if (i < nvec) st_plain(ov + i, shift16(w0[u], w1[u], k, r));
        }
      }
    }
  }
}

}  // namespace

__global__ void __launch_bounds__(kVecThreads) k_sm_copy_vec(CopyArgs a) {
  prefetch_first_tile<kVecUnroll>(a);
  pdl_enter();
  copy_tiles_vec<false, false, kVecUnroll>(a);
}
__global__ void __launch_bounds__(kVecThreads) k_sm_copy_vec_any(CopyArgs a) {
  prefetch_first_tile<kVecUnroll>(a);
  pdl_enter();
  copy_tiles_vec<false, true, kVecUnroll>(a);
}
__global__ void __launch_bounds__(kVecThreads) k_sm_copy_vec8k(CopyArgs a) {
  prefetch_first_tile<1>(a);
  pdl_enter();
  copy_tiles_vec<false, false, 1>(a);
}
__global__ void __launch_bounds__(kVecThreads) k_sm_copy_vec8k_any(CopyArgs a) {
  prefetch_first_tile<1>(a);
  pdl_enter();
  copy_tiles_vec<false, true, 1>(a);
}
__global__ void __launch_bounds__(kVecThreads) k_zc_copy(CopyArgs a) {
  pdl_enter();
  copy_tiles_vec<true, false, kVecUnroll>(a);
}
__global__ void __launch_bounds__(kVecThreads) k_zc_copy_any(CopyArgs a) {
  pdl_enter();
  copy_tiles_vec<true, true, kVecUnroll>(a);
}

namespace {
__device__ __forceinline__ uint64_t mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}
}  // namespace

__global__ void __launch_bounds__(256) k_hash(const uint8_t* p, uint64_t n, unsigned long long* out) {
  constexpr uint64_t kGamma = 0x9E3779B97F4A7C15ull;
  const uint64_t nw = (n + 7) >> 3;
  const bool aligned = (reinterpret_cast<uintptr_t>(p) & 7) == 0;
  uint64_t acc = 0;
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t w = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; w < nw; w += stride) {
    uint64_t v = 0;
    if (aligned && (w + 1) * 8 <= n) {
      v = __ldcs(reinterpret_cast<const unsigned long long*>(p) + w);
    } else {
      for (int b = 0; b < 8; ++b) {
        const uint64_t i = w * 8 + b;
        if (i < n) v |= (uint64_t)p[i] << (8 * b);
      }
    }
    acc += mix64(v ^ (w * kGamma));
  }
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  __shared__ uint64_t warp_sum[8];
  if ((threadIdx.x & 31) == 0) warp_sum[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    uint64_t s = 0;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) s += warp_sum[i];
    if (blockIdx.x == 0) s += mix64(n);
    atomicAdd(out, (unsigned long long)s);
  }
}

// ---- host side -------------------------------------------------------------------------

int make_copy_args(CopyArgs& a, const void* src, void* dst, const RangeDesc* ranges, int n,
                   int variant, uint32_t* status, uint32_t bulk_cfg) {
  a.src = static_cast<const uint8_t*>(src);
  a.dst = static_cast<uint8_t*>(dst);
  a.status = status;
  a.bulk_cfg = variant == 1 ? bulk_cfg : 0;
  a.piece = variant == 1 ? bulk_config(bulk_cfg).stage_bytes : 0;
  a.nranges = 0;
  a.any_shift = 0;
  uint64_t tiles = 0;
  a.tile_start[0] = 0;
  for (int i = 0; i < n && i < kInlineRanges; ++i) {
    RangeDesc d = ranges[i];
    if (d.bytes == 0) continue;
    const uintptr_t s = reinterpret_cast<uintptr_t>(src) + d.src_off;
    const uintptr_t o = reinterpret_cast<uintptr_t>(dst) + d.dst_off;
    d.head = (uint32_t)std::min<uint64_t>(d.bytes, (16 - (o & 15)) & 15);
    d.shift = (uint32_t)((s + d.head) & 15);
    if (variant == 1 && d.shift) return kArgsNeedVec;
    if (d.shift) a.any_shift = 1;
    const uint64_t body = ((d.bytes - d.head) >> 4) << 4;
    const uint64_t tile_vecs = variant == 3 ? (uint64_t)kVecThreads : kVecTileVecs;
    uint64_t t = variant == 1 ? (body + a.piece - 1) / a.piece : ((body >> 4) + tile_vecs - 1) / tile_vecs;
    if (t == 0) t = 1;  // a range too short for a body still needs its edge bytes copied
    a.r[a.nranges] = d;
    tiles += t;
    a.tile_start[a.nranges + 1] = (uint32_t)tiles;
    a.nranges++;
  }
  for (uint32_t i = a.nranges + 1; i <= (uint32_t)kInlineRanges; ++i) a.tile_start[i] = (uint32_t)tiles;
  a.ntiles = (uint32_t)tiles;
  return tiles < (1ull << 31) ? kArgsOk : kArgsTooLarge;
}

}  // namespace mpt
