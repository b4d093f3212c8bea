// Device-side copy helpers shared by the copy kernels: 128-bit loads and stores, and the
// assembly of a destination-aligned 16-byte word from two aligned source words when source
// and destination differ modulo 16 (so no path ever falls back to byte-by-byte copies).
#pragma once
#include <cstdint>

namespace mpt {

// Programmatic dependent launch.  A copy kernel launched with programmatic stream
// serialization may start while the kernel before it on the stream is finishing; it waits
// here, before touching memory, until that kernel has completed and its writes are visible,
// then lets the next such kernel begin its own launch.  Launched without the attribute
// (graph nodes, plain launches) both instructions are no-ops.
__device__ __forceinline__ void pdl_enter() {
  asm volatile("griddepcontrol.wait;" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// Global timer in nanoseconds: the clock every bounded device-side wait measures against.
__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// A wait ran out: record (site << 8) | MPT_ETIMEDOUT in the context's status word, unless
// an earlier failure is already recorded there.
__device__ __forceinline__ void record_timeout(uint32_t* status, uint32_t site) {
  constexpr uint32_t kTimedOut = 4;  // MPT_ETIMEDOUT
  if (status) atomicCAS(status, 0u, (site << 8) | kTimedOut);
}

// A kernel refused its arguments: record (site << 8) | MPT_EINVAL the same way.
__device__ __forceinline__ void record_invalid(uint32_t* status, uint32_t site) {
  constexpr uint32_t kInvalid = 1;  // MPT_EINVAL
  if (status) atomicCAS(status, 0u, (site << 8) | kInvalid);
}

// Read-only path (ld.global.nc): only for data no agent writes while the kernel runs.
__device__ __forceinline__ uint4 ld_stream(const uint4* p) {
  uint4 v;
  asm volatile("ld.global.nc.L1::no_allocate.v4.u32 {%0,%1,%2,%3}, [%4];"
               : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
               : "l"(p));
  return v;
}

__device__ __forceinline__ uint4 ld_plain(const uint4* p) {
  uint4 v;
  asm volatile("ld.global.v4.u32 {%0,%1,%2,%3}, [%4];" : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w) : "l"(p));
  return v;
}

__device__ __forceinline__ void st_plain(uint4* p, const uint4& v) {
  asm volatile("st.global.v4.u32 [%0], {%1,%2,%3,%4};" ::"l"(p), "r"(v.x), "r"(v.y), "r"(v.z), "r"(v.w)
               : "memory");
}

// Index of the range that launch tile t belongs to (ranges are few: a linear scan).
template <typename Args>
__device__ __forceinline__ int find_range(const Args& a, uint32_t t) {
  int r = 0;
  while (r + 1 < (int)a.nranges && t >= a.tile_start[r + 1]) ++r;
  return r;
}

// Head (bytes before the destination-aligned body) and tail (bytes after it) of a range;
// threads 0..15 copy the head, threads 32..47 the tail (blocks of at least 48 threads).
template <typename Range>
__device__ __forceinline__ void copy_edges(const uint8_t* s, uint8_t* o, const Range& d, uint64_t body_bytes) {
  const uint32_t tid = threadIdx.x;
  if (tid < d.head) o[tid] = s[tid];
  const uint64_t tail_start = d.head + body_bytes;
  const uint32_t tail = (uint32_t)(d.bytes - tail_start);
  if (tid >= 32 && tid < 32 + tail) o[tail_start + (tid - 32)] = s[tail_start + (tid - 32)];
}

// Bytes [4k + r/8, 4k + r/8 + 16) of the 32-byte little-endian concatenation w0 | w1
// (k in 0..3 words, r in {0, 8, 16, 24} bits): each output word is a funnel shift of two
// neighbouring input words.
__device__ __forceinline__ uint4 shift16(const uint4& w0, const uint4& w1, uint32_t k, uint32_t r) {
  const uint32_t a[8] = {w0.x, w0.y, w0.z, w0.w, w1.x, w1.y, w1.z, w1.w};
  uint4 o;
  switch (k) {
    case 0:
      o = make_uint4(__funnelshift_r(a[0], a[1], r), __funnelshift_r(a[1], a[2], r), __funnelshift_r(a[2], a[3], r),
                     __funnelshift_r(a[3], a[4], r));
      break;
    case 1:
      o = make_uint4(__funnelshift_r(a[1], a[2], r), __funnelshift_r(a[2], a[3], r), __funnelshift_r(a[3], a[4], r),
                     __funnelshift_r(a[4], a[5], r));
      break;
    case 2:
      o = make_uint4(__funnelshift_r(a[2], a[3], r), __funnelshift_r(a[3], a[4], r), __funnelshift_r(a[4], a[5], r),
                     __funnelshift_r(a[5], a[6], r));
      break;
    default:
      o = make_uint4(__funnelshift_r(a[3], a[4], r), __funnelshift_r(a[4], a[5], r), __funnelshift_r(a[5], a[6], r),
                     __funnelshift_r(a[6], a[7], r));
      break;
  }
  return o;
}

// The whole CTA copies n bytes s -> o: bytes until o is 16-byte aligned, 16-byte words
// (straight when s is then aligned too, else -- only if kAny -- assembled from two aligned
// source words), and the remaining tail bytes.  Reads never leave the 16-byte blocks that
// hold source bytes.  Without kAny the caller guarantees s and o agree modulo 16.
template <bool kCoherent, bool kAny>
__device__ __forceinline__ void cta_copy(const uint8_t* s, uint8_t* o, uint64_t n) {
  const uint32_t tid = threadIdx.x, bd = blockDim.x;
  const uint64_t head = ((16u - (uint32_t)(reinterpret_cast<uintptr_t>(o) & 15)) & 15u) < n
                            ? ((16u - (uint32_t)(reinterpret_cast<uintptr_t>(o) & 15)) & 15u)
                            : n;
  if (tid < head) o[tid] = s[tid];
  const uint8_t* s1 = s + head;
  uint8_t* o1 = o + head;
  const uint64_t n1 = n - head;
  const uint64_t nv = n1 >> 4;
  uint4* ov = reinterpret_cast<uint4*>(o1);
  const uint32_t m = kAny ? (uint32_t)(reinterpret_cast<uintptr_t>(s1) & 15) : 0u;
  uint64_t v = tid;
  if (m == 0) {
    const uint4* sv = reinterpret_cast<const uint4*>(s1);
    for (; v + 3ull * bd < nv; v += 4ull * bd) {
      uint4 r0, r1, r2, r3;
      if (kCoherent) {
        r0 = ld_plain(sv + v); r1 = ld_plain(sv + v + bd); r2 = ld_plain(sv + v + 2 * bd); r3 = ld_plain(sv + v + 3 * bd);
      } else {
        r0 = ld_stream(sv + v); r1 = ld_stream(sv + v + bd); r2 = ld_stream(sv + v + 2 * bd); r3 = ld_stream(sv + v + 3 * bd);
      }
      st_plain(ov + v, r0);
      st_plain(ov + v + bd, r1);
      st_plain(ov + v + 2 * bd, r2);
      st_plain(ov + v + 3 * bd, r3);
    }
    for (; v < nv; v += bd) st_plain(ov + v, kCoherent ? ld_plain(sv + v) : ld_stream(sv + v));
  } else {
    const uint4* sw = reinterpret_cast<const uint4*>(s1 - m);
    const uint32_t k = m >> 2, r = (m & 3u) * 8u;
#pragma unroll 2
    for (; v < nv; v += bd) {
      const uint4 a0 = kCoherent ? ld_plain(sw + v) : ld_stream(sw + v);
      const uint4 a1 = kCoherent ? ld_plain(sw + v + 1) : ld_stream(sw + v + 1);
      st_plain(ov + v, shift16(a0, a1, k, r));
    }
  }
  for (uint64_t b = (nv << 4) + tid; b < n1; b += bd) o1[b] = s1[b];
}

}  // namespace mpt
