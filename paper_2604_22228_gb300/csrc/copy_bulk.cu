// SM copy kernel, bulk-copy variant, written for sm_103a: the device-to-device path the SMs add
// next to the copy engines (Sec. 4.3's horizontal split over paths), with the 16-byte-aligned
// body of each range moved by the tensor memory accelerator instead of by registers.
//
// A launch cuts its ranges into tiles of one stage each; CTA b takes tiles b, b + grid, ...
// through a ring of kStages shared-memory stages, two threads in two warps:
//   producer (thread 0)   for each tile, once its stage is free, one cp.async.bulk
//                         global->shared load (non-multicast), counted in by the stage's
//                         "full" mbarrier (complete_tx);
//   consumer (thread 32)  for each tile, once its stage is full, one cp.async.bulk
//                         shared->global store; when the store of the tile kKeep behind it has
//                         finished reading shared memory (wait_group.read), that tile's stage
//                         goes back to the producer through its "empty" mbarrier.
// Loads run up to kStages - kKeep tiles ahead of the stores and neither thread waits on the
// other's operations, only on stage state.  Bytes before and after each range's body go with
// plain loads and stores by the CTA that owns the range's first tile.
//
// Every wait is bounded by the global timer: a wait that runs out records MPT_ETIMEDOUT in the
// context's status word, raises the CTA's abort flag (the other thread stops too), and the
// consumer then lets loads still in flight land (again bounded) before the CTA's shared memory
// is released.
#include "mpt.h"
#include "kernels.cuh"
#include "bulk_config.h"
#include "copy_device.cuh"

namespace mpt {

namespace {

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ bool mbar_test(uint32_t bar, uint32_t parity) {
  uint32_t done;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(done)
      : "r"(bar), "r"(parity)
      : "memory");
  return done != 0;
}

// Wait for the phase of parity `parity` of a barrier to complete.  False when the deadline
// passes or (abort non-null) the CTA's abort flag is raised first.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, uint64_t deadline,
                                          const volatile uint32_t* abort) {
  while (!mbar_test(bar, parity)) {
    if (abort && *abort) return false;
    if (global_ns() > deadline) return false;
  }
  return true;
}

// kHint 1: both directions carry an L2 evict-first policy (each byte is touched once).
template <int kHint>
__device__ __forceinline__ void bulk_load(uint32_t dst_smem, const void* src, uint32_t bytes, uint32_t bar,
                                          uint64_t policy) {
  if (kHint) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1], %2, [%3], %4;" ::"r"(
            dst_smem),
        "l"(src), "r"(bytes), "r"(bar), "l"(policy)
        : "memory");
  } else {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     dst_smem),
                 "l"(src), "r"(bytes), "r"(bar)
                 : "memory");
  }
}

template <int kHint>
__device__ __forceinline__ void bulk_store(void* dst, uint32_t src_smem, uint32_t bytes, uint64_t policy) {
  if (kHint) {
    asm volatile("cp.async.bulk.global.shared::cta.bulk_group.L2::cache_hint [%0], [%1], %2, %3;" ::"l"(dst),
                 "r"(src_smem), "r"(bytes), "l"(policy)
                 : "memory");
  } else {
    asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(dst), "r"(src_smem), "r"(bytes)
                 : "memory");
  }
}

__device__ __forceinline__ uint64_t evict_first_policy() {
  uint64_t p;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
  return p;
}

__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }

template <int N>
__device__ __forceinline__ void bulk_wait_read() {
  asm volatile("cp.async.bulk.wait_group.read %0;" ::"n"(N) : "memory");
}

__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }

// Global addresses and length of the body piece of launch tile t (0 when the tile lies past
// its range's body: a range too short for a body still has one tile for its edges).
template <uint32_t kPiece>
__device__ __forceinline__ uint32_t body_piece(const CopyArgs& a, uint32_t t, const uint8_t*& gs, uint8_t*& gd) {
  const int r = find_range(a, t);
  const uint32_t lt = t - a.tile_start[r];
  const RangeDesc& d = a.r[r];
  const uint64_t body = ((d.bytes - d.head) >> 4) << 4;
  const uint64_t off = (uint64_t)lt * kPiece;
  gs = a.src + d.src_off + d.head + off;
  gd = a.dst + d.dst_off + d.head + off;
  if (off >= body) return 0;
  const uint64_t n = body - off;
  return n < kPiece ? (uint32_t)n : kPiece;
}

}  // namespace

template <int kStages, uint32_t kStageBytes, int kKeep, int kPerSm, int kHint>
__global__ void __launch_bounds__(kBulkThreads, kPerSm) k_sm_copy_bulk(CopyArgs a) {
  static_assert(kKeep >= 1 && kKeep < kStages, "stores kept reading must leave stages for loads");
  static_assert(kStageBytes % 1024 == 0, "stages stay 1 KiB aligned in shared memory");
  extern __shared__ __align__(1024) uint8_t smem[];
  __shared__ __align__(8) uint64_t full[kStages];
  __shared__ __align__(8) uint64_t empty[kStages];
  __shared__ uint32_t abort_flag, issued, consumed;
  const uint32_t tid = threadIdx.x;
  pdl_enter();
  if (a.piece != kStageBytes) {  // host and kernel disagree on the tiling: copy nothing
    if (tid == 0 && blockIdx.x == 0) record_invalid(a.status, kSiteBulkArgs);
    return;
  }

  // edges of every range whose first tile is this CTA's
  for (uint32_t t = blockIdx.x; t < a.ntiles; t += gridDim.x) {
    const int r = find_range(a, t);
    if (t != a.tile_start[r]) continue;
    const RangeDesc d = a.r[r];
    copy_edges(a.src + d.src_off, a.dst + d.dst_off, d, ((d.bytes - d.head) >> 4) << 4);
  }

  if (tid == 0) {
    for (int s = 0; s < kStages; ++s) {
      mbar_init(smem_addr(&full[s]), 1);
      mbar_init(smem_addr(&empty[s]), 1);
    }
    abort_flag = 0;
    issued = 0;
    consumed = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  __syncthreads();

  const uint32_t n_my = blockIdx.x < a.ntiles ? (a.ntiles - blockIdx.x + gridDim.x - 1) / gridDim.x : 0;
  const uint32_t base = smem_addr(smem);
  volatile uint32_t* abort_v = &abort_flag;
  const uint64_t deadline = global_ns() + kDefaultTimeoutNs;
  const uint64_t policy = kHint ? evict_first_policy() : 0;

  if (tid == 0) {  // producer
    for (uint32_t i = 0; i < n_my; ++i) {
      const uint32_t s = i % kStages;
      if (i >= (uint32_t)kStages && !mbar_wait(smem_addr(&empty[s]), ((i / kStages) - 1) & 1u, deadline, abort_v)) {
        if (!*abort_v) record_timeout(a.status, kSiteBulkLoad);
        *abort_v = 1;
        break;
      }
      const uint8_t* gs;
      uint8_t* gd;
      const uint32_t n = body_piece<kStageBytes>(a, blockIdx.x + i * gridDim.x, gs, gd);
      const uint32_t fb = smem_addr(&full[s]);
      if (n) {
        mbar_arrive_expect_tx(fb, n);
        bulk_load<kHint>(base + s * kStageBytes, gs, n, fb, policy);
      } else {
        mbar_arrive(fb);
      }
      *(volatile uint32_t*)&issued = i + 1;
    }
  } else if (tid == 32) {  // consumer
    uint32_t i = 0;
    for (; i < n_my; ++i) {
      const uint32_t s = i % kStages;
      if (!mbar_wait(smem_addr(&full[s]), (i / kStages) & 1u, deadline, abort_v)) {
        if (!*abort_v) record_timeout(a.status, kSiteBulkLoad);
        *abort_v = 1;
        break;
      }
      const uint8_t* gs;
      uint8_t* gd;
      const uint32_t n = body_piece<kStageBytes>(a, blockIdx.x + i * gridDim.x, gs, gd);
      if (n) bulk_store<kHint>(gd, base + s * kStageBytes, n, policy);
      bulk_commit();
      if (i >= (uint32_t)kKeep) {
        bulk_wait_read<kKeep>();  // the store of tile i - kKeep has read its stage
        mbar_arrive(smem_addr(&empty[(i - kKeep) % kStages]));
      }
    }
    *(volatile uint32_t*)&consumed = i;
    bulk_wait_all();
  }
  __syncthreads();
  if (tid == 32 && *abort_v) {
    // loads issued but never consumed still write this CTA's shared memory: let them land
    const uint64_t drain = global_ns() + kDefaultTimeoutNs;
    const uint32_t hi = *(volatile uint32_t*)&issued;
    for (uint32_t j = *(volatile uint32_t*)&consumed; j < hi; ++j)
      mbar_wait(smem_addr(&full[j % kStages]), (j / kStages) & 1u, drain, nullptr);
  }
}

namespace {

// The configurations compiled in.  On GB300 (CUDA events, back-to-back launches of one
// message, 32 CTAs per SM) configurations 0, 3 and 5 move 6.9-7.05 TB/s at 1-4 GiB; at
// 256 MiB configuration 3 keeps 6.74 TB/s where 0 falls to 5.1 (a tile or so per CTA, and
// one resident CTA per SM cannot hide a CTA's start).  Smaller and deeper rings (16 KiB and
// 12 KiB stages) measured 2-5 % slower in one wave and were dropped.
template <int S, uint32_t B, int K, int P, int H = 0>
BulkConfig cfg() {
  return BulkConfig{(uint32_t)S, B, (uint32_t)K, (uint32_t)P,
                    reinterpret_cast<const void*>(&k_sm_copy_bulk<S, B, K, P, H>)};
}

const BulkConfig kConfigs[] = {
    cfg<4, 48 * 1024, 1, 1>(),     // 0: 192 KiB, four 48 KiB stages
    cfg<4, 48 * 1024, 1, 1, 1>(),  // 1: as 0, L2 evict-first on loads and stores
    cfg<3, 64 * 1024, 1, 1>(),     // 2: 192 KiB, three 64 KiB stages
    cfg<2, 48 * 1024, 1, 2>(),     // 3: 2 x 96 KiB, two 48 KiB stages each (default)
    cfg<2, 48 * 1024, 1, 2, 1>(),  // 4: as 3, L2 evict-first
    cfg<3, 32 * 1024, 1, 2>(),     // 5: 2 x 96 KiB, three 32 KiB stages each
    cfg<8, 24 * 1024, 2, 1>(),     // 6: 192 KiB, eight 24 KiB stages, two stores reading
};

}  // namespace

static_assert(sizeof kConfigs / sizeof kConfigs[0] == MPT_BULK_CONFIGS, "mpt.h lists every configuration");

uint32_t bulk_config_count() { return (uint32_t)(sizeof kConfigs / sizeof kConfigs[0]); }

const BulkConfig& bulk_config(uint32_t i) { return kConfigs[i < bulk_config_count() ? i : kBulkDefaultConfig]; }

}  // namespace mpt
