// Batched transfers: one persistent kernel walks a device-resident descriptor table and
// moves many messages of uneven sizes in one launch, replayed as a CUDA graph.
//
// The paper's windowed benchmarks keep several messages in flight at once and find that
// graphs pay off when many operations share one launch (Sec. 5.3, windows 1/4/16; Sec. 6).
// Here a batch is a table of (src, dst, bytes) descriptors; the kernel's CTAs claim fixed
// size tiles of the whole batch through one atomic cursor, so short and long messages,
// device-to-device and host<->device ones, share the SMs without per-message launches.
// A per-descriptor tile counter detects the last tile of a message; that CTA stamps the
// completion time and raises the message's flag in page-locked host memory, which is how
// a host thread (the serving loop) sees individual messages finish while the batch runs.
//
// Each context owns a ring of batch slots.  A slot holds the page-locked and device copies
// of its table, its counters and flags, and one instantiated graph
//   [table host->device copy] -> [batch kernel]
// The descriptor count lives in the table header, so any batch up to the slot capacity
// replays the same graph; only the copy's size follows the batch (the table is packed, so
// a short batch copies a few hundred bytes).  The kernel leaves its counters at zero when
// it ends, so no reset node runs between replays: a one-request batch costs one small copy
// and one kernel.
#include <algorithm>
#include <iterator>
#include <chrono>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <thread>

#include "copy_device.cuh"
#include "ctx.h"

#define CUDA_TRY(expr)                                                                           \
  do {                                                                                           \
    cudaError_t e_ = (expr);                                                                     \
    if (e_ != cudaSuccess)                                                                       \
      return mpt::fail(MPT_ECUDA, "%s: %s (%s:%d)", #expr, cudaGetErrorString(e_), __FILE__, __LINE__); \
  } while (0)

namespace mpt {

namespace {

__device__ __forceinline__ uint64_t now_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

}  // namespace

template <bool kAny>
__device__ __forceinline__ void batch_body(const BatchArgs& a) {
  __shared__ uint32_t s_item;
  const BatchHeader h = *a.hdr;
  const uint32_t* order = reinterpret_cast<const uint32_t*>(a.desc + h.n);
  if (threadIdx.x == 0) {
    const uint64_t t = now_ns();
    atomicMax(a.start_inv, ~t);
    // when the first and the last CTA of the grid started: a spread far above the launch
    // time means the grid was only partly resident (other kernels held the SMs)
    const uint32_t k = atomicAdd(a.started, 1u);
    if (k == 0) a.host_stamps[0] = t;
    if (k == gridDim.x - 1) a.host_stamps[1] = t;
  }
  __shared__ uint32_t s_link;
  const uint32_t dev_tiles = h.total_tiles - h.link_tiles;
  // thread 0's claiming state: the class it claims from, and whether it has switched yet.
  // CTAs [0, link_ctas) take link tiles first, then device tiles; the others take device
  // tiles only.  That bounds the host-link reads and writes this launch keeps in flight,
  // and with them the queue that every other user of the link (another batch's table copy,
  // its completion flags, its host-side bytes) waits behind.
  const bool may_link = blockIdx.x < h.link_ctas;
  bool on_link = may_link && h.link_tiles > 0;
  bool switched = !may_link;
  while (true) {
    if (threadIdx.x == 0) {
      uint32_t item = ~0u;
      while (true) {
        const uint32_t lim = on_link ? h.link_tiles : dev_tiles;
        if (lim) {
          const uint32_t k = atomicAdd(on_link ? a.cursor : a.cursor_dev, 1u);
          if (k < lim) {
            item = k;
            break;
          }
        }
        if (switched) break;
        switched = true;
        on_link = !on_link;
      }
      s_item = item;
      s_link = on_link ? 1u : 0u;
    }
    __syncthreads();
    const uint32_t item = s_item;
    const bool link = s_link != 0;
    __syncthreads();
    if (item == ~0u) break;
    // descriptor owning this tile: within its class, the last one whose first tile is <= item
    uint32_t lo = link ? 0 : h.n_link, hi = (link ? h.n_link : h.n_tiled) - 1;
    while (lo < hi) {
      const uint32_t mid = (lo + hi + 1) >> 1;
      if (a.desc[order[mid]].first_tile <= item) lo = mid;
      else hi = mid - 1;
    }
    lo = order[lo];
    const BatchDesc d = a.desc[lo];
    const uint64_t off = (uint64_t)(item - d.first_tile) * h.tile_bytes;
    if (off < d.bytes) {
      const uint64_t len = d.bytes - off < h.tile_bytes ? d.bytes - off : h.tile_bytes;
      const uint8_t* src = reinterpret_cast<const uint8_t*>(d.src) + off;
      uint8_t* dst = reinterpret_cast<uint8_t*>(d.dst) + off;
      // coherent loads for every descriptor: one copy loop keeps the kernel at 40
      // registers (three 512-thread CTAs per SM); host-memory sources need them anyway
      cta_copy<true, kAny>(src, dst, len);
    }
    if (d.flags & kDescHostDst) __threadfence_system();
    else __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
      const uint32_t prev = atomicAdd(a.done + lo, 1u);
      if (prev + 1 == d.ntiles) {
        a.times[lo] = now_ns();
        // the release store's system-scope fence orders the tiles counted through `done`
        // (each published by its CTA's fence before the count) ahead of the flag
        asm volatile("st.release.sys.global.u32 [%0], %1;" ::"l"(a.host_flags + lo), "r"(h.epoch) : "memory");
        a.done[lo] = 0;  // every tile of lo is counted: no CTA of this launch touches it again
      }
    }
  }
  if (threadIdx.x == 0) {
    __threadfence();
    // the last CTA out: every CTA has stopped claiming, so the cursors and the start
    // counters can go back to zero for the slot's next launch
    if (atomicAdd(a.exited, 1u) == gridDim.x - 1) {
      *a.start_out = atomicExch(a.start_inv, 0ull);
      *a.cursor = 0;
      *a.cursor_dev = 0;
      *a.started = 0;
      __threadfence();
      *a.exited = 0;
    }
  }
}

__global__ void k_batch_dma_done(BatchArgs a, const uint32_t* dma_map, uint32_t item) {
  if (threadIdx.x != 0) return;
  const uint32_t idx = dma_map[item];
  if (idx == ~0u) return;
  a.times[idx] = now_ns();
  // the lane's copy finished before this kernel began (graph edge); the release store
  // publishes the flag after it
  asm volatile("st.release.sys.global.u32 [%0], %1;" ::"l"(a.host_flags + idx), "r"(a.hdr->epoch) : "memory");
}

__global__ void __launch_bounds__(kVecThreads, 3) k_batch(BatchArgs a) { batch_body<false>(a); }
__global__ void __launch_bounds__(kVecThreads) k_batch_any(BatchArgs a) { batch_body<true>(a); }

namespace {

constexpr uint32_t kDefaultSlots = 4;
constexpr uint32_t kDefaultMaxXfers = 4096;
constexpr uint32_t kDefaultTile = 256 * 1024;
constexpr uint64_t kMinAdaptiveTile = 32 * 1024;  // smallest tile a short batch is cut into
// CTAs of a launch that may take link tiles (MPT_BATCH_LINK_CTAS overrides).  32 CTAs keep
// 1 MiB of host-link traffic in flight, about 5 us of the link: enough to hold it at its
// rate (host-to-device 204 GB/s, device-to-host 176 GB/s, as with every CTA), while a longer
// queue only delays whatever else crosses the link
constexpr uint32_t kDefaultLinkCtas = 32;
constexpr uint32_t kDmaDirs = 3;  // lanes per direction: D2D, H2D, D2H

uint64_t host_ns() {
  return (uint64_t)std::chrono::duration_cast<std::chrono::nanoseconds>(
             std::chrono::steady_clock::now().time_since_epoch())
      .count();
}

void slot_free(BatchSlot& s) {
  for (int i = 0; i < 2; ++i) {
    if (s.exec[i]) cudaGraphExecDestroy(s.exec[i]);
    if (s.graph[i]) cudaGraphDestroy(s.graph[i]);
  }
  if (s.done_ev) cudaEventDestroy(s.done_ev);
  if (s.t0_ev) cudaEventDestroy(s.t0_ev);
  if (s.t1_ev) cudaEventDestroy(s.t1_ev);
  if (s.h_scratch) cudaFreeHost(s.h_scratch);
  if (s.h_table) cudaFreeHost(s.h_table);
  if (s.h_flags) cudaFreeHost(s.h_flags);
  if (s.h_stamps) cudaFreeHost(s.h_stamps);
  if (s.d_mem) cudaFree(s.d_mem);
  s = BatchSlot{};
}

mpt_status slot_init(mpt_ctx_t c, BatchSlot& s, uint32_t max_xfers, uint32_t ctas) {
  s.max_xfers = max_xfers;
  s.dma_lanes = c->batch_dma_lanes;
  s.dma_items = c->batch_dma_lanes ? c->batch_dma_items : 0;
  const uint32_t ndma = kDmaDirs * s.dma_lanes * s.dma_items;
  // table: header | lane map[ndma] | desc[n] | order[n] (BatchArgs): a batch copies its first
  // desc_off + n * 44 bytes
  const size_t map_off = sizeof(BatchHeader);
  s.desc_off = (map_off + (size_t)ndma * sizeof(uint32_t) + 15) & ~(size_t)15;
  s.table_bytes = s.desc_off + (size_t)max_xfers * (sizeof(BatchDesc) + sizeof(uint32_t));
  CUDA_TRY(cudaHostAlloc(&s.h_table, s.table_bytes, cudaHostAllocPortable));
  CUDA_TRY(cudaHostAlloc(reinterpret_cast<void**>(&s.h_flags), (size_t)max_xfers * sizeof(uint32_t),
                         cudaHostAllocMapped | cudaHostAllocPortable));
  std::memset(s.h_flags, 0, (size_t)max_xfers * sizeof(uint32_t));
  // device block: table | ctrl (cursors, start, counters) | done[max] | times[max]; zeroed
  // here once, kept zero between launches by the kernel
  const size_t ctrl_off = (s.table_bytes + 255) & ~(size_t)255;
  s.ctrl_bytes = 256 + (size_t)max_xfers * sizeof(uint32_t);
  const size_t times_off = (ctrl_off + s.ctrl_bytes + 255) & ~(size_t)255;
  const size_t scratch_off = (times_off + (size_t)max_xfers * sizeof(uint64_t) + 255) & ~(size_t)255;
  CUDA_TRY(cudaMalloc(&s.d_mem, scratch_off + 256));
  uint8_t* base = static_cast<uint8_t*>(s.d_mem);
  s.d_table = base;
  s.d_ctrl = base + ctrl_off;
  s.d_times = reinterpret_cast<unsigned long long*>(base + times_off);
  CUDA_TRY(cudaMemset(s.d_mem, 0, scratch_off + 256));
  s.h_dma_map = reinterpret_cast<uint32_t*>(s.h_table + map_off);
  for (uint32_t k = 0; k < ndma; ++k) s.h_dma_map[k] = ~0u;
  if (ndma) CUDA_TRY(cudaHostAlloc(&s.h_scratch, 64, cudaHostAllocPortable));
  uint8_t* d_scratch = base + scratch_off;
  const uint32_t* d_map = reinterpret_cast<const uint32_t*>(s.d_table + map_off);
  CUDA_TRY(cudaEventCreateWithFlags(&s.done_ev, cudaEventDisableTiming));
  s.args.hdr = reinterpret_cast<const BatchHeader*>(s.d_table);
  s.args.desc = reinterpret_cast<const BatchDesc*>(s.d_table + s.desc_off);
  s.args.cursor = reinterpret_cast<uint32_t*>(s.d_ctrl);
  s.args.cursor_dev = reinterpret_cast<uint32_t*>(s.d_ctrl + 24);
  s.args.start_inv = reinterpret_cast<unsigned long long*>(s.d_ctrl + 8);
  s.args.start_out = reinterpret_cast<unsigned long long*>(s.d_ctrl + 32);
  s.args.done = reinterpret_cast<uint32_t*>(s.d_ctrl + 256);
  s.args.started = reinterpret_cast<uint32_t*>(s.d_ctrl + 16);
  s.args.exited = reinterpret_cast<uint32_t*>(s.d_ctrl + 20);
  CUDA_TRY(cudaHostAlloc(reinterpret_cast<void**>(&s.h_stamps), 2 * sizeof(unsigned long long),
                         cudaHostAllocMapped | cudaHostAllocPortable));
  s.h_stamps[0] = s.h_stamps[1] = 0;
  CUDA_TRY(cudaHostGetDevicePointer(reinterpret_cast<void**>(&s.args.host_stamps), s.h_stamps, 0));
  s.args.times = s.d_times;
  uint32_t* hf_dev = nullptr;
  CUDA_TRY(cudaHostGetDevicePointer(reinterpret_cast<void**>(&hf_dev), s.h_flags, 0));
  s.args.host_flags = hf_dev;
  // graphs: the table copy, then the kernel (aligned-only or any alignment); the copy's size
  // follows the batch (mpt_batch_submit)
  for (int gi = 0; gi < 2; ++gi) {
    CUDA_TRY(cudaGraphCreate(&s.graph[gi], 0));
    cudaGraphNode_t cp, kn;
    CUDA_TRY(cudaGraphAddMemcpyNode1D(&cp, s.graph[gi], nullptr, 0, s.d_table, s.h_table, s.table_bytes,
                                      cudaMemcpyHostToDevice));
    s.table_cp[gi] = cp;
    s.table_cp_bytes[gi] = s.table_bytes;
    cudaGraphNode_t deps[1] = {cp};
    void* params[] = {&s.args};
    cudaKernelNodeParams kp{};
    kp.func = gi == 0 ? reinterpret_cast<void*>(&k_batch) : reinterpret_cast<void*>(&k_batch_any);
    // the general kernel holds two CTAs per SM (64 registers): keep all of them resident
    kp.gridDim = dim3(gi == 0 ? ctas : std::min<uint32_t>(ctas, 2u * (uint32_t)c->sms));
    kp.blockDim = dim3(kVecThreads);
    kp.kernelParams = params;
    CUDA_TRY(cudaGraphAddKernelNode(&kn, s.graph[gi], deps, 1, &kp));
    // DMA lanes beside the kernel: per direction, chains of memcpy -> completion kernel.
    // Instantiation-time operands are scratch buffers of the lane's memory kinds (a
    // retargeted memcpy node keeps the kinds it was built with).
    s.dma_cp[gi].assign(ndma, nullptr);
    s.dma_fin[gi].assign(ndma, nullptr);
    for (uint32_t dir = 0; dir < kDmaDirs; ++dir) {
      void* to = dir == MPT_D2H ? s.h_scratch : static_cast<void*>(d_scratch);
      const void* from = dir == MPT_H2D ? s.h_scratch : static_cast<const void*>(d_scratch + 128);
      for (uint32_t l = 0; l < s.dma_lanes; ++l) {
        cudaGraphNode_t prev = nullptr;
        for (uint32_t j = 0; j < s.dma_items; ++j) {
          const uint32_t item = (dir * s.dma_lanes + l) * s.dma_items + j;
          cudaGraphNode_t cn, fn;
          if (prev) {
            CUDA_TRY(cudaGraphAddMemcpyNode1D(&cn, s.graph[gi], &prev, 1, to, from, 16, cudaMemcpyDefault));
          } else {
            CUDA_TRY(cudaGraphAddMemcpyNode1D(&cn, s.graph[gi], deps, 1, to, from, 16, cudaMemcpyDefault));
          }
          uint32_t it = item;
          void* fparams[] = {&s.args, const_cast<uint32_t**>(&d_map), &it};
          cudaKernelNodeParams fp{};
          fp.func = reinterpret_cast<void*>(&k_batch_dma_done);
          fp.gridDim = dim3(1);
          fp.blockDim = dim3(32);
          fp.kernelParams = fparams;
          CUDA_TRY(cudaGraphAddKernelNode(&fn, s.graph[gi], &cn, 1, &fp));
          s.dma_cp[gi][item] = cn;
          s.dma_fin[gi][item] = fn;
          prev = fn;
        }
      }
    }
    CUDA_TRY(cudaGraphInstantiate(&s.exec[gi], s.graph[gi], 0));
    for (uint32_t k = 0; k < ndma; ++k) {  // every lane item starts disabled
      CUDA_TRY(cudaGraphNodeSetEnabled(s.exec[gi], s.dma_cp[gi][k], 0));
      CUDA_TRY(cudaGraphNodeSetEnabled(s.exec[gi], s.dma_fin[gi][k], 0));
    }
    s.dma_on[gi].assign(ndma, 0);
  }
  return MPT_OK;
}

// Classify [p, p+n) against registered arenas (fast path) or the CUDA runtime.
int range_kind(mpt_ctx_t c, const void* p, uint64_t n) {
  const uint64_t a = (uint64_t)(uintptr_t)p;
  for (const Arena& r : c->arenas)
    if (a >= r.base && a + n <= r.base + r.bytes && a + n >= a) return r.kind;
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return -1;
  }
  if ((at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged) && at.device == c->device) return 0;
  if (at.type == cudaMemoryTypeHost) return 1;
  // pageable host memory: the batch kernel reads and writes it directly when the GPU can
  // (a copy-engine graph node cannot: such entries stay with the kernel)
  if (at.type == cudaMemoryTypeUnregistered && c->pageable) return 2;
  return -1;
}

uint64_t env_or(const char* name, uint64_t dflt) {
  const char* v = std::getenv(name);
  if (!v || !*v) return dflt;
  char* end = nullptr;
  const unsigned long long x = std::strtoull(v, &end, 0);
  return (end && *end == 0) ? (uint64_t)x : dflt;
}

}  // namespace

mpt_status batch_setup(mpt_ctx_t c) {
  if (!c->slots.empty()) return MPT_OK;
  const uint32_t nslots = c->batch_slots ? c->batch_slots
                                         : (uint32_t)std::max<uint64_t>(1, std::min<uint64_t>(64, env_or("MPT_BATCH_SLOTS", kDefaultSlots)));
  const uint32_t maxx = c->batch_max_xfers ? c->batch_max_xfers : kDefaultMaxXfers;
  // three 512-thread CTAs per SM (the aligned kernel's register limit): high occupancy,
  // which the latency of host-link reads needs; all CTAs resident at once
  const uint32_t ctas = c->batch_ctas ? c->batch_ctas : 3u * (uint32_t)c->sms;
  if (!c->batch_tile) c->batch_tile = kDefaultTile;
  c->batch_split = env_or("MPT_BATCH_SPLIT", 1) != 0;
  c->batch_link_ctas = (uint32_t)env_or("MPT_BATCH_LINK_CTAS", 0);
  if (!c->batch_dma_set) {
    c->batch_dma_lanes = (uint32_t)std::min<uint64_t>(8, env_or("MPT_BATCH_DMA_LANES", 0));
    c->batch_dma_items = (uint32_t)std::max<uint64_t>(1, std::min<uint64_t>(64, env_or("MPT_BATCH_DMA_ITEMS", 8)));
    c->batch_dma_min = std::max<uint64_t>(16, env_or("MPT_BATCH_DMA_MIN", 4ull << 20));
  }
  c->slots.resize(nslots);
  for (auto& s : c->slots) {
    mpt_status st = slot_init(c, s, maxx, ctas);
    if (st != MPT_OK) {
      for (auto& t : c->slots) slot_free(t);
      c->slots.clear();
      return st;
    }
  }
  return MPT_OK;
}

void batch_teardown(mpt_ctx_t c) {
  for (auto& s : c->slots) slot_free(s);
  c->slots.clear();
  for (cudaEvent_t e : c->each_ev) cudaEventDestroy(e);
  c->each_ev.clear();
}

mpt_status batch_check_xfer(mpt_ctx_t c, const mpt_xfer& x, int* src_kind, int* dst_kind) {
  *src_kind = *dst_kind = -1;
  if (x.dir > MPT_D2H) return fail(MPT_EINVAL, "transfer has direction %u", x.dir);
  if (x.bytes == 0) return MPT_OK;
  if (!x.src || !x.dst) return fail(MPT_EINVAL, "transfer has a NULL pointer");
  const int ks = range_kind(c, x.src, x.bytes), kd = range_kind(c, x.dst, x.bytes);
  const int want_s = x.dir == MPT_H2D ? 1 : 0, want_d = x.dir == MPT_D2H ? 1 : 0;
  if ((ks == 2 ? 1 : ks) != want_s || (kd == 2 ? 1 : kd) != want_d)
    return fail(MPT_EINVAL, "transfer pointers do not match direction %u", x.dir);
  *src_kind = ks;
  *dst_kind = kd;
  return MPT_OK;
}

}  // namespace mpt

struct mpt_batch_s {
  mpt_ctx_t ctx;
  uint32_t slot;
  uint32_t epoch;
  size_t n;
  uint64_t submit_ns;
};

uint64_t mpt::batch_cta_spread_ns(mpt_batch_t b) {
  const volatile unsigned long long* t = b->ctx->slots[b->slot].h_stamps;
  const uint64_t first = t[0], last = t[1];
  return last >= first ? last - first : 0;
}

float mpt::batch_gpu_ms(mpt_batch_t b) {
  const mpt::BatchSlot& s = b->ctx->slots[b->slot];
  float ms = -1.0f;
  if (!s.timed || cudaEventElapsedTime(&ms, s.t0_ev, s.t1_ev) != cudaSuccess) return -1.0f;
  return ms;
}

using namespace mpt;

extern "C" {

mpt_status mpt_batch_configure(mpt_ctx_t c, uint32_t slots, uint32_t max_xfers, uint32_t ctas, uint32_t tile_bytes) {
  if (!c) return fail(MPT_EINVAL, "mpt_batch_configure: NULL context");
  for (auto& s : c->slots)
    if (s.held) return fail(MPT_EAGAIN, "mpt_batch_configure: a batch is still held");
  if (slots > 64 || max_xfers > (1u << 20) || (tile_bytes && (tile_bytes < 4096 || tile_bytes % 16)))
    return fail(MPT_EINVAL, "mpt_batch_configure: slots <= 64, max_xfers <= 2^20, tile >= 4096 and a multiple of 16");
  CUDA_TRY(cudaSetDevice(c->device));
  CUDA_TRY(cudaDeviceSynchronize());
  batch_teardown(c);
  c->batch_slots = slots;
  c->batch_max_xfers = max_xfers;
  c->batch_ctas = ctas;
  c->batch_tile = tile_bytes;
  return batch_setup(c);
}

mpt_status mpt_batch_configure_dma(mpt_ctx_t c, uint32_t lanes, uint32_t items_per_lane, uint64_t min_bytes) {
  if (!c) return fail(MPT_EINVAL, "mpt_batch_configure_dma: NULL context");
  for (auto& s : c->slots)
    if (s.held) return fail(MPT_EAGAIN, "mpt_batch_configure_dma: a batch is still held");
  if (lanes > 8 || items_per_lane > 64 || (lanes && (items_per_lane == 0 || min_bytes < 16)))
    return fail(MPT_EINVAL, "mpt_batch_configure_dma: lanes <= 8, 1 <= items <= 64, min_bytes >= 16");
  CUDA_TRY(cudaSetDevice(c->device));
  CUDA_TRY(cudaDeviceSynchronize());
  batch_teardown(c);
  c->batch_dma_lanes = lanes;
  c->batch_dma_items = lanes ? items_per_lane : 0;
  c->batch_dma_min = lanes ? min_bytes : 0;
  c->batch_dma_set = true;
  return batch_setup(c);
}

mpt_status mpt_batch_tune(mpt_ctx_t c, const mpt_xfer* xfers, size_t n, uint32_t objective, uint32_t reps, void* stream,
                          mpt_batch_tuning* out) {
  if (!c || !xfers || n == 0) return fail(MPT_EINVAL, "mpt_batch_tune: NULL or empty batch");
  if (objective > MPT_BATCH_TUNE_P99) return fail(MPT_EINVAL, "mpt_batch_tune: unknown objective %u", objective);
  for (auto& s : c->slots)
    if (s.held) return fail(MPT_EAGAIN, "mpt_batch_tune: a batch is still held");
  if (reps == 0) reps = 3;
  const uint32_t sms = (uint32_t)c->sms;
  struct Setting {
    uint32_t ctas, tile, lanes, items;
    uint64_t min;
  };
  std::vector<Setting> cand;
  for (uint32_t k : {1u, 2u, 3u})
    for (uint32_t tile : {64u << 10, 128u << 10, 256u << 10, 512u << 10, 1024u << 10})
      for (uint32_t lanes : {0u, 2u}) cand.push_back(Setting{k * sms, tile, lanes, lanes ? 8u : 0u, lanes ? 4ull << 20 : 0});
  const uint32_t keep_slots = c->batch_slots, keep_max = c->batch_max_xfers;
  std::vector<uint64_t> t(n);
  const cudaStream_t cs = static_cast<cudaStream_t>(stream);
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  CUDA_TRY(cudaEventCreate(&e0));
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return fail(MPT_ECUDA, "mpt_batch_tune: events");
  }
  struct Events {
    cudaEvent_t a, b;
    ~Events() {
      cudaEventDestroy(a);
      cudaEventDestroy(b);
    }
  } ev{e0, e1};
  mpt_batch_tuning best{};
  double best_score = 1e300;
  bool have = false;
  for (const Setting& k : cand) {
    c->batch_dma_lanes = k.lanes;
    c->batch_dma_items = k.items;
    c->batch_dma_min = k.min;
    c->batch_dma_set = true;
    mpt_status st = mpt_batch_configure(c, keep_slots, keep_max, k.ctas, k.tile);
    if (st != MPT_OK) return st;
    std::vector<double> times, p99s;
    for (uint32_t r = 0; r < reps + 1; ++r) {
      mpt_batch_t b = nullptr;
      CUDA_TRY(cudaEventRecord(e0, cs));
      st = mpt_batch_submit(c, xfers, n, stream, &b);
      if (st != MPT_OK) return st;
      if (cudaEventRecord(e1, cs) != cudaSuccess) st = fail(MPT_ECUDA, "mpt_batch_tune: event");
      if (st == MPT_OK) st = mpt_batch_wait(b, 600ull * 1000000000ull);
      if (st == MPT_OK) st = mpt_batch_times(b, t.data());
      mpt_batch_release(b);
      if (st != MPT_OK) return st;
      float ms = 0;
      CUDA_TRY(cudaEventSynchronize(e1));
      CUDA_TRY(cudaEventElapsedTime(&ms, e0, e1));
      if (r == 0) continue;  // the first run warms up
      std::vector<uint64_t> sorted(t);
      std::sort(sorted.begin(), sorted.end());
      const size_t i99 = std::min(n - 1, (size_t)std::ceil(0.99 * (double)n) - (n > 0 ? 1 : 0));
      p99s.push_back((double)sorted[i99] / 1e3);
      times.push_back((double)ms * 1e3);
    }
    std::sort(times.begin(), times.end());
    std::sort(p99s.begin(), p99s.end());
    const double bt = times[times.size() / 2], p99 = p99s[p99s.size() / 2];
    const double score = objective == MPT_BATCH_TUNE_P99 ? p99 : bt;
    if (!have || score < best_score) {
      have = true;
      best_score = score;
      best = mpt_batch_tuning{k.ctas, k.tile, k.lanes, k.items, k.min, bt, p99, 0, 0};
    }
  }
  best.candidates = (uint32_t)cand.size();
  c->batch_dma_lanes = best.dma_lanes;
  c->batch_dma_items = best.dma_items;
  c->batch_dma_min = best.dma_min_bytes;
  c->batch_dma_set = true;
  mpt_status st = mpt_batch_configure(c, keep_slots, keep_max, best.ctas, best.tile_bytes);
  if (st != MPT_OK) return st;
  if (out) *out = best;
  return MPT_OK;
}

mpt_status mpt_batch_register(mpt_ctx_t c, const void* base, uint64_t bytes) {
  if (!c || !base || bytes == 0) return fail(MPT_EINVAL, "mpt_batch_register: bad argument");
  CUDA_TRY(cudaSetDevice(c->device));
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, base) != cudaSuccess) {
    cudaGetLastError();
    return fail(MPT_EINVAL, "mpt_batch_register: %p is not CUDA memory", base);
  }
  int kind;
  if ((at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged) && at.device == c->device) kind = 0;
  else if (at.type == cudaMemoryTypeHost) kind = 1;
  else return fail(MPT_EINVAL, "mpt_batch_register: %p is neither this GPU's memory nor page-locked host memory", base);
  c->arenas.push_back(Arena{(uint64_t)(uintptr_t)base, bytes, kind});
  return MPT_OK;
}

mpt_status mpt_batch_submit(mpt_ctx_t c, const mpt_xfer* xfers, size_t n, void* stream, mpt_batch_t* out) {
  if (!c || !out || (n > 0 && !xfers)) return fail(MPT_EINVAL, "mpt_batch_submit: NULL argument");
  *out = nullptr;
  CUDA_TRY(cudaSetDevice(c->device));
  mpt_status st = batch_setup(c);
  if (st != MPT_OK) return st;
  if (n == 0 || n > c->slots[0].max_xfers)
    return fail(MPT_EINVAL, "mpt_batch_submit: %zu transfers (1..%u per batch)", n, c->slots[0].max_xfers);
  uint32_t si = 0;
  while (si < c->slots.size() && c->slots[si].held) ++si;
  if (si == c->slots.size()) return fail(MPT_EAGAIN, "mpt_batch_submit: every batch slot is held");
  BatchSlot& s = c->slots[si];
  // validate: direction, memory kinds, and non-overlapping destinations (Sec. 4.5: each
  // transfer owns its destination region)
  // scratch owned by the context (one thread per context): no allocation per batch
  std::vector<std::pair<uint64_t, uint64_t>>& spans = c->batch_spans;
  spans.clear();
  std::vector<uint32_t>& dma_cand = c->batch_cand;  // entries large enough for a copy-engine lane
  dma_cand.clear();
  for (size_t i = 0; i < n; ++i) {
    const mpt_xfer& x = xfers[i];
    int ks, kd;
    if (batch_check_xfer(c, x, &ks, &kd) != MPT_OK)
      return fail(MPT_EINVAL, "mpt_batch_submit: transfer %zu: %s", i, mpt_last_error());
    if (x.bytes == 0) continue;
    spans.emplace_back((uint64_t)(uintptr_t)x.dst, (uint64_t)(uintptr_t)x.dst + x.bytes);
    if (s.dma_lanes && x.bytes >= c->batch_dma_min && ks != 2 && kd != 2) dma_cand.push_back((uint32_t)i);
  }
  std::sort(spans.begin(), spans.end());
  for (size_t i = 1; i < spans.size(); ++i)
    if (spans[i].first < spans[i - 1].second)
      return fail(MPT_EINVAL, "mpt_batch_submit: destination regions overlap");
  // no source may overlap a destination: the batch's transfers run at the same time
  for (size_t i = 0; i < n; ++i) {
    const mpt_xfer& x = xfers[i];
    if (x.bytes == 0) continue;
    const uint64_t a = (uint64_t)(uintptr_t)x.src, b = a + x.bytes;
    // spans are sorted and disjoint: only the last one starting at or before a, and the
    // first one starting after a, can reach into [a, b)
    auto it = std::upper_bound(spans.begin(), spans.end(), std::pair<uint64_t, uint64_t>(a, UINT64_MAX));
    if ((it != spans.begin() && std::prev(it)->second > a) || (it != spans.end() && it->first < b))
      return fail(MPT_EINVAL, "mpt_batch_submit: the source of transfer %zu overlaps a destination of the batch", i);
  }
  // the slot's previous batch must be done reading its table
  CUDA_TRY(cudaEventSynchronize(s.done_ev));
  s.epoch++;
  if (s.epoch == 0) s.epoch = 1;
  BatchHeader* h = reinterpret_cast<BatchHeader*>(s.h_table);
  BatchDesc* d = reinterpret_cast<BatchDesc*>(s.h_table + s.desc_off);
  uint32_t* order = reinterpret_cast<uint32_t*>(d + n);
  // DMA lanes: largest eligible entries first, each to the least-loaded lane of its
  // direction with a free item (longest-processing-time order); the rest stay with the kernel
  const uint32_t ndma = kDmaDirs * s.dma_lanes * s.dma_items;
  std::vector<uint8_t>& to_dma = c->batch_to_dma;
  to_dma.assign(n, 0);
  for (uint32_t k = 0; k < ndma; ++k) s.h_dma_map[k] = ~0u;
  if (!dma_cand.empty()) {
    std::sort(dma_cand.begin(), dma_cand.end(),
              [&](uint32_t a, uint32_t b) { return xfers[a].bytes > xfers[b].bytes || (xfers[a].bytes == xfers[b].bytes && a < b); });
    std::vector<uint64_t> load(kDmaDirs * s.dma_lanes, 0);
    std::vector<uint32_t> used(kDmaDirs * s.dma_lanes, 0);
    for (uint32_t i : dma_cand) {
      const uint32_t dir = xfers[i].dir;
      int best = -1;
      for (uint32_t l = 0; l < s.dma_lanes; ++l) {
        const uint32_t li = dir * s.dma_lanes + l;
        if (used[li] < s.dma_items && (best < 0 || load[li] < load[(uint32_t)best])) best = (int)li;
      }
      if (best < 0) continue;
      s.h_dma_map[(uint32_t)best * s.dma_items + used[(uint32_t)best]] = i;
      used[(uint32_t)best]++;
      load[(uint32_t)best] += xfers[i].bytes;
      to_dma[i] = 1;
    }
  }
  // tiles numbered within two classes, link (a host side) and device, each descriptor's
  // tiles contiguous in its class; order lists the descriptors with tiles, link class first
  bool any_shift = false;
  uint64_t kernel_bytes = 0;
  for (size_t i = 0; i < n; ++i) {
    if (to_dma[i]) continue;
    const mpt_xfer& x = xfers[i];
    any_shift |= (((uintptr_t)x.src ^ (uintptr_t)x.dst) & 15) != 0 && x.bytes >= 16;
    kernel_bytes += x.bytes;
  }
  const int gi = any_shift ? 1 : 0;
  const uint32_t ctas = c->batch_ctas ? c->batch_ctas : 3u * (uint32_t)c->sms;
  const uint32_t grid = gi == 0 ? ctas : std::min<uint32_t>(ctas, 2u * (uint32_t)c->sms);  // as slot_init
  // tile size: the configured one, unless the batch is too small to give every CTA a full
  // tile; then the power of two at or above the kernel's bytes per CTA, at least 32 KiB (a
  // CTA moves 32 KiB per round of loads), so that a short batch spreads over the grid
  // instead of queueing its bytes behind a few CTAs
  uint64_t tile = c->batch_tile;
  {
    const uint64_t per_cta = (kernel_bytes + grid - 1) / grid;
    uint64_t t = kMinAdaptiveTile;
    while (t < per_cta && t < tile) t <<= 1;  // bounded by the configured tile: no overflow
    tile = std::min<uint64_t>(tile, t);
  }
  uint64_t tiles[2] = {0, 0};  // [0] link, [1] device
  uint32_t n_link = 0, n_dev = 0;
  for (size_t i = 0; i < n; ++i) {
    const mpt_xfer& x = xfers[i];
    const uint32_t fl = (x.dir == MPT_D2H ? kDescHostDst : 0u) | (x.dir != MPT_D2D ? kDescHostSide : 0u) |
                        (to_dma[i] ? kDescDma : 0u);
    const uint64_t t = to_dma[i] ? 0 : std::max<uint64_t>(1, (x.bytes + tile - 1) / tile);
    // one class for everything when the split is off
    const int cls = (c->batch_split && x.dir == MPT_D2D) ? 1 : 0;
    d[i] = BatchDesc{(uint64_t)(uintptr_t)x.src, (uint64_t)(uintptr_t)x.dst, x.bytes, (uint32_t)tiles[cls],
                     (uint32_t)t, fl, 0u};
    tiles[cls] += t;
    if (t) (cls ? n_dev : n_link)++;
  }
  if (tiles[0] + tiles[1] >= (1ull << 32))
    return fail(MPT_EINVAL, "mpt_batch_submit: batch too large for 32-bit tile indices");
  {
    uint32_t li = 0, di = n_link;
    for (size_t i = 0; i < n; ++i) {
      if (!d[i].ntiles) continue;
      const bool dev = c->batch_split && xfers[i].dir == MPT_D2D;
      order[dev ? di++ : li++] = (uint32_t)i;
    }
  }
  uint32_t link_ctas = grid;  // split off: one class, every CTA on it
  if (c->batch_split && tiles[0])
    link_ctas = std::min(grid, c->batch_link_ctas ? c->batch_link_ctas : kDefaultLinkCtas);
  *h = BatchHeader{(uint32_t)n, (uint32_t)(tiles[0] + tiles[1]), (uint32_t)tile, s.epoch,
                   (uint32_t)tiles[0], n_link, n_link + n_dev, link_ctas};
  for (uint32_t k = 0; k < ndma; ++k) {  // retarget used lane items, switch the rest off
    const uint32_t i = s.h_dma_map[k];
    const uint8_t want = i != ~0u;
    if (want)
      CUDA_TRY(cudaGraphExecMemcpyNodeSetParams1D(s.exec[gi], s.dma_cp[gi][k], xfers[i].dst, xfers[i].src,
                                                  xfers[i].bytes, cudaMemcpyDefault));
    if (want != s.dma_on[gi][k]) {
      CUDA_TRY(cudaGraphNodeSetEnabled(s.exec[gi], s.dma_cp[gi][k], want));
      CUDA_TRY(cudaGraphNodeSetEnabled(s.exec[gi], s.dma_fin[gi][k], want));
      s.dma_on[gi][k] = want;
    }
  }
  // copy the used part of the table, rounded up to a power of two (at least 256 bytes) so
  // that batches of similar length reuse the node's size without an update
  {
    const size_t used = s.desc_off + n * (sizeof(BatchDesc) + sizeof(uint32_t));
    size_t want = 256;
    while (want < used) want <<= 1;
    want = std::min(want, s.table_bytes);
    if (want != s.table_cp_bytes[gi]) {
      CUDA_TRY(cudaGraphExecMemcpyNodeSetParams1D(s.exec[gi], s.table_cp[gi], s.d_table, s.h_table, want,
                                                  cudaMemcpyHostToDevice));
      s.table_cp_bytes[gi] = want;
    }
  }
  const cudaStream_t cs = static_cast<cudaStream_t>(stream);
  const bool timed = c->batch_timing;
  if (timed && !s.t0_ev) {
    CUDA_TRY(cudaEventCreate(&s.t0_ev));
    CUDA_TRY(cudaEventCreate(&s.t1_ev));
  }
  if (timed) CUDA_TRY(cudaEventRecord(s.t0_ev, cs));
  CUDA_TRY(cudaGraphLaunch(s.exec[gi], cs));
  if (timed) CUDA_TRY(cudaEventRecord(s.t1_ev, cs));
  CUDA_TRY(cudaEventRecord(s.done_ev, cs));
  s.timed = timed;
  s.held = true;
  s.n = n;
  mpt_batch_s* b = new mpt_batch_s{c, si, s.epoch, n, host_ns()};
  *out = b;
  return MPT_OK;
}

mpt_status mpt_batch_poll(mpt_batch_t b, size_t* done, uint8_t* flags) {
  if (!b || !done) return fail(MPT_EINVAL, "mpt_batch_poll: NULL argument");
  const BatchSlot& s = b->ctx->slots[b->slot];
  volatile const uint32_t* f = s.h_flags;
  size_t k = 0;
  for (size_t i = 0; i < b->n; ++i) {
    const bool fin = f[i] == b->epoch;
    k += fin;
    if (flags) flags[i] = fin ? 1 : 0;
  }
  *done = k;
  return MPT_OK;
}

mpt_status mpt_batch_wait(mpt_batch_t b, uint64_t timeout_ns) {
  if (!b) return fail(MPT_EINVAL, "mpt_batch_wait: NULL batch");
  const BatchSlot& s = b->ctx->slots[b->slot];
  const uint64_t t0 = host_ns();
  while (true) {
    const cudaError_t e = cudaEventQuery(s.done_ev);
    if (e == cudaSuccess) break;
    if (e != cudaErrorNotReady) return fail(MPT_ECUDA, "mpt_batch_wait: %s", cudaGetErrorString(e));
    if (host_ns() - t0 >= timeout_ns) return fail(MPT_ETIMEDOUT, "mpt_batch_wait: batch still running");
    std::this_thread::yield();
  }
  return MPT_OK;
}

mpt_status mpt_batch_times(mpt_batch_t b, uint64_t* out_ns) {
  if (!b || !out_ns) return fail(MPT_EINVAL, "mpt_batch_times: NULL argument");
  const BatchSlot& s = b->ctx->slots[b->slot];
  CUDA_TRY(cudaEventSynchronize(s.done_ev));
  std::vector<unsigned long long> t(b->n + 1);
  unsigned long long start_inv = 0;
  CUDA_TRY(cudaMemcpy(t.data(), s.d_times, b->n * sizeof(unsigned long long), cudaMemcpyDeviceToHost));
  CUDA_TRY(cudaMemcpy(&start_inv, s.args.start_out, sizeof start_inv, cudaMemcpyDeviceToHost));
  const unsigned long long start = ~start_inv;
  for (size_t i = 0; i < b->n; ++i) out_ns[i] = t[i] >= start ? t[i] - start : 0;
  return MPT_OK;
}

mpt_status mpt_batch_watch(mpt_batch_t b, uint64_t t0_ns, uint64_t* out_ns, uint64_t timeout_ns) {
  if (!b || !out_ns) return fail(MPT_EINVAL, "mpt_batch_watch: NULL argument");
  const BatchSlot& s = b->ctx->slots[b->slot];
  volatile const uint32_t* f = s.h_flags;
  const size_t n = b->n;
  std::vector<uint8_t> seen(n, 0);
  size_t left = n, lo = 0;
  const uint64_t start = host_ns();
  bool finished = false;  // the batch's completion event has fired: one last scan decides
  while (left) {
    const uint64_t now = host_ns();
    for (size_t i = lo; i < n; ++i) {
      if (!seen[i] && f[i] == b->epoch) {
        seen[i] = 1;
        out_ns[i] = now >= t0_ns ? now - t0_ns : 0;
        --left;
      }
    }
    while (lo < n && seen[lo]) ++lo;
    if (!left) break;
    if (finished) return fail(MPT_ETIMEDOUT, "mpt_batch_watch: the batch ended with %zu transfers unflagged", left);
    const cudaError_t e = cudaEventQuery(s.done_ev);
    if (e == cudaSuccess) {
      finished = true;
      continue;
    }
    if (e != cudaErrorNotReady) return fail(MPT_ECUDA, "mpt_batch_watch: %s", cudaGetErrorString(e));
    if (now - start >= timeout_ns) return fail(MPT_ETIMEDOUT, "mpt_batch_watch: batch still running");
  }
  return MPT_OK;
}

mpt_status mpt_copy_each(mpt_ctx_t c, const mpt_xfer* xfers, size_t n, void* const* streams, uint64_t* out_ns,
                         uint64_t timeout_ns) {
  const uint64_t t0 = host_ns();
  if (!c || (n && (!xfers || !streams))) return fail(MPT_EINVAL, "mpt_copy_each: NULL argument");
  for (size_t i = 0; i < n; ++i) {
    const mpt_xfer& x = xfers[i];
    if (x.dir > MPT_D2H) return fail(MPT_EINVAL, "mpt_copy_each: transfer %zu has direction %u", i, x.dir);
    if (x.bytes && (!x.src || !x.dst)) return fail(MPT_EINVAL, "mpt_copy_each: transfer %zu has a NULL pointer", i);
  }
  CUDA_TRY(cudaSetDevice(c->device));
  if (out_ns) {
    while (c->each_ev.size() < n) {
      cudaEvent_t e;
      CUDA_TRY(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
      c->each_ev.push_back(e);
    }
  }
  std::vector<size_t> order[3];  // per direction, transfer indices in issue order
  for (size_t i = 0; i < n; ++i) {
    const mpt_xfer& x = xfers[i];
    cudaStream_t s = static_cast<cudaStream_t>(streams[x.dir]);
    if (x.bytes) CUDA_TRY(cudaMemcpyAsync(x.dst, x.src, x.bytes, cudaMemcpyDefault, s));
    if (out_ns) {
      CUDA_TRY(cudaEventRecord(c->each_ev[i], s));
      order[x.dir].push_back(i);
    }
  }
  if (!out_ns) return MPT_OK;
  // one stream's copies finish in issue order: poll only the oldest unfinished one of each
  size_t head[3] = {0, 0, 0}, left = n;
  while (left) {
    for (int d = 0; d < 3; ++d) {
      while (head[d] < order[d].size()) {
        const size_t i = order[d][head[d]];
        const cudaError_t e = cudaEventQuery(c->each_ev[i]);
        if (e == cudaErrorNotReady) break;
        if (e != cudaSuccess) return fail(MPT_ECUDA, "mpt_copy_each: %s", cudaGetErrorString(e));
        out_ns[i] = host_ns() - t0;
        ++head[d];
        --left;
      }
    }
    if (left && host_ns() - t0 >= timeout_ns) return fail(MPT_ETIMEDOUT, "mpt_copy_each: copies still running");
  }
  return MPT_OK;
}

mpt_status mpt_batch_release(mpt_batch_t b) {
  if (!b) return MPT_OK;
  BatchSlot& s = b->ctx->slots[b->slot];
  if (s.held && s.epoch == b->epoch) s.held = false;
  delete b;
  return MPT_OK;
}

}  // extern "C"
